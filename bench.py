"""Benchmark: body-steps/s of the ReLCP time step on the compacting-suspension
workload (32,768 ellipsoids, semi-axes U[0.4, 1.0], volume fraction 0.1 ->
0.55 by affine compaction over 2,000 steps of dt = 5e-3, overdamped,
eps_NCP = 1e-3 x smallest semi-axis), mixed-precision path, with the plain
FP64 GPU path timed on the same steps for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  A "step" is one full time step of Algorithm 1
(broad phase, SNSD, LCP solves, trial re-evaluations, augmentations).
Timing: W untimed warm-up steps on a separate context, then K steps from the
initial state, each bracketed by CUDA events on the library's stream, with a
256 MiB L2 flush between steps (outside the events); barrier +
synchronize around the timed region; max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "compacting ellipsoid suspension, 32768 bodies, phi 0.1->0.55 over 2000 steps, dt 5e-3, overdamped"
METRIC = "body-steps/sec at 32k ellipsoids, mixed+learned vs plain FP64 GPU, equal overlap tol"
UNIT = "body-steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def build_scene(n, seed=1, steps=2000):
    from paper_2506_14097_gb300 import scenes

    return scenes.suspension_scene(seed=seed, n=n, phi=0.1, phi_final=0.55, steps=steps, dt=5e-3)


EXTRA_FLAGS = 0


def make_cfg(R, sc, precision, guess, timing="lcp"):
    """timing: None, "lcp" (CUDA events around the LCP launches only, for the
    roofline; what the timed runs use) or "phases" (events between all phases,
    ~2 us of host time each: a separate breakdown run)."""
    amin = float(sc.axes.min())
    tf = {None: 0, False: 0, "lcp": R.RELCP_FLAG_LCP_TIMING, "phases": R.RELCP_FLAG_PHASE_TIMING}[timing]
    return R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=precision, guess=guess, dt=sc.dt,
                         eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin,
                         strain_rate=sc.meta["strain_rate"], length_scale=amin, lcp_max_iter=20000,
                         flags=tf | EXTRA_FLAGS)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_batched(R, torch, n_scenes, steps=100, reps=3, rank=0, world=1, dist=None):
    """The batched-scene workload: n_scenes independent lattice scenes (bodies
    log-uniform in [2, 512], own seed and dt), `steps` steps of every scene in
    ONE persistent launch, block size from the autotuner.  Each timed launch
    starts from the initial state (reloaded untimed); median of `reps`.  With
    several ranks each takes a contiguous, cost-balanced range of scenes (no
    collective on the data path); the time is the maximum over ranks."""
    from paper_2506_14097_gb300 import scenes
    from paper_2506_14097_gb300.sharding import shard_scenes

    all_scs = scenes.batched_scenes(n_scenes=n_scenes)
    a, b_ = shard_scenes([sc.n for sc in all_scs], world)[rank]
    total_bodies = sum(sc.n for sc in all_scs)
    scs = all_scs[a:b_]
    offsets, x, q, axes, vel, params = scenes.pack_scenes(scs)
    b = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    threads = b.autotune(None)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, status = [], set()
    for k in range(reps + 1):
        b.set_scenes(offsets, x, q, axes, params, vel=vel)
        torch.cuda.synchronize()
        ev0.record()
        st = b.step(steps, allow=(R.RELCP_ERR_NOT_CONVERGED, R.RELCP_ERR_RECURSION_LIMIT))
        ev1.record()
        torch.cuda.synchronize()
        if k > 0:  # the first launch is the warm-up
            times.append(ev0.elapsed_time(ev1))
            status.add(R.STATUS_NAMES[st])
    ss = b.scene_stats()
    b.close()
    ms = float(np.median(times))
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    nb = total_bodies
    return {"workload": f"{n_scenes} independent periodic lattice scenes, bodies log-uniform in [2, 512] "
                        f"({nb} in all), dt ~ U[1e-3, 1e-2], inertial, {steps} steps in one persistent launch",
            "value": nb * steps / (ms / 1e3), "unit": UNIT, "ms_per_launch": ms, "steps_per_launch": steps,
            "scaling": "strong (scenes sharded by cost-balanced contiguous ranges)" if world > 1 else None,
            "threads_per_cta": threads, "status": sorted(status), "depth_max": max(s.depth_max for s in ss),
            "lcp_iters_total": int(sum(s.lcp_iters for s in ss)),
            "max_overlap_within_eps": bool(all(s.max_overlap <= params[i, 4] for i, s in enumerate(ss))),
            "timing": "CUDA events around the launch (graph replay); median of %d" % reps}


def new_sim(R, sc, precision, guess, timing, stream, mlp_params):
    sim = R.Simulation(make_cfg(R, sc, precision, guess, timing=timing), stream)
    if guess == R.RELCP_GUESS_MLP:
        R.relcp_load_mlp(sim.ctx, mlp_params)
    return sim


def run_gpu_arm(R, torch, sc, precision, guess, steps, warmup, flush, stream, nvtx_from=None, mlp_params=None,
                timing="lcp", nvtx_to=None):
    """W warm-up steps on one context, then `steps` timed steps from the initial
    state on a fresh context.  Returns per-step times and accumulated stats."""
    x, q, axes = (np.ascontiguousarray(a) for a in (sc.x, sc.q, sc.axes))
    if warmup > 0:
        sim = new_sim(R, sc, precision, guess, None, stream.cuda_stream, mlp_params)
        sim.set_bodies(x, q, axes)
        for _ in range(warmup):
            sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        sim.close()
    sim = new_sim(R, sc, precision, guess, timing, stream.cuda_stream, mlp_params)
    sim.set_bodies(x, q, axes)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    acc = dict(lcp_ms=0.0, lcp_bytes=0.0, lcp_launches=0, snsd_ms=0.0, snsd_evals=0, snsd_launches=0, depth_max=0,
               depth_sum=0, rows_max=0, pairs_max=0, lcp_iters=0, max_overlap=0.0, not_converged=0, status=set(),
               ms_broadphase=0.0, ms_lcp_phase=0.0, ms_other=0.0, ms_step_events=0.0, rebuilds=0)
    launches0 = R.relcp_kernel_launches()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            if nvtx_from is not None and k == nvtx_from:
                torch.cuda.nvtx.range_push("relcp_profile")
            if nvtx_from is not None and nvtx_to is not None and k == nvtx_to:
                torch.cuda.nvtx.range_pop()
            ev[k][0].record(stream)
            st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
            ev[k][1].record(stream)
            s = sim.stats()
            acc["status"].add(R.STATUS_NAMES[st])
            acc["not_converged"] += int(st == R.RELCP_ERR_NOT_CONVERGED)
            acc["lcp_ms"] += s.ms_lcp_kernel
            acc["lcp_bytes"] += s.lcp_alg_bytes
            acc["lcp_launches"] += s.lcp_launches
            acc["snsd_ms"] += s.ms_snsd_kernel
            acc["snsd_evals"] += s.snsd_evals
            acc["snsd_launches"] += s.snsd_launches
            acc["depth_max"] = max(acc["depth_max"], s.depth)
            acc["depth_sum"] += s.depth
            acc["rows_max"] = max(acc["rows_max"], s.n_rows)
            acc["pairs_max"] = max(acc["pairs_max"], s.n_pairs)
            acc["lcp_iters"] += s.lcp_iters_total
            acc["max_overlap"] = max(acc["max_overlap"], s.max_overlap)
            acc["ms_broadphase"] += s.ms_broadphase
            acc["ms_lcp_phase"] += s.ms_lcp
            acc["ms_other"] += s.ms_augment
            acc["ms_step_events"] += s.ms_total
            acc["rebuilds"] += s.pair_list_rebuilt
            acc["guess_steps"] = acc.get("guess_steps", 0) + s.guess_used
            acc["newton_c0"] = acc.get("newton_c0", 0) + s.newton_iters_c0
            acc["pairs_total"] = acc.get("pairs_total", 0) + s.n_pairs
    torch.cuda.synchronize()
    if nvtx_from is not None and nvtx_from < steps and (nvtx_to is None or nvtx_to >= steps):
        torch.cuda.nvtx.range_pop()
    acc["launches"] = R.relcp_kernel_launches() - launches0
    times = [a.elapsed_time(b) for a, b in ev]
    acc["box_final"] = list(R.relcp_get_box(sim.ctx))
    sim.close()
    acc["status"] = sorted(acc["status"])
    return times, acc


def run_e2e(R, torch, sc, precision, guess, steps, mlp_params=None):
    """The same steps through the public C ABI with host buffers: every step
    copies the body state in (set_bodies: x, q, semi-axes) and the result out
    (get_bodies: x, q and the step velocity).  The workload has no background
    velocity or external force, so none is passed in."""
    n = sc.n
    # copies: relcp_get_bodies writes each step's result into x and q, and the
    # scene's own arrays must keep the initial state for the runs after this one
    x, q, axes = (np.array(a, dtype=np.float64, order="C", copy=True) for a in (sc.x, sc.q, sc.axes))
    u = np.zeros((n, 6))
    cfg = make_cfg(R, sc, precision, guess, timing=None)
    sim = R.Simulation(cfg)
    if guess == R.RELCP_GUESS_MLP:
        R.relcp_load_mlp(sim.ctx, mlp_params)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    box = np.asarray(sc.box, dtype=np.float64)
    for _ in range(steps):
        for k in range(3):
            cfg.box[k] = box[k]
        R.relcp_set_config(sim.ctx, cfg)
        sim.set_bodies(x, q, axes)
        sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        R.relcp_get_bodies(sim.ctx, x, q, u)
        box = R.relcp_get_box(sim.ctx)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sim.close()
    h2d = n * (3 + 4 + 3) * 8
    d2h = n * (3 + 4 + 6) * 8
    return dt, h2d, d2h


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def _oracle_worker(n, steps, budget_s, out_q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import relcp_oracle as O

    sc = build_scene(n)
    amin = float(sc.axes.min())
    cfg = O.Config(dynamics=O.OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin,
                   strain_rate=sc.meta["strain_rate"])
    x, q, box = sc.x, sc.q, np.asarray(sc.box)
    vol = sc.meta["volume"]
    done = 0
    t0 = time.perf_counter()
    phi0 = vol / np.prod(box)
    while done < steps:
        r = O.step(O.Config(**{**cfg.__dict__, "box": tuple(box)}), x, q, sc.axes)
        x, q, box = r.x, r.q, r.box
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    out_q.put({"bodies": n, "steps": done, "seconds": el, "phi_start": phi0, "phi_end": vol / np.prod(box)})


def oracle_rate(n, steps, budget_s):
    """The oracle as it stands, single-threaded (BLAS threads pinned to 1), in
    a spawned process (no GPU context)."""
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        qq = ctx.Queue()
        p = ctx.Process(target=_oracle_worker, args=(n, steps, budget_s, qq))
        p.start()
        res = qq.get()
        p.join()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res["value"] = res["bodies"] * res["steps"] / res["seconds"]
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    # warm-up: a few oracle steps (compiles/loads the C core)
    oracle_rate(1024, max(1, args.warmup), 60.0)
    res = oracle_rate(1024, args.steps, args.ref_budget)
    sample = (f"first {res['steps']} steps (phi {res['phi_start']:.4f}->{res['phi_end']:.4f}) of the 1,024-body "
              f"version of the workload (same schedule), single-threaded FP64 oracle, {res['seconds']:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": res["steps"], "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_bodies": 1024},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bodies", type=int, default=32768)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=150.0)
    ap.add_argument("--jacobi", type=int, default=0, help="1: Jacobi-scaled projected-gradient steps")
    ap.add_argument("--cold", action="store_true", help="cold SNSD start only (no learned guess)")
    ap.add_argument("--phase-breakdown", type=int, default=1, help="1: extra run with per-phase events")
    ap.add_argument("--batched-scenes", type=int, default=2048,
                    help="scenes of the batched-scene measurement (0 skips it)")
    ap.add_argument("--nvtx-from", type=int, default=None,
                    help="profiling aid: wrap timed steps >= this index in the NVTX range relcp_profile")
    ap.add_argument("--nvtx-to", type=int, default=None, help="profiling aid: end of that range (exclusive)")
    ap.add_argument("--step-times", default=None,
                    help="write the headline run's per-step CUDA-event times (ms, one per line) to this file")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2506_14097_gb300 import relcp as R

    R.load()
    global EXTRA_FLAGS
    if args.jacobi:
        EXTRA_FLAGS |= R.RELCP_FLAG_JACOBI
    sc = build_scene(args.bodies)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    precision = R.RELCP_MIXED
    # learned SNSD guess: trained before the timed region on pairs the method
    # generates in a separate, smaller compaction (another seed)
    mlp_params, learned_info = None, None
    guess = R.RELCP_GUESS_COLD
    if not args.cold:
        from paper_2506_14097_gb300 import learned

        t_tr = time.perf_counter()
        feat, targ = learned.harvest_compaction(n=4096, seed=11, steps=300, every=10)
        mlp_params, losses = learned.train(feat, targ, epochs=20, batch=4096, lr=2e-3, seed=0)
        torch.cuda.synchronize()
        learned_info = {"train_samples": int(feat.shape[0]), "epochs": 20, "loss_first": losses[0],
                        "loss_last": losses[-1], "train_s": time.perf_counter() - t_tr,
                        "harvest": "4,096-body compaction, seed 11, every 10th of 300 steps, FP64 SNSD targets"}
        guess = R.RELCP_GUESS_MLP
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    times, acc = run_gpu_arm(R, torch, sc, precision, guess, args.steps, args.warmup, flush, stream, args.nvtx_from,
                             mlp_params, nvtx_to=args.nvtx_to)
    if args.step_times and rank == 0:
        with open(args.step_times, "w") as f:
            f.write("".join("%.6f\n" % t for t in times))
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = float(sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * sc.n * args.steps / (total_ms / 1e3)

    cold = None
    if guess == R.RELCP_GUESS_MLP and not args.no_fp64:
        times_c, acc_c = run_gpu_arm(R, torch, sc, precision, R.RELCP_GUESS_COLD, args.steps, args.warmup, flush,
                                     stream)
        tc = float(sum(times_c))
        cold = {"value": sc.n * args.steps / (tc / 1e3), "unit": UNIT, "ms_per_step": tc / args.steps,
                "newton_iters_per_pair_c0": acc_c.get("newton_c0", 0) / max(acc_c.get("pairs_total", 1), 1),
                "max_overlap": acc_c["max_overlap"], "lcp_iters_total": acc_c["lcp_iters"],
                "lcp_kernel_ms": acc_c["lcp_ms"], "gpu_launches": acc_c["launches"]}

    fp64 = None
    if not args.no_fp64:
        times64, acc64 = run_gpu_arm(R, torch, sc, R.RELCP_FP64, R.RELCP_GUESS_COLD, args.steps, args.warmup, flush,
                                     stream)
        t64 = float(sum(times64))
        fp64 = {"value": sc.n * args.steps / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / args.steps,
                "depth_max": acc64["depth_max"], "max_overlap": acc64["max_overlap"], "status": acc64["status"],
                "lcp_iters_total": acc64["lcp_iters"]}

    e2e_steps = args.steps if args.e2e_steps is None else args.e2e_steps
    if e2e_steps > 0:
        if dist:
            dist.barrier()
        e2e_t, h2d, d2h = run_e2e(R, torch, sc, precision, guess, e2e_steps, mlp_params)
        if dist:
            # the slowest replica sets the job's rate, as for the timed region
            t = torch.tensor([e2e_t], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_t = float(t.item())
        e2e_value = world * sc.n * e2e_steps / e2e_t
    else:
        e2e_value, h2d, d2h = None, 0, 0

    batched = (run_batched(R, torch, args.batched_scenes, rank=rank, world=world, dist=dist)
               if args.batched_scenes > 0 else None)

    # phase breakdown: a separate run of the headline configuration with events
    # between all phases (their host cost inflates its step times, so it is not
    # the timed run)
    phases, accp = None, None
    if args.phase_breakdown and rank == 0:
        _, accp = run_gpu_arm(R, torch, sc, precision, guess, args.steps, args.warmup, flush, stream, None, mlp_params,
                              timing="phases")
        phases = {"broadphase": accp["ms_broadphase"], "snsd_kernels": accp["snsd_ms"],
                  "lcp_incl_csr": accp["ms_lcp_phase"], "rest": accp["ms_other"],
                  "to_last_sync": accp["ms_step_events"], "note": "separate run with per-phase CUDA events"}

    hbm, peak_kind = peaks()
    lcp_gbs = acc["lcp_bytes"] / (acc["lcp_ms"] / 1e3) / 1e9 if acc["lcp_ms"] > 0 else 0.0
    line = None
    if rank == 0:
        cpu = oracle_rate(1024, 10 ** 6, args.cpu_budget) if args.cpu_budget > 0 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "bodies": sc.n, "precision": "mixed (FP32 bulk, FP64 checks)",
                       "guess": "learned" if guess == R.RELCP_GUESS_MLP else "cold",
                       "lcp_steps": "jacobi-scaled BB" if args.jacobi else "BB",
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": acc["launches"],
            "roofline": {"kernel": "lcp_kernel (persistent BB projected gradient)", "bound": "hbm",
                         "achieved": lcp_gbs, "peak": hbm, "unit": "GB/s", "frac": lcp_gbs / hbm,
                         "traffic": None, "peak_kind": peak_kind, "launches": acc["lcp_launches"],
                         "kernel_ms_total": acc["lcp_ms"]},
            "cpu_baseline": None if cpu is None else {
                "value": cpu["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": (f"first {cpu['steps']} steps (phi {cpu['phi_start']:.4f}->{cpu['phi_end']:.4f})"
                           f" of the 1,024-body version of the workload, {cpu['seconds']:.1f} s")},
            "clocks": clk,
            "fp64_gpu": fp64,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "mixed_cold": cold,
            "learned": learned_info,
            "batched": batched,
            "stats": {"depth_max": acc["depth_max"], "depth_mean": acc["depth_sum"] / args.steps,
                      "rows_max": acc["rows_max"], "pairs_max": acc["pairs_max"],
                      "lcp_iters_total": acc["lcp_iters"], "max_overlap": acc["max_overlap"],
                      "eps_ncp": 1e-3 * float(sc.axes.min()), "status": acc["status"],
                      "snsd_kernel_ms": accp["snsd_ms"] if accp else None,
                      "snsd_evals": accp["snsd_evals"] if accp else None,
                      "lcp_kernel_ms": acc["lcp_ms"], "wall_s": t_wall,
                      "phase_ms": phases,
                      "pair_list_rebuilds": acc["rebuilds"],
                      "learned_start_steps": acc.get("guess_steps", 0),
                      "newton_iters_per_pair_c0": acc.get("newton_c0", 0) / max(acc.get("pairs_total", 1), 1),
                      "phi_final": sc.meta["volume"] / float(np.prod(acc["box_final"]))},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
