"""Benchmark: body-steps/s of the ReLCP time step on the compacting-suspension
workload (32,768 ellipsoids, semi-axes U[0.4, 1.0], volume fraction 0.1 ->
0.55 by affine compaction over 2,000 steps of dt = 5e-3, overdamped,
eps_NCP = 1e-3 x smallest semi-axis), mixed-precision path, with the plain
FP64 GPU path timed on the same steps for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  A "step" is one full time step of Algorithm 1
(broad phase, SNSD, LCP solves, trial re-evaluations, augmentations).
Timing: W untimed warm-up steps on a separate context; then the whole
2,000-step schedule runs on a fresh context and K of its steps, spread evenly
over it (step (i + 1/2) 2000 / K for i < K; all of them when K >= 2000), are
timed, each bracketed by CUDA events on the library's stream after a 256 MiB
L2 flush (outside the events); the steps in between run untimed.  Barrier +
synchronize around the timed region; max over ranks.  The rate is
bodies x K / (sum of the K step times): the schedule's mean step cost,
estimated from the sample.
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
SCHEDULE_STEPS = 2000
# DRAM bytes (read + write) of one lcp_kernel launch at the dense end of the
# schedule, from the ncu capture summarised in profiles/
LCP_DRAM_BYTES_PER_LAUNCH = 12.69e6


def timed_indices(total: int, k: int) -> list:
    """K step indices spread evenly over a schedule of `total` steps (the
    midpoints of K equal windows); every step when K >= total."""
    if k >= total:
        return list(range(total))
    return sorted({min(total - 1, int((i + 0.5) * total / k)) for i in range(k)})


METRIC = "body-steps/sec at 32k ellipsoids, mixed+learned vs plain FP64 GPU, equal overlap tol"
UNIT = "body-steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def build_scene(n, seed=1, steps=SCHEDULE_STEPS):
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


def run_batched(R, torch, n_scenes, steps=100, reps=3, rank=0, world=1, dist=None, threads=None):
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
    if threads:
        b.set_threads(threads)
    else:
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


def run_gpu_arm(R, torch, sc, precision, guess, total, timed, warmup, flush, stream, nvtx_from=None,
                mlp_params=None, timing="lcp", nvtx_to=None):
    """W warm-up steps on one context, then the whole schedule of `total`
    steps from the initial state on a fresh context, with the steps listed in
    `timed` timed.  Returns the per-step times of the timed steps, their
    accumulated stats (the window), and stats over every step."""
    x, q, axes = (np.ascontiguousarray(a) for a in (sc.x, sc.q, sc.axes))
    if warmup > 0:
        sim = new_sim(R, sc, precision, guess, None, stream.cuda_stream, mlp_params)
        sim.set_bodies(x, q, axes)
        for _ in range(warmup):
            sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        sim.close()
    sim = new_sim(R, sc, precision, guess, timing, stream.cuda_stream, mlp_params)
    sim.set_bodies(x, q, axes)
    timed_set = set(timed)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in timed]
    acc = dict(lcp_ms=0.0, lcp_bytes=0.0, lcp_launches=0, snsd_ms=0.0, snsd_evals=0, snsd_launches=0, depth_max=0,
               depth_sum=0, rows_max=0, pairs_max=0, lcp_iters=0, max_overlap=0.0, not_converged=0, status=set(),
               ms_broadphase=0.0, ms_lcp_phase=0.0, ms_other=0.0, ms_step_events=0.0, rebuilds=0, launches=0,
               rows_sum=0)
    whole = dict(max_overlap=0.0, depth_max=0, depth_steps=0, lcp_iters=0, status=set(), rows_max=0)
    windows = []
    vol = sc.meta["volume"]
    box = np.asarray(sc.box, dtype=np.float64)
    j = 0
    with torch.cuda.stream(stream):
        for k in range(total):
            if nvtx_from is not None and k == nvtx_from:
                torch.cuda.nvtx.range_push("relcp_profile")
            if nvtx_from is not None and nvtx_to is not None and k == nvtx_to:
                torch.cuda.nvtx.range_pop()
            if k in timed_set:
                flush.zero_()
                l0 = R.relcp_kernel_launches()
                ev[j][0].record(stream)
                st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
                ev[j][1].record(stream)
                acc["launches"] += R.relcp_kernel_launches() - l0
            else:
                st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
            s = sim.stats()
            whole["status"].add(R.STATUS_NAMES[st])
            whole["max_overlap"] = max(whole["max_overlap"], s.max_overlap)
            whole["depth_max"] = max(whole["depth_max"], s.depth)
            whole["depth_steps"] += int(s.depth > 0)
            whole["lcp_iters"] += s.lcp_iters_total
            whole["rows_max"] = max(whole["rows_max"], s.n_rows)
            if k in timed_set:
                windows.append({"step": k, "phi": vol / float(np.prod(box)), "lcp_iters": s.lcp_iters_total,
                                "rows": s.n_rows, "depth": s.depth})
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
                acc["rows_sum"] += s.n_rows
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
                j += 1
            box = np.array(s.box[:3], dtype=np.float64)
    torch.cuda.synchronize()
    if nvtx_from is not None and nvtx_from < total and (nvtx_to is None or nvtx_to >= total):
        torch.cuda.nvtx.range_pop()
    times = [a.elapsed_time(b) for a, b in ev]
    for w, t in zip(windows, times):
        w["ms"] = t
    acc["windows"] = windows
    acc["box_final"] = list(R.relcp_get_box(sim.ctx))
    sim.close()
    acc["status"] = sorted(acc["status"])
    whole["status"] = sorted(whole["status"])
    acc["whole"] = whole
    return times, acc


def run_e2e(R, torch, sc, precision, guess, total, timed, mlp_params=None):
    """The same schedule through the public C ABI with host buffers: every
    step copies the body state in (set_bodies: x, q, semi-axes) and the result
    out (get_bodies: x, q and the step velocity); the steps listed in `timed`
    are timed on the host clock (device synchronised before each), from the
    set_bodies call to the return of get_bodies.  The workload has no
    background velocity or external force, so none is passed in."""
    n = sc.n
    # copies: relcp_get_bodies writes each step's result into x and q, and the
    # scene's own arrays must keep the initial state for the runs after this one
    x, q, axes = (np.array(a, dtype=np.float64, order="C", copy=True) for a in (sc.x, sc.q, sc.axes))
    u = np.zeros((n, 6))
    cfg = make_cfg(R, sc, precision, guess, timing=None)
    sim = R.Simulation(cfg)
    if guess == R.RELCP_GUESS_MLP:
        R.relcp_load_mlp(sim.ctx, mlp_params)
    timed_set = set(timed)
    box = np.asarray(sc.box, dtype=np.float64)
    el = 0.0
    for k in range(total):
        if k in timed_set:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        for i in range(3):
            cfg.box[i] = box[i]
        R.relcp_set_config(sim.ctx, cfg)
        sim.set_bodies(x, q, axes)
        sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        R.relcp_get_bodies(sim.ctx, x, q, u)
        box = R.relcp_get_box(sim.ctx)
        if k in timed_set:
            el += time.perf_counter() - t0
    torch.cuda.synchronize()
    sim.close()
    h2d = n * (3 + 4 + 3) * 8
    d2h = n * (3 + 4 + 6) * 8
    return el, h2d, d2h


def run_colony(R, torch, cells, mlp_params, shapes=("ellipsoid",), seconds=600.0):
    """The growing colony from one cell to `cells` cells, mixed path, with the
    learned start (when a trained network is given) and with the cold start."""
    from paper_2506_14097_gb300 import studies

    out = {"workload": f"planar colony, 1 -> {cells} cells, dt 0.05, growth N(0.01, 0.001), division at L = 2 "
                       f"with N(0, 0.05) rad jitter, eps 5e-4, mixed path"}
    for shp in shapes:
        shape = R.RELCP_SHAPE_SPHEROCYLINDER if shp == "spherocylinder" else R.RELCP_SHAPE_ELLIPSOID
        arms = [("cold", R.RELCP_GUESS_COLD)]
        if mlp_params is not None and shape == R.RELCP_SHAPE_ELLIPSOID:
            arms.insert(0, ("learned", R.RELCP_GUESS_MLP))
        for name, guess in arms:
            out[f"{shp}_{name}"] = studies.colony_run(cells, shape=shape, guess=guess, mlp_params=mlp_params,
                                                      max_seconds=seconds)
    return out


def learned_fresh_state(R, torch, sc, mlp_params, flush, stream, at_step=1500, reps=5):
    """Where the learned start runs: a step whose SNSD at C^k is evaluated
    afresh for every candidate pair (a state given by set_bodies, as after a
    restart or any change of the bodies).  The compaction's state after
    `at_step` untimed steps is stepped once, `reps` times on fresh contexts,
    with the cold start and with the learned start: step time (CUDA events,
    L2 flushed before), Newton iterations per pair at C^k, and the pairs whose
    start the network declined."""
    sim = R.Simulation(make_cfg(R, sc, R.RELCP_MIXED, R.RELCP_GUESS_COLD, timing=None), stream.cuda_stream)
    sim.set_bodies(sc.x, sc.q, sc.axes)
    sim.step(at_step, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    x, q, _ = sim.bodies()
    box = R.relcp_get_box(sim.ctx)
    sim.close()
    out = {"state": f"compaction state after {at_step} steps, phi {sc.meta['volume'] / float(np.prod(box)):.3f}"}
    for name, guess in (("cold", R.RELCP_GUESS_COLD), ("learned", R.RELCP_GUESS_MLP)):
        times, its, evals, declined, used = [], [], [], [], []
        for _ in range(reps):
            cfg = make_cfg(R, sc, R.RELCP_MIXED, guess, timing=None)
            for k in range(3):
                cfg.box[k] = float(box[k])
            sim = R.Simulation(cfg, stream.cuda_stream)
            if guess == R.RELCP_GUESS_MLP:
                R.relcp_load_mlp(sim.ctx, mlp_params)
            sim.set_bodies(x, q, sc.axes)
            with torch.cuda.stream(stream):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
                e1.record(stream)
            torch.cuda.synchronize()
            st = sim.stats()
            times.append(e0.elapsed_time(e1))
            its.append(st.newton_iters_c0 / max(st.snsd_c0_evaluated, 1))
            evals.append(int(st.snsd_c0_evaluated))
            declined.append(int(st.newton_fallbacks))
            used.append(int(st.guess_used))
            sim.close()
        out[name] = {"ms_step_median": float(np.median(times)), "newton_iters_per_pair_c0": float(np.median(its)),
                     "pairs_evaluated_c0": evals[0], "declined_pairs": declined[0], "learned_start_used": used[0]}
    out["newton_iters_ratio"] = out["learned"]["newton_iters_per_pair_c0"] / max(out["cold"]["newton_iters_per_pair_c0"],
                                                                              1e-30)
    out["step_time_ratio"] = out["learned"]["ms_step_median"] / out["cold"]["ms_step_median"]
    return out


def augmentation_at_scale(R, torch, sc, flush, stream, at_step=1990, factors=(1, 20), reps=3):
    """The recursion on the full-size workload: the schedule's dense state
    after `at_step` steps (volume fraction ~0.55) stepped once with the time
    step scaled by each of `factors` (the strain rate unchanged, so the box
    compacts that many steps' worth in one), on fresh contexts, on both
    precision paths: step time (CUDA events, L2 flushed before; median of
    `reps`), recursion depth, rows and LCP iterations per recursion level,
    accepted overlap against eps_NCP and the step status.  At the schedule's
    own time step no row is appended; a step 20 times longer appends rows at
    every level the overlap test finds violated."""
    sim = R.Simulation(make_cfg(R, sc, R.RELCP_MIXED, R.RELCP_GUESS_COLD, timing=None), stream.cuda_stream)
    sim.set_bodies(sc.x, sc.q, sc.axes)
    sim.step(at_step, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    x, q, _ = sim.bodies()
    box = R.relcp_get_box(sim.ctx)
    sim.close()
    eps = 1e-3 * float(sc.axes.min())
    out = {"state": f"compaction state after {at_step} steps, phi {sc.meta['volume'] / float(np.prod(box)):.3f}",
           "eps_ncp": eps, "runs": []}
    for factor in factors:
        for name, prec in (("mixed", R.RELCP_MIXED), ("fp64", R.RELCP_FP64)):
            times, st_last, status = [], None, set()
            for _ in range(reps):
                cfg = make_cfg(R, sc, prec, R.RELCP_GUESS_COLD, timing=None)
                cfg.dt = factor * sc.dt
                for k in range(3):
                    cfg.box[k] = float(box[k])
                sim = R.Simulation(cfg, stream.cuda_stream)
                sim.set_bodies(x, q, sc.axes)
                with torch.cuda.stream(stream):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED, R.RELCP_ERR_RECURSION_LIMIT))
                    e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                status.add(R.STATUS_NAMES[st])
                st_last = sim.stats()
                sim.close()
            d = int(st_last.depth)
            levels = min(d + 1, len(st_last.rows_per_rec))
            out["runs"].append({"dt_factor": factor, "path": name, "ms_step_median": float(np.median(times)),
                                "depth": d, "rows_per_level": [int(v) for v in st_last.rows_per_rec[:levels]],
                                "lcp_iters_per_level": [int(v) for v in st_last.lcp_iters[:levels]],
                                "max_overlap": float(st_last.max_overlap),
                                "max_overlap_within_eps": bool(st_last.max_overlap <= eps),
                                "status": sorted(status)})
    for factor in factors:
        r = {x_["path"]: x_ for x_ in out["runs"] if x_["dt_factor"] == factor}
        out[f"speedup_vs_fp64_dt_x{factor}"] = r["fp64"]["ms_step_median"] / r["mixed"]["ms_step_median"]
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg, subset errors and reference arm)
# ---------------------------------------------------------------------------
SNAPSHOTS = os.path.join(ROOT, "tests", "golden", "compaction1024_snapshots.npz")
SUBSET_BODIES = 1024


def subset_states():
    """C^k of the 1,024-body version of the schedule at the start (from the
    seeded generator) and at the steps stored in the snapshot file, which the
    FP64 oracle's own trajectory wrote (tests/golden/make_compaction_snapshots.py).
    Returns the scene and a list of (step, x, q, box)."""
    sc = build_scene(SUBSET_BODIES)
    states = [(0, sc.x, sc.q, np.asarray(sc.box, dtype=np.float64))]
    if os.path.exists(SNAPSHOTS):
        d = np.load(SNAPSHOTS)
        if not np.array_equal(d["axes"], sc.axes):
            raise RuntimeError("snapshot file does not belong to this scene")
        for i, k in enumerate(d["steps"]):
            states.append((int(k), d["x"][i], d["q"][i], d["box"][i]))
    return sc, states


def _oracle_steps_worker(x, q, axes, box, dt, eps, skin, rate, nsteps):
    """`nsteps` consecutive oracle steps from one state (spawned process, one
    thread); per step the results the parity check compares and its time."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    from oracle import relcp_oracle as O

    out = []
    box = np.asarray(box, dtype=np.float64)
    for _ in range(nsteps):
        cfg = O.Config(dynamics=O.OVERDAMPED, dt=dt, eps_ncp=eps, box=tuple(box), skin=skin, strain_rate=rate)
        t0 = time.perf_counter()
        r = O.step(cfg, x, q, axes)
        el = time.perf_counter() - t0
        out.append({"seconds": el, "pairs": r.pairs, "ids": np.stack([r.rows_ia, r.rows_ib, r.rows_rec,
                                                                      r.rows_pair], axis=1).astype(np.int32),
                    "vel": r.vel, "uc": r.U_contact, "gamma": r.gamma, "depth": r.depth,
                    "max_overlap": r.max_overlap,
                    "status": r.status, "ambiguous": r.ambiguous, "rows": int(r.rows_ia.size)})
        x, q, box = r.x, r.q, np.asarray(r.box)
    return out


def run_oracle_pool(jobs, processes):
    """Run (state, nsteps) oracle jobs in spawned worker processes (no GPU
    context is inherited).  Returns the results in job order and the pool's
    wall time."""
    from concurrent.futures import ProcessPoolExecutor

    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ProcessPoolExecutor(max_workers=processes, mp_context=ctx) as ex:
        futs = [ex.submit(_oracle_steps_worker, *job) for job in jobs]
        res = [f.result() for f in futs]
    return res, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _max_known(vals):
    vals = [v for v in vals if v is not None]
    return max(vals) if vals else None


def subset_check(R, torch, arms, nsteps=2, processes=None, max_step=1750):
    """The oracle on the 1,024-body subset (the baseline leg) and the error of
    each GPU arm against it.  From every subset state both the oracle and each
    GPU arm take `nsteps` consecutive steps (the GPU carrying its SNSD values,
    warm starts and cached pair list from its first step to the next, as in
    the timed run).  Per step: candidate pairs and constraint ids (a, b,
    recursion, pair) bit for bit, velocities, contact velocities and the
    constraint impulses gamma as max-norm relative errors (gamma where the
    constraint sets agree), and the GPU's max overlap against eps_NCP.  The
    first step starts from the identical state; later steps start from each
    side's own previous result."""
    sc, states = subset_states()
    # (states past max_step, at volume fractions above 0.44, cost the oracle
    # a minute or more per step: the leg stays a bounded sample)
    states = [st for st in states if st[0] <= max_step]
    amin = float(sc.axes.min())
    eps, skin, rate = 1e-3 * amin, 0.1 * amin, sc.meta["strain_rate"]
    jobs = [(x, q, sc.axes, box, sc.dt, eps, skin, rate, nsteps) for (_, x, q, box) in states]
    processes = processes or max(1, min(len(jobs), host_cores()))
    orc, wall = run_oracle_pool(jobs, processes)
    vol = sc.meta["volume"]

    def rel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0

    report = {}
    for name, (precision, guess, mlp_params) in arms.items():
        per = []
        for (k, x, q, box), ores in zip(states, orc):
            cfg = make_cfg(R, sc, precision, guess, timing=None)
            for i in range(3):
                cfg.box[i] = float(box[i])
            sim = R.Simulation(cfg)
            if guess == R.RELCP_GUESS_MLP:
                R.relcp_load_mlp(sim.ctx, mlp_params)
            sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
            for j, o in enumerate(ores):
                st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
                s = sim.stats()
                pairs, _ = R.relcp_get_pairs(sim.ctx)
                ids, _, gam = R.relcp_get_rows(sim.ctx)
                _, _, v = sim.bodies()
                uc = R.relcp_get_contact_velocity(sim.ctx, sc.n)
                same_rows = bool(np.array_equal(ids, o["ids"]))
                per.append({"step": k + j, "phi": vol / float(np.prod(box)) if j == 0 else None,
                            "from_identical_state": j == 0, "status": R.STATUS_NAMES[st],
                            "pairs_equal": bool(np.array_equal(pairs, o["pairs"])),
                            "rows_equal": same_rows, "rows": o["rows"],
                            "depth": [int(s.depth), int(o["depth"])], "vel_rel_err": rel(v, o["vel"]),
                            "contact_vel_rel_err": rel(uc, o["uc"]),
                            "gamma_rel_err": rel(gam, o["gamma"]) if same_rows else None,
                            "max_overlap": float(s.max_overlap),
                            "oracle_ambiguous": int(o["ambiguous"])})
            sim.close()
        first = [p for p in per if p["from_identical_state"]]
        report[name] = {
            "identical_start": {"pairs_equal": all(p["pairs_equal"] for p in first),
                                "rows_equal": all(p["rows_equal"] for p in first),
                                "vel_rel_err_max": max(p["vel_rel_err"] for p in first),
                                "contact_vel_rel_err_max": max(p["contact_vel_rel_err"] for p in first),
                                "gamma_rel_err_max": _max_known(p["gamma_rel_err"] for p in first)},
            "all_steps": {"pairs_equal": all(p["pairs_equal"] for p in per),
                          "rows_equal": all(p["rows_equal"] for p in per),
                          "vel_rel_err_max": max(p["vel_rel_err"] for p in per),
                          "contact_vel_rel_err_max": max(p["contact_vel_rel_err"] for p in per),
                          "gamma_rel_err_max": _max_known(p["gamma_rel_err"] for p in per)},
            "max_overlap": max(p["max_overlap"] for p in per), "max_overlap_within_eps":
                all(p["max_overlap"] <= eps for p in per), "steps": per}
    steps_done = sum(len(o) for o in orc)
    cpu_s = sum(r["seconds"] for o in orc for r in o)
    sample = (f"{nsteps} consecutive oracle steps from each of {len(states)} states of the 1,024-body version of "
              f"the schedule (steps {', '.join(str(k) for k, *_ in states)}; phi "
              f"{vol / np.prod(states[0][3]):.3f}-{vol / np.prod(states[-1][3]):.3f}), one process per state on "
              f"{processes} host cores, {wall:.1f} s wall, {cpu_s:.1f} s of oracle time")
    cpu = {"value": SUBSET_BODIES * steps_done / wall, "unit": UNIT, "cores": processes, "kind": "oracle",
           "sample": sample, "per_core_value": SUBSET_BODIES * steps_done / cpu_s,
           "note": "1,024-body subset; not extrapolated to 32k"}
    report["eps_ncp"] = eps
    report["bounds"] = {"fp64": "relative 1e-9", "mixed": "relative 1e-5",
                        "sets": "pairs and constraint ids bit for bit"}
    return cpu, report


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, on the host cores.
    Each of the K sampled steps is one oracle step of the 1,024-body version of
    the workload from the stored state nearest before its place in the
    schedule (step (i + 1/2) 2000 / K), the steps run one per process."""
    if rank != 0:
        return
    sc, states = subset_states()
    amin = float(sc.axes.min())
    eps, skin, rate = 1e-3 * amin, 0.1 * amin, sc.meta["strain_rate"]
    pos = timed_indices(SCHEDULE_STEPS, args.steps)
    picks = [max((st for st in states if st[0] <= p), key=lambda st: st[0]) for p in pos]
    processes = max(1, min(len(picks), host_cores()))
    # warm-up: W steps from the initial state (loads and compiles the C core)
    run_oracle_pool([(sc.x, sc.q, sc.axes, states[0][3], sc.dt, eps, skin, rate, args.warmup)], 1)
    jobs = [(x, q, sc.axes, box, sc.dt, eps, skin, rate, 1) for (_, x, q, box) in picks]
    res, wall = run_oracle_pool(jobs, processes)
    cpu_s = sum(r[0]["seconds"] for r in res)
    n = len(picks)
    value = SUBSET_BODIES * n / wall
    sample = (f"{n} oracle steps of the 1,024-body version of the workload, one per sampled place in the "
              f"2,000-step schedule, each from the stored state nearest before it (steps "
              f"{', '.join(str(st[0]) for st in picks)}), {processes} processes, {wall:.1f} s wall, "
              f"{cpu_s:.1f} s of oracle time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * wall / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_bodies": SUBSET_BODIES},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": processes, "kind": "oracle", "sample": sample,
                             "per_core_value": SUBSET_BODIES * n / cpu_s},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=SCHEDULE_STEPS,
                    help="timed steps, spread evenly over the 2,000-step schedule (all of it at 2000)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bodies", type=int, default=32768)
    ap.add_argument("--schedule-steps", type=int, default=SCHEDULE_STEPS)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run through host buffers")
    ap.add_argument("--subset-steps", type=int, default=2,
                    help="consecutive steps per 1,024-body subset state in the oracle leg (0 skips the leg)")
    ap.add_argument("--jacobi", type=int, default=0, help="1: Jacobi-scaled projected-gradient steps")
    ap.add_argument("--cold", action="store_true", help="cold SNSD start only (no learned guess)")
    ap.add_argument("--phase-breakdown", type=int, default=1, help="1: extra run with per-phase events")
    ap.add_argument("--refinement", type=int, default=1,
                    help="1: the two-ellipsoid refinement sweep (dt 0.1 .. 1e-4, about a minute)")
    ap.add_argument("--batched-scenes", type=int, default=2048,
                    help="scenes of the batched-scene measurement (0 skips it)")
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--batched-threads", type=int, default=0,
                    help="fixed block size of the batched kernel (0: autotuned)")
    ap.add_argument("--augmentation", type=int, default=1,
                    help="1: the recursion on the dense 32k state with a 20x time step, both paths")
    ap.add_argument("--only-augmentation", action="store_true", help="only the recursion on the dense 32k state")
    ap.add_argument("--colony-cells", type=int, default=0,
                    help="grow the planar colony (ellipsoidal cells, learned and cold start) to this many cells "
                         "(0 skips it: tens of thousands of steps, see --only-colony)")
    ap.add_argument("--colony-seconds", type=float, default=600.0, help="time budget of each colony run")
    ap.add_argument("--only-colony", action="store_true",
                    help="run only the colony measurement (both cell shapes) and print its JSON")
    ap.add_argument("--only-learned", action="store_true",
                    help="profiling aid: harvest, train (20 epochs) and one learned-start step on a fresh state")
    ap.add_argument("--only-refinement", action="store_true",
                    help="run only the two-ellipsoid refinement sweep down to dt 1e-5 (about 7 minutes) and print it")
    ap.add_argument("--only-batched", action="store_true",
                    help="profiling aid: run only the batched-scene measurement and print its JSON")
    ap.add_argument("--nvtx-from", type=int, default=None,
                    help="profiling aid: wrap schedule steps >= this index in the NVTX range relcp_profile")
    ap.add_argument("--nvtx-to", type=int, default=None, help="profiling aid: end of that range (exclusive)")
    ap.add_argument("--step-times", default=None,
                    help="write the headline run's timed steps (schedule index, ms) to this file")
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
    if args.only_refinement:
        from paper_2506_14097_gb300 import studies

        t_r = time.perf_counter()
        out = studies.refinement_sweep(dts=(1e-1, 1e-2, 1e-3, 1e-4, 1e-5))
        out["wall_s"] = time.perf_counter() - t_r
        print(json.dumps(out), flush=True)
        return
    if args.only_learned:
        from paper_2506_14097_gb300 import learned

        feat, targ = learned.harvest_compaction(n=4096, seed=11, steps=300, every=10)
        t0 = time.perf_counter()
        mlp, losses = learned.train(feat, targ, epochs=20, batch=4096, lr=2e-3, seed=0)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        sc = build_scene(args.bodies, steps=args.schedule_steps)
        stream = torch.cuda.Stream()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        out = learned_fresh_state(R, torch, sc, mlp, flush, stream, reps=1)
        out["train_s"] = t_train
        out["loss"] = [losses[0], losses[-1]]
        print(json.dumps(out), flush=True)
        return
    if args.only_colony:
        mlp = None
        if not args.cold:
            from paper_2506_14097_gb300 import learned

            feat, targ = learned.harvest_compaction(n=4096, seed=11, steps=300, every=10)
            mlp, _ = learned.train(feat, targ, epochs=20, batch=4096, lr=2e-3, seed=0)
        print(json.dumps(run_colony(R, torch, args.colony_cells, mlp, shapes=("ellipsoid", "spherocylinder"),
                                    seconds=args.colony_seconds)), flush=True)
        return
    if args.only_augmentation:
        sc = build_scene(args.bodies, steps=args.schedule_steps)
        stream = torch.cuda.Stream()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(augmentation_at_scale(R, torch, sc, flush, stream)), flush=True)
        return
    if args.only_batched:
        out = run_batched(R, torch, args.batched_scenes, steps=args.batched_steps, reps=1,
                          threads=args.batched_threads or None)
        print(json.dumps(out), flush=True)
        return
    global EXTRA_FLAGS
    if args.jacobi:
        EXTRA_FLAGS |= R.RELCP_FLAG_JACOBI
    sc = build_scene(args.bodies, steps=args.schedule_steps)
    total = args.schedule_steps
    timed = timed_indices(total, args.steps)
    K = len(timed)
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
    times, acc = run_gpu_arm(R, torch, sc, precision, guess, total, timed, args.warmup, flush, stream,
                             args.nvtx_from, mlp_params, nvtx_to=args.nvtx_to)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    if args.step_times and rank == 0:
        with open(args.step_times, "w") as f:
            f.write("".join("%d %.6f\n" % (k, t) for k, t in zip(timed, times)))
    total_ms = float(sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * sc.n * K / (total_ms / 1e3)

    def arm_summary(times_, acc_):
        t_ = float(sum(times_))
        return {"value": sc.n * K / (t_ / 1e3), "unit": UNIT, "ms_per_step": t_ / K,
                "lcp_iters_total": acc_["lcp_iters"], "lcp_kernel_ms": acc_["lcp_ms"], "rows_max": acc_["rows_max"],
                "depth_max": acc_["depth_max"], "max_overlap": acc_["max_overlap"], "status": acc_["status"],
                "gpu_launches": acc_["launches"],
                "whole_schedule": {"max_overlap": acc_["whole"]["max_overlap"],
                                   "depth_max": acc_["whole"]["depth_max"],
                                   "lcp_iters": acc_["whole"]["lcp_iters"], "status": acc_["whole"]["status"]}}

    cold = None
    if guess == R.RELCP_GUESS_MLP and not args.no_fp64:
        times_c, acc_c = run_gpu_arm(R, torch, sc, precision, R.RELCP_GUESS_COLD, total, timed, args.warmup, flush,
                                     stream)
        cold = arm_summary(times_c, acc_c)
        cold["newton_iters_per_pair_c0"] = acc_c.get("newton_c0", 0) / max(acc_c.get("pairs_total", 1), 1)

    fp64 = None
    if not args.no_fp64:
        times64, acc64 = run_gpu_arm(R, torch, sc, R.RELCP_FP64, R.RELCP_GUESS_COLD, total, timed, args.warmup,
                                     flush, stream)
        fp64 = arm_summary(times64, acc64)

    if not args.no_e2e:
        if dist:
            dist.barrier()
        e2e_t, h2d, d2h = run_e2e(R, torch, sc, precision, guess, total, timed, mlp_params)
        if dist:
            # the slowest replica sets the job's rate, as for the timed region
            t = torch.tensor([e2e_t], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_t = float(t.item())
        e2e_value = world * sc.n * K / e2e_t
    else:
        e2e_value, h2d, d2h = None, 0, 0

    batched = (run_batched(R, torch, args.batched_scenes, steps=args.batched_steps, rank=rank, world=world, dist=dist,
                           threads=args.batched_threads or None)
               if args.batched_scenes > 0 else None)
    fresh = (learned_fresh_state(R, torch, sc, mlp_params, flush, stream)
             if (mlp_params is not None and rank == 0 and total >= 1500) else None)
    augmentation = (augmentation_at_scale(R, torch, sc, flush, stream)
                    if (args.augmentation and rank == 0 and total >= 1990) else None)
    colony = (run_colony(R, torch, args.colony_cells, mlp_params, seconds=args.colony_seconds)
              if (args.colony_cells > 0 and rank == 0) else None)
    refinement = None
    if args.refinement and rank == 0:
        from paper_2506_14097_gb300 import studies

        t_r = time.perf_counter()
        refinement = studies.refinement_sweep(dts=(1e-1, 1e-2, 1e-3, 1e-4))
        refinement["wall_s"] = time.perf_counter() - t_r
        refinement["workload"] = ("two ellipsoids (radii 1, 1, 2) at 45 degrees, unit opposing forces, overdamped "
                                  "(xi = 1), eps 1e-5, t in [0, 40], FP64 batched path")

    # phase breakdown: a separate run of the headline configuration with events
    # between all phases (their host cost inflates its step times, so it is not
    # the timed run)
    phases, accp = None, None
    if args.phase_breakdown and rank == 0:
        _, accp = run_gpu_arm(R, torch, sc, precision, guess, total, timed, args.warmup, flush, stream, None,
                              mlp_params, timing="phases")
        phases = {"broadphase": accp["ms_broadphase"], "snsd_kernels": accp["snsd_ms"],
                  "lcp_incl_csr": accp["ms_lcp_phase"], "rest": accp["ms_other"],
                  "to_last_sync": accp["ms_step_events"],
                  "note": "separate run with per-phase CUDA events, summed over the timed steps"}

    hbm, peak_kind = peaks()
    lcp_gbs = acc["lcp_bytes"] / (acc["lcp_ms"] / 1e3) / 1e9 if acc["lcp_ms"] > 0 else 0.0
    line = None
    if rank == 0:
        cpu, subset = None, None
        if args.subset_steps > 0 and world == 1:
            arms = {"mixed_learned": (precision, guess, mlp_params), "fp64": (R.RELCP_FP64, R.RELCP_GUESS_COLD, None)}
            cpu, subset = subset_check(R, torch, arms, nsteps=args.subset_steps)
        vol = sc.meta["volume"]
        wins = acc["windows"]
        if len(wins) > 40:  # one entry per tenth of the sample
            idx = sorted({int(i * len(wins) / 10) for i in range(10)})
            wins = [wins[i] for i in idx]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "bodies": sc.n, "precision": "mixed (FP32 bulk, FP64 checks)",
                       "guess": "learned" if guess == R.RELCP_GUESS_MLP else "cold",
                       "lcp_steps": "jacobi-scaled BB" if args.jacobi else "BB",
                       "timed_steps": (f"{K} of the {total} schedule steps, spread evenly (step (i + 1/2) {total}/"
                                       f"{K}); the rest run untimed" if K < total else "all schedule steps"),
                       "phi_timed": ([acc["windows"][0]["phi"], acc["windows"][-1]["phi"]]
                                     if acc["windows"] else None),
                       "l2": "flushed before each timed step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": K, "how": "set_bodies + step + get_bodies per step on host arrays, the same sampled "
                                       "steps timed on the host clock"},
            "gpu_launches": acc["launches"],
            "roofline": {"kernel": "lcp_kernel (persistent BB projected gradient)", "bound": "hbm",
                         "achieved": lcp_gbs, "peak": hbm, "unit": "GB/s", "frac": lcp_gbs / hbm,
                         "traffic": LCP_DRAM_BYTES_PER_LAUNCH,
                         "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of the dense-end launch "
                                         "(schedule step 1950, 103 iterations; 6.02 MB at step 1050): "
                                         "profiles/lcp_kernel_traffic_compaction32k.md",
                         "peak_kind": peak_kind, "launches": acc["lcp_launches"],
                         "kernel_ms_total": acc["lcp_ms"],
                         "bytes": "per iteration 76 B per row + 75 B per body (FP32 rows, FP64 offsets)"},
            "cpu_baseline": cpu,
            "oracle_subset": subset,
            "clocks": clk,
            "fp64_gpu": fp64,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "mixed_cold": cold,
            "learned": learned_info,
            "learned_fresh_state": fresh,
            "batched": batched,
            "refinement": refinement,
            "augmentation_at_scale": augmentation,
            "colony": colony,
            "stats": {"depth_max": acc["depth_max"], "depth_mean": acc["depth_sum"] / K,
                      "rows_max": acc["rows_max"], "rows_mean": acc["rows_sum"] / K, "pairs_max": acc["pairs_max"],
                      "lcp_iters_total": acc["lcp_iters"], "max_overlap": acc["max_overlap"],
                      "eps_ncp": 1e-3 * float(sc.axes.min()), "status": acc["status"],
                      "snsd_kernel_ms": accp["snsd_ms"] if accp else None,
                      "snsd_evals": accp["snsd_evals"] if accp else None,
                      "lcp_kernel_ms": acc["lcp_ms"], "wall_s": t_wall,
                      "phase_ms": phases,
                      "pair_list_rebuilds": acc["rebuilds"],
                      "learned_start_steps": acc.get("guess_steps", 0),
                      "newton_iters_per_pair_c0": acc.get("newton_c0", 0) / max(acc.get("pairs_total", 1), 1),
                      "phi_final": vol / float(np.prod(acc["box_final"])),
                      "whole_schedule": acc["whole"],
                      "windows": wins},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
