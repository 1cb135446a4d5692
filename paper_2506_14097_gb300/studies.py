"""Drivers of the validation workloads (host logic only: they set up scenes,
call the C ABI through the binding and sample the trajectory; every step of
the method runs in the library's kernels).

Two-ellipsoid refinement study (Sec. 5.2, Table tab:two_ellipsoids): two
identical ellipsoids (radii 1, 1, 2), long axes at 45 degrees in the x-y
plane, centres one unit apart in x, pushed past each other by equal and
opposite unit forces, overdamped local drag (Eq. ellipsoid_mobility, xi = 1),
overlap tolerance 1e-5.  The sweep runs each time step as a one-scene batch
(the whole step loop of a launch stays on the device, which is what makes the
4 x 10^6 steps of dt = 1e-5 affordable) and samples the state every `sample`
time units.  With max_recursion = 0 the same study runs LCP-SNSD, the
single-constraint formulation the recursion reduces to.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import relcp as R
from . import scenes

E1_OFFSET_Y = 4.2  # initial vertical centre separation (the paper does not state it)
E1_T = 40.0        # contact starts near t = 2.5 and ends near t = 36 with xi = 1
E1_EPS = 1e-5
E1_SKIN = 0.5


def long_axis_angle(q: np.ndarray) -> np.ndarray:
    """In-plane angle of each body's long (body z) axis: atan2 of the y and x
    components of R(q) e_z (a read-out of the state, (s, w) quaternions)."""
    q = np.asarray(q, dtype=np.float64)
    s, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    ex = 2 * (x * z + s * y)
    ey = 2 * (y * z - s * x)
    return np.arctan2(ey, ex)


def two_ellipsoid_trajectory(dt: float, T: float = E1_T, sample: float = 0.5, max_recursion: int = 64,
                             precision: int = R.RELCP_FP64, lcp_tol: float = 1e-12):
    """One run of the refinement scene.  Returns a dict with the sample times,
    the positions and long-axis angles of both bodies at those times, the
    deepest recursion, the number of steps that appended rows, the largest
    overlap after any step, the worst status and the device time."""
    sc = scenes.two_ellipsoid_scene(offset_y=E1_OFFSET_Y)
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=precision, max_recursion=max_recursion,
                        lcp_max_iter=100000)
    b = R.Batch(cfg)
    params = np.array([[0.0, 0.0, 0.0, dt, E1_EPS, E1_SKIN, lcp_tol, E1_SKIN]])
    offsets = np.array([0, 2], dtype=np.int32)
    b.set_scenes(offsets, sc.x, sc.q, sc.axes, params, fext=sc.fext)
    b.set_threads(64)
    per = max(1, int(round(sample / dt)))
    nsamp = int(round(T / (per * dt)))
    ts, xs, angs, statuses = [], [], [], set()
    t0 = time.perf_counter()
    for k in range(nsamp):
        st = b.step(per, allow=(R.RELCP_ERR_RECURSION_LIMIT, R.RELCP_ERR_NOT_CONVERGED))
        statuses.add(R.STATUS_NAMES[st])
        x, q, _ = b.bodies()
        ts.append((k + 1) * per * dt)
        xs.append(x.copy())
        angs.append(long_axis_angle(q))
    wall = time.perf_counter() - t0
    ss = b.scene_stats()[0]
    b.close()
    return {"dt": dt, "t": np.array(ts), "x": np.array(xs), "angle": np.array(angs), "steps": per * nsamp,
            "depth_max": int(ss.depth_max), "aug_steps": int(ss.aug_steps), "lcp_iters": int(ss.lcp_iters),
            "max_overlap": float(ss.max_overlap_all), "status": sorted(statuses), "wall_s": wall}


def l2_errors(run: dict, ref: dict) -> dict:
    """Discrete L2 norms in time, sqrt(sum_k h (e(t_k))^2) over the common
    sample times (spacing h), of body 0's x and y position and long-axis angle
    against the reference run (the paper's norm is not stated)."""
    tr = np.round(run["t"], 9)
    tf = np.round(ref["t"], 9)
    common, ia, ib = np.intersect1d(tr, tf, return_indices=True)
    h = float(common[1] - common[0]) if common.size > 1 else 1.0
    ex = run["x"][ia, 0, 0] - ref["x"][ib, 0, 0]
    ey = run["x"][ia, 0, 1] - ref["x"][ib, 0, 1]
    ea = np.angle(np.exp(1j * (run["angle"][ia, 0] - ref["angle"][ib, 0])))
    f = lambda e: float(math.sqrt(h * float(np.sum(e * e))))
    return {"x": f(ex), "y": f(ey), "angle": f(ea)}


def refinement_sweep(dts=(1e-1, 1e-2, 1e-3, 1e-4, 1e-5), sample: float = 0.5, lcp_snsd_dts=(1e-1, 1e-2)):
    """ReLCP at every dt against the smallest dt's trajectory (self-
    convergence), plus LCP-SNSD (max_recursion = 0) at the listed dts."""
    runs = {dt: two_ellipsoid_trajectory(dt, sample=sample) for dt in dts}
    ref = runs[min(dts)]
    out = {"reference_dt": min(dts), "relcp": [], "lcp_snsd": []}
    for dt in dts:
        r = runs[dt]
        out["relcp"].append({"dt": dt, "l2_error": l2_errors(r, ref), "depth_max": r["depth_max"],
                             "aug_steps": r["aug_steps"], "steps": r["steps"], "max_overlap": r["max_overlap"],
                             "status": r["status"], "wall_s": r["wall_s"]})
    for dt in lcp_snsd_dts:
        r = two_ellipsoid_trajectory(dt, sample=sample, max_recursion=0)
        out["lcp_snsd"].append({"dt": dt, "l2_error": l2_errors(r, ref), "steps_over_tolerance": r["aug_steps"],
                                "max_overlap": r["max_overlap"], "status": r["status"]})
    return out


COLONY_DT = 0.05
COLONY_EPS = 5e-4   # 1e-3 x the cells' radius 0.5
COLONY_SKIN = 0.05


def colony_run(target_cells: int, shape: int = R.RELCP_SHAPE_ELLIPSOID, guess: int = R.RELCP_GUESS_MLP,
               mlp_params=None, precision: int = R.RELCP_MIXED, seed: int = 0, rate: float = 0.01,
               max_steps: int = 10 ** 6, stream=None, lcp_tol: float = 5e-8, lcp_max_iter: int = 5000,
               max_seconds: float = 600.0):
    """Grow a colony (scenes.Colony: rate N(0.01, 0.001) per cell, division
    at L = 2 with N(0, 0.05) rad jitter, dt = 0.05, planar overdamped
    dynamics) from one cell until it holds `target_cells` cells (or
    `max_seconds` pass), the GPU stepping it and the host loop growing and
    dividing the cells between steps (every step hands the library the new
    bodies); steps whose LCP hit its iteration cap or whose recursion hit its
    cap are counted and the run goes on.  Returns the steps, the
    final cell count, the host wall time, the summed device-synchronised step
    time, the largest accepted overlap, the steps whose C^k evaluation the
    learned start seeded and the Newton iterations per pair at C^k."""
    import torch

    from . import scenes as S

    col = S.Colony(seed=seed, rate=rate, dt=COLONY_DT)
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED_2D, precision=precision, dt=COLONY_DT, eps_ncp=COLONY_EPS,
                        box=(0, 0, 0), skin=COLONY_SKIN, lcp_tol=lcp_tol, lcp_max_iter=lcp_max_iter, shape=shape,
                        guess=guess)
    sim = R.Simulation(cfg, stream)
    if guess == R.RELCP_GUESS_MLP:
        R.relcp_load_mlp(sim.ctx, mlp_params)
    steps, maxov, learned, its, evals, worst, body_steps, capped, deep = 0, 0.0, 0, 0, 0, set(), 0, 0, 0
    t0 = time.perf_counter()
    step_s = 0.0
    while col.n < target_cells and steps < max_steps and time.perf_counter() - t0 < max_seconds:
        sim.set_bodies(np.ascontiguousarray(col.x), col.q(), col.axes())
        torch.cuda.synchronize()
        ts = time.perf_counter()
        st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED, R.RELCP_ERR_RECURSION_LIMIT))
        x, q, _ = sim.bodies()
        step_s += time.perf_counter() - ts
        s = sim.stats()
        worst.add(R.STATUS_NAMES[st])
        capped += int(st == R.RELCP_ERR_NOT_CONVERGED)
        deep += int(st == R.RELCP_ERR_RECURSION_LIMIT)
        maxov = max(maxov, s.max_overlap)
        learned += s.guess_used
        its += s.newton_iters_c0
        evals += s.snsd_c0_evaluated
        body_steps += col.n
        col.advance(x, q)
        steps += 1
    wall = time.perf_counter() - t0
    sim.close()
    return {"cells": col.n, "steps": steps, "divisions": col.divisions, "wall_s": wall, "step_s": step_s,
            "body_steps_per_s": body_steps / max(step_s, 1e-30),
            "max_overlap": maxov, "eps_ncp": COLONY_EPS, "status": sorted(worst), "lcp_capped_steps": capped,
            "recursion_capped_steps": deep,
            "learned_start_steps": learned,
            "newton_iters_per_pair_c0": its / max(evals, 1)}
