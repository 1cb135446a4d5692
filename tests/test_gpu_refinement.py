"""Two-ellipsoid refinement study (Sec. 5.2, Table tab:two_ellipsoids) on the
GPU, through the batched entry points (one scene per run, the step loop on the
device):

* at dt = 0.1 and 0.01 the GPU trajectory (FP64 path) equals the oracle's,
  step for step, sampled every half time unit, for ReLCP and for LCP-SNSD
  (recursion capped at 0);
* under refinement the trajectories self-converge: the L2 errors against the
  finest run fall monotonically, as in the paper's table (whose exact values
  depend on the unstated drag coefficient and initial offset);
* the recursion appends rows at dt = 0.1 and never at the finest step
  (reduction to the single-constraint SNSD-LCP, Corollary "reduction to
  single-constraint SNSD-LCP"), and ReLCP keeps every accepted overlap within
  the tolerance while LCP-SNSD at dt = 0.1 does not.
"""
import numpy as np
import pytest

from paper_2506_14097_gb300 import scenes

pytestmark = pytest.mark.gpu


def oracle_trajectory(orc, dt, T, sample, max_recursion=64):
    from paper_2506_14097_gb300 import studies

    sc = scenes.two_ellipsoid_scene(offset_y=studies.E1_OFFSET_Y)
    cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=dt, eps_ncp=studies.E1_EPS, box=(0, 0, 0), skin=studies.E1_SKIN,
                     max_recursion=max_recursion)
    per = int(round(sample / dt))
    x, q = sc.x, sc.q
    xs, angs, depth_steps, depth_max, maxov = [], [], 0, 0, 0.0
    for k in range(int(round(T / dt))):
        r = orc.step(cfg, x, q, sc.axes, None, sc.fext)
        assert r.status in (0, 5)
        x, q = r.x, r.q
        depth_max = max(depth_max, r.depth)
        depth_steps += int(r.depth > 0 or r.status == 5)
        maxov = max(maxov, r.max_overlap)
        if (k + 1) % per == 0:
            xs.append(x.copy())
            angs.append(studies.long_axis_angle(q))
    return np.array(xs), np.array(angs), depth_max, depth_steps, maxov


@pytest.mark.parametrize("dt,max_recursion", [(0.1, 64), (0.01, 64), (0.1, 0)])
def test_refinement_trajectory_matches_oracle(relcp_gpu, orc, dt, max_recursion):
    from paper_2506_14097_gb300 import studies

    T, sample = studies.E1_T, 0.5
    g = studies.two_ellipsoid_trajectory(dt, T=T, sample=sample, max_recursion=max_recursion)
    ox, oa, odepth, osteps, oov = oracle_trajectory(orc, dt, T, sample, max_recursion)
    assert g["x"].shape == ox.shape
    # FP64 path: the per-step relative 1e-9 accumulated over up to 4,000 steps
    assert np.abs(g["x"] - ox).max() <= 1e-7 * (1 + np.abs(ox).max())
    assert np.abs(g["angle"] - oa).max() <= 1e-7
    assert g["depth_max"] == odepth and g["aug_steps"] == osteps
    assert abs(g["max_overlap"] - oov) <= 1e-9
    if max_recursion == 64:
        assert g["max_overlap"] <= studies.E1_EPS and g["status"] == ["OK"]
        if dt == 0.1:
            assert odepth >= 1  # the recursion appends rows at the coarse step
    else:
        assert g["max_overlap"] > studies.E1_EPS and osteps >= 1  # LCP-SNSD leaves overlaps


def test_refinement_self_convergence_and_reduction(relcp_gpu):
    from paper_2506_14097_gb300 import studies

    dts = (1e-1, 1e-2, 1e-3, 1e-4)
    runs = {dt: studies.two_ellipsoid_trajectory(dt) for dt in dts}
    ref = runs[1e-4]
    errs = [studies.l2_errors(runs[dt], ref) for dt in dts[:-1]]
    for key in ("x", "y", "angle"):
        e = [er[key] for er in errs]
        assert e[0] > e[1] > e[2], (key, e)
    assert runs[1e-1]["depth_max"] >= 1
    assert runs[1e-4]["depth_max"] == 0 and runs[1e-4]["aug_steps"] == 0
    for dt in dts:
        assert runs[dt]["max_overlap"] <= studies.E1_EPS and runs[dt]["status"] == ["OK"]
    snsd = studies.two_ellipsoid_trajectory(1e-1, max_recursion=0)
    assert snsd["max_overlap"] > studies.E1_EPS and snsd["aug_steps"] >= 1
