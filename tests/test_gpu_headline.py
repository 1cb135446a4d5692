"""Oracle step parity of the benchmark's own configuration: the 1,024-body
version of the compacting suspension (overdamped, affine compaction of a
periodic box), mixed precision, from states of the FP64 oracle's own
trajectory through the schedule (tests/golden/compaction1024_snapshots.npz,
written by make_compaction_snapshots.py).

* consecutive steps with the carried SNSD values, the warm starts and the
  cached pair list live, cold and learned start: every step's candidate pairs
  and constraint ids equal the oracle trajectory's bit for bit, velocities,
  the contact velocities (which the affine background does not dwarf) and the
  constraint impulses gamma within relative 1e-5 on the first step from the
  identical state and within the divergence the two trajectories accumulate
  afterwards (5e-5), and every accepted overlap within eps_NCP;
* the same with the state handed over from the oracle before every step
  (the library keeps the pair list and warm starts of moved bodies): relative
  1e-5 on every step;
* one step from each of the two densest stored states (volume fractions 0.505
  and 0.545), relative 1e-5;
* a step twenty times longer on the dense state (the same strain rate, so
  twenty times the compaction of a step), where the recursion appends rows
  (depth >= 1), with the same bounds.

The library's default LCP stop for the mixed path (1e-8 a_min) is what these
bounds need: the error of a stopped projected-gradient iterate follows the
stop, and 1e-7 a_min leaves up to 4e-5 on these states in any precision.
"""
import os

import numpy as np
import pytest

from paper_2506_14097_gb300 import scenes

pytestmark = pytest.mark.gpu

SNAP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "compaction1024_snapshots.npz")


def rel_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0


def snapshot(step):
    d = np.load(SNAP)
    sc = scenes.suspension_scene(seed=int(d["seed"]), n=d["x"].shape[1], phi=0.1, phi_final=0.55, steps=2000,
                                 dt=float(d["dt"]))
    assert np.array_equal(sc.axes, d["axes"])
    i = int(np.nonzero(d["steps"] == step)[0][0])
    return sc, d["x"][i].copy(), d["q"][i].copy(), d["box"][i].copy()


def configs(R, orc, sc, box, precision, guess, dt=None, flags=0):
    amin = float(sc.axes.min())
    dt = sc.dt if dt is None else dt
    rate = sc.meta["strain_rate"]
    ocfg = orc.Config(dynamics=orc.OVERDAMPED, dt=dt, eps_ncp=1e-3 * amin, box=tuple(box), skin=0.1 * amin,
                      strain_rate=rate)
    gcfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=precision, guess=guess, dt=dt, eps_ncp=1e-3 * amin,
                         box=tuple(box), skin=0.1 * amin, strain_rate=rate, length_scale=amin, flags=flags)
    return ocfg, gcfg


def compare(R, sim, ref, n, bound, eps):
    pairs, _ = R.relcp_get_pairs(sim.ctx)
    ids, _, gam = R.relcp_get_rows(sim.ctx)
    _, _, v = sim.bodies()
    uc = R.relcp_get_contact_velocity(sim.ctx, n)
    st = sim.stats()
    assert ref.ambiguous == 0 and ref.status == 0
    assert np.array_equal(pairs, ref.pairs)
    assert np.array_equal(ids, np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1))
    assert st.depth == ref.depth
    assert rel_err(v, ref.vel) <= bound, rel_err(v, ref.vel)
    assert rel_err(uc, ref.U_contact) <= bound, rel_err(uc, ref.U_contact)
    assert rel_err(gam, ref.gamma) <= bound, rel_err(gam, ref.gamma)
    assert st.max_overlap <= eps
    return st


@pytest.fixture(scope="module")
def oracle_trajectory(orc):
    """Three consecutive oracle steps from the stored state at step 1750
    (volume fraction 0.44): per step the state it starts from and its result."""
    from paper_2506_14097_gb300 import relcp as R

    sc, x, q, box = snapshot(1750)
    ocfg, _ = configs(R, orc, sc, box, R.RELCP_MIXED, R.RELCP_GUESS_COLD)
    out = []
    for _ in range(3):
        ref = orc.step(orc.Config(**{**ocfg.__dict__, "box": tuple(box)}), x, q, sc.axes)
        out.append(((x, q, box), ref))
        x, q, box = ref.x, ref.q, np.asarray(ref.box)
    return sc, ocfg, out


@pytest.fixture(scope="module")
def mlp_params():
    from paper_2506_14097_gb300 import learned

    feat, targ = learned.harvest_compaction(n=2048, seed=11, steps=200, every=20)
    params, _ = learned.train(feat, targ, epochs=5, batch=4096, lr=2e-3, seed=0)
    return params


@pytest.mark.parametrize("guess", ["cold", "learned"])
def test_consecutive_steps_match_oracle_trajectory(relcp_gpu, orc, oracle_trajectory, mlp_params, guess):
    R = relcp_gpu
    sc, ocfg, traj = oracle_trajectory
    (x, q, box), _ = traj[0]
    g = R.RELCP_GUESS_MLP if guess == "learned" else R.RELCP_GUESS_COLD
    # (the learned start serves batches of 4,096 new pairs or more; the flag
    # lets it serve this 1,024-body scene's first step)
    _, gcfg = configs(R, orc, sc, box, R.RELCP_MIXED, g,
                      flags=R.RELCP_FLAG_LEARNED_ALWAYS if g == R.RELCP_GUESS_MLP else 0)
    sim = R.Simulation(gcfg)
    if g == R.RELCP_GUESS_MLP:
        R.relcp_load_mlp(sim.ctx, mlp_params)
    sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
    reused = 0
    for k, (_, ref) in enumerate(traj):
        assert sim.step(1) == R.RELCP_OK
        st = compare(R, sim, ref, sc.n, 1e-5 if k == 0 else 5e-5, ocfg.eps_ncp)
        assert st.n_rows > 2000
        if k == 0:
            assert st.guess_used == (1 if g == R.RELCP_GUESS_MLP else 0)
        else:
            reused += st.n_pairs - st.snsd_c0_evaluated
    assert reused > 0  # the carried SNSD values were used
    sim.close()


def test_handed_over_states_match_oracle(relcp_gpu, orc, oracle_trajectory):
    R = relcp_gpu
    sc, ocfg, traj = oracle_trajectory
    _, gcfg = configs(R, orc, sc, traj[0][0][2], R.RELCP_MIXED, R.RELCP_GUESS_COLD)
    sim = R.Simulation(gcfg)
    for (x, q, box), ref in traj:
        for i in range(3):
            gcfg.box[i] = float(box[i])
        R.relcp_set_config(sim.ctx, gcfg)
        sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
        assert sim.step(1) == R.RELCP_OK
        compare(R, sim, ref, sc.n, 1e-5, ocfg.eps_ncp)
    sim.close()


@pytest.mark.parametrize("step", [1900, 1990])
def test_densest_states_match_oracle(relcp_gpu, orc, step):
    """One step from the stored states at the dense end of the schedule
    (volume fractions 0.505 and 0.545, 2,600-3,000 rows, the most iterations
    per solve), cold start."""
    R = relcp_gpu
    sc, x, q, box = snapshot(step)
    ocfg, gcfg = configs(R, orc, sc, box, R.RELCP_MIXED, R.RELCP_GUESS_COLD)
    ref = orc.step(ocfg, x, q, sc.axes)
    sim = R.Simulation(gcfg)
    sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
    assert sim.step(1) == R.RELCP_OK
    st = compare(R, sim, ref, sc.n, 1e-5, ocfg.eps_ncp)
    assert st.n_rows > 2500
    sim.close()


def test_long_step_recursion_on_dense_state(relcp_gpu, orc):
    R = relcp_gpu
    sc, x, q, box = snapshot(1750)
    ocfg, gcfg = configs(R, orc, sc, box, R.RELCP_MIXED, R.RELCP_GUESS_COLD, dt=20 * sc.dt)
    ref = orc.step(ocfg, x, q, sc.axes)
    assert ref.depth >= 1
    sim = R.Simulation(gcfg)
    sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
    assert sim.step(1) == R.RELCP_OK
    compare(R, sim, ref, sc.n, 1e-5, ocfg.eps_ncp)
    sim.close()


def test_refinement_below_the_fp32_floor(relcp_gpu, orc):
    """The mixed LCP's iterative refinement (FP32 iterations to 10 x lcp_tol,
    the FP64 residual of that iterate, an FP32 solve of the correction) at a
    stop of 1e-9 a_min on the volume-fraction-0.505 state, below what plain
    FP32 iterates resolve there: the refined step converges in fewer
    iterations than plain FP32 iterations take (or reach at their cap) and
    stays within the mixed bound.  (Its distance from the oracle, ~6e-6 here,
    is that of the FP32 Newton normals and lever arms the rows are built from,
    relative ~1e-6, which no LCP stop changes.)"""
    R = relcp_gpu
    sc, x, q, box = snapshot(1900)
    ocfg, _ = configs(R, orc, sc, box, R.RELCP_MIXED, R.RELCP_GUESS_COLD)
    ref = orc.step(ocfg, x, q, sc.axes)
    amin = float(sc.axes.min())
    out = {}
    for flags in (0, R.RELCP_FLAG_NO_LCP_REFINE):
        _, gcfg = configs(R, orc, sc, box, R.RELCP_MIXED, R.RELCP_GUESS_COLD, flags=flags)
        gcfg.lcp_tol = 1e-9 * amin
        gcfg.lcp_max_iter = 3000
        sim = R.Simulation(gcfg)
        sim.set_bodies(np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
        st = sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        ids, _, gam = R.relcp_get_rows(sim.ctx)
        assert np.array_equal(ids, np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1))
        uc = R.relcp_get_contact_velocity(sim.ctx, sc.n)
        out[flags] = (st, sim.stats().lcp_iters_total, max(rel_err(gam, ref.gamma), rel_err(uc, ref.U_contact)))
        sim.close()
    print(out)
    st, iters, err = out[0]
    assert st == R.RELCP_OK and err <= 1e-5, out
    assert iters < out[R.RELCP_FLAG_NO_LCP_REFINE][1], out
