"""Batched scenes: many independent scenes stepped by one persistent launch
(each CTA runs the whole of Algorithm 1 for its scene).

Checks, per scene, against the FP64 oracle's step from the same state
(candidate pair list and constraint ids (a, b, recursion, pair) bit for bit,
recursion depth equal, velocities / positions / orientations within the path's
tolerance: FP64 1e-9, mixed 1e-5, normwise relative; scenes of 2 to 512
bodies), against
the single-scene path over several steps, bitwise determinism, the edge cases
(empty, one-body and maximum scenes, capacity, bad arguments) and the block-size
autotuner with its JSON cache."""
import json

import numpy as np
import pytest

from paper_2506_14097_gb300 import scenes

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if b.size == 0:
        return 0.0
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dense_scenes(spec, spacing=1.8, dt=1e-2, vel=3.0, om=1.5):
    """Lattice scenes closer than the bodies' sizes with fast bodies, so that
    contacts, appended rows and recursion occur within a few steps."""
    return [scenes.lattice_scene(seed=s, n=n, spacing=spacing, dt=dt, vel_sigma=vel, omega_sigma=om) for s, n in spec]


def new_batch(R, scs, precision, dynamics=None):
    dyn = R.RELCP_INERTIAL if dynamics is None else dynamics
    offsets, x, q, axes, vel, params = scenes.pack_scenes(scs, precision_fp64=(precision == R.RELCP_FP64))
    b = R.Batch(R.make_config(dynamics=dyn, precision=precision))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    return b, offsets, params


@pytest.mark.parametrize("precision,bound", [(0, 1e-9), (1, 1e-5)])
def test_batch_steps_match_oracle(relcp_gpu, orc, precision, bound):
    R = relcp_gpu
    scs = dense_scenes([(2, 64), (3, 27), (4, 9), (5, 2), (6, 216), (7, 343), (8, 512)])
    state = [(sc.x.copy(), sc.q.copy(), sc.vel.copy()) for sc in scs]
    depths, big_rows = [], 0
    for k in range(6):
        cur = [scenes.Scene(x=x, q=q, axes=sc.axes, vel=v, fext=sc.fext, box=sc.box, dt=sc.dt)
               for sc, (x, q, v) in zip(scs, state)]
        b, offsets, params = new_batch(R, cur, precision)
        b.step(1)
        xb, qb, vb = b.bodies()
        st = b.scene_stats()
        contacts = [b.contacts(s) for s in range(len(cur))]
        b.close()
        nxt = []
        for s, sc in enumerate(cur):
            amin = float(sc.axes.min())
            ocfg = orc.Config(dynamics=orc.INERTIAL, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box),
                              skin=0.1 * amin)
            ref = orc.step(ocfg, sc.x, sc.q, sc.axes, sc.vel)
            assert ref.ambiguous == 0 and ref.status == 0
            sl = slice(offsets[s], offsets[s + 1])
            assert st[s].status == 0 and st[s].steps_done == 1
            assert st[s].n_pairs == len(ref.pairs), (k, s)
            pairs, ids = contacts[s]
            assert np.array_equal(pairs, ref.pairs), (k, s)
            ref_ids = np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1)
            assert np.array_equal(ids, ref_ids), (k, s)
            if sc.n >= 200:
                big_rows += ids.shape[0]
            assert st[s].depth_max == ref.depth, (k, s)
            assert rel_err(vb[sl], ref.vel) <= bound, (k, s, rel_err(vb[sl], ref.vel))
            dx = orc.min_image(xb[sl] - ref.x, np.asarray(ref.box))
            assert np.abs(dx).max() <= bound * (1 + np.abs(ref.x).max())
            qs = np.sign(np.sum(qb[sl] * ref.q, axis=1))[:, None]
            assert np.abs(qb[sl] - qs * ref.q).max() <= bound
            assert st[s].max_overlap <= ocfg.eps_ncp
            depths.append(ref.depth)
            nxt.append((ref.x, ref.q, ref.vel))
        state = nxt
    assert max(depths) >= 1  # the recursion ran inside the persistent launch
    assert big_rows > 1000  # the 216- to 512-body scenes carried many constraints


@pytest.mark.parametrize("precision,tol", [(0, 1e-7), (1, 1e-4)])
def test_batch_matches_single_scene_path(relcp_gpu, precision, tol):
    """Ten steps of each scene in one launch against the same scene stepped by
    the single-scene path (grid-wide kernels): the same method, different
    reduction orders, so the trajectories agree to the solver tolerances."""
    R = relcp_gpu
    scs = dense_scenes([(11, 150), (12, 64), (13, 30), (14, 5)], spacing=2.0)
    b, offsets, params = new_batch(R, scs, precision)
    b.step(10, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    xb, qb, vb = b.bodies()
    st = b.scene_stats()
    b.close()
    for s, sc in enumerate(scs):
        p = params[s]
        cfg = R.make_config(dynamics=R.RELCP_INERTIAL, precision=precision, dt=p[3], eps_ncp=p[4], box=tuple(p[:3]),
                            skin=p[5], phi_skin=p[7], lcp_tol=p[6], flags=R.RELCP_FLAG_NO_SNSD_REUSE)
        sim = R.Simulation(cfg)
        sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        for _ in range(10):
            sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        x, q, v = sim.bodies()
        sim.close()
        sl = slice(offsets[s], offsets[s + 1])
        d = xb[sl] - x
        d -= sc.box * np.round(d / sc.box)
        assert np.abs(d).max() <= tol, (s, np.abs(d).max())
        assert rel_err(vb[sl], v) <= 10 * tol
        assert st[s].steps_done == 10


def test_batch_deterministic(relcp_gpu):
    R = relcp_gpu
    scs = dense_scenes([(21, 100), (22, 40), (23, 7)])
    outs = []
    for _ in range(2):
        b, _, _ = new_batch(R, scs, R.RELCP_MIXED)
        b.step(6, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        outs.append(b.bodies())
        b.close()
    for a, c in zip(outs[0], outs[1]):
        assert np.array_equal(a, c)


def test_batch_edge_cases(relcp_gpu):
    R = relcp_gpu
    empty = scenes.Scene(x=np.zeros((0, 3)), q=np.zeros((0, 4)), axes=np.zeros((0, 3)), vel=np.zeros((0, 6)),
                         fext=np.zeros((0, 6)), box=np.array([5.0] * 3), dt=1e-3)
    one = scenes.lattice_scene(seed=31, n=1, dt=1e-3)
    big = scenes.lattice_scene(seed=32, n=1024, dt=1e-3)
    scs = [one, empty, big, scenes.lattice_scene(seed=33, n=2, dt=1e-3)]
    offsets, x, q, axes, vel, params = scenes.pack_scenes(scs)
    b = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    b.step(2)
    xb, _, vb = b.bodies()
    st = b.scene_stats()
    assert [s.steps_done for s in st] == [2, 2, 2, 2]
    # a lone body moves freely: x + 2 dt v (wrapped)
    exp = (one.x + 2 * one.dt * one.vel[:, :3]) % one.box
    assert np.abs(xb[0:1] - exp).max() <= 1e-12
    # too many bodies in one scene, bad parameters: rejected before any work
    offs_bad = np.array([0, 1025], dtype=np.int32)
    xs = np.zeros((1025, 3))
    qs = np.tile([1.0, 0, 0, 0], (1025, 1))
    with pytest.raises(R.RelcpError):
        b.set_scenes(offs_bad, xs, qs, np.ones((1025, 3)), np.tile(params[:1], (1, 1)))
    bad = params.copy()
    bad[0, 3] = 0.0
    with pytest.raises(R.RelcpError):
        b.set_scenes(offsets, x, q, axes, bad, vel=vel)
    with pytest.raises(R.RelcpError):
        b.set_threads(48)
    b.close()


def test_batch_capacity_keeps_state(relcp_gpu):
    """A scene with more candidate pairs than its capacity (16 n + 32) reports
    RELCP_ERR_CAPACITY and keeps its state; the other scenes step normally."""
    R = relcp_gpu
    rng = np.random.default_rng(41)
    n = 40
    clump = scenes.Scene(x=5.0 + 0.01 * rng.standard_normal((n, 3)), q=scenes.random_quaternions(rng, n),
                         axes=np.full((n, 3), 0.5), vel=np.zeros((n, 6)), fext=np.zeros((n, 6)),
                         box=np.array([10.0] * 3), dt=1e-3)
    ok = scenes.lattice_scene(seed=42, n=27, dt=1e-3)
    offsets, x, q, axes, vel, params = scenes.pack_scenes([clump, ok])
    b = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    assert b.step(3, allow=(R.RELCP_ERR_CAPACITY,)) == R.RELCP_ERR_CAPACITY
    xb, qb, _ = b.bodies()
    st = b.scene_stats()
    assert st[0].status == R.RELCP_ERR_CAPACITY and st[0].steps_done == 0
    assert np.array_equal(xb[:n], x[:n])
    assert st[1].status == 0 and st[1].steps_done == 3
    b.close()


def test_batch_autotune_and_cache(relcp_gpu, tmp_path):
    R = relcp_gpu
    scs = scenes.batched_scenes(n_scenes=64, seed0=500, nmax=256)
    offsets, x, q, axes, vel, params = scenes.pack_scenes(scs)
    b = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    x0, q0, _ = b.bodies()
    path = tmp_path / "tune.json"
    t = b.autotune(str(path))
    assert t in (64, 128, 256, 512)
    cache = json.loads(path.read_text())
    assert list(cache.values()) == [t]
    # timing restored the scenes' state
    x1, q1, _ = b.bodies()
    assert np.array_equal(x0, x1) and np.array_equal(q0, q1)
    assert all(s.steps_done == 0 for s in b.scene_stats())
    # a second tuner call reads the cache
    b2 = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b2.set_scenes(offsets, x, q, axes, params, vel=vel)
    assert b2.autotune(str(path)) == t
    # same block size, same result, bit for bit
    b.step(2)
    b2.step(2)
    for a, c in zip(b.bodies(), b2.bodies()):
        assert np.array_equal(a, c)
    b.close()
    b2.close()


def test_batched_workload_sample(relcp_gpu, orc):
    """The 2,048-scene workload (bodies log-uniform in [2, 512]) for a few
    steps in one launch: every scene steps, keeps its overlap within eps_NCP,
    and a sample of its scenes matches the oracle's first step."""
    R = relcp_gpu
    scs = scenes.batched_scenes(n_scenes=2048)
    offsets, x, q, axes, vel, params = scenes.pack_scenes(scs)
    b = R.Batch(R.make_config(dynamics=R.RELCP_INERTIAL, precision=R.RELCP_MIXED))
    b.set_scenes(offsets, x, q, axes, params, vel=vel)
    b.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    xb, qb, vb = b.bodies()
    st = b.scene_stats()
    assert all(s.steps_done == 1 for s in st)
    assert all(s.max_overlap <= params[i, 4] for i, s in enumerate(st))
    rng = np.random.default_rng(7)
    small = [s for s, sc in enumerate(scs) if sc.n <= 40]
    large = [s for s, sc in enumerate(scs) if sc.n >= 200]
    picks = list(rng.choice(small, size=4, replace=False)) + list(rng.choice(large, size=4, replace=False))
    for s in picks:
        sc = scs[s]
        amin = float(sc.axes.min())
        ocfg = orc.Config(dynamics=orc.INERTIAL, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
        ref = orc.step(ocfg, sc.x, sc.q, sc.axes, sc.vel)
        sl = slice(offsets[s], offsets[s + 1])
        pairs, ids = b.contacts(s)
        assert np.array_equal(pairs, ref.pairs), s
        assert np.array_equal(ids, np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1)), s
        assert rel_err(vb[sl], ref.vel) <= 1e-5
    b.step(4, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    st = b.scene_stats()
    assert all(s.steps_done == 5 for s in st)
    assert all(s.max_overlap <= params[i, 4] for i, s in enumerate(st))
    b.close()
