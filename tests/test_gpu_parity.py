"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated here, derived in the design notes):
  * candidate pairs and constraint index sets: bit-exact;
  * FP64 path: normwise relative 1e-9 on velocities and gamma
    (max |a - b| <= 1e-9 max |b|), SNSD Phi/n/r to 1e-10;
  * mixed path: normwise relative 1e-5, and the accepted configuration's
    max overlap <= eps_NCP.
Decisions that sit within 1e-9 of a threshold in the oracle are reported as
ambiguous; the seeded cases below have none (asserted).
"""
import numpy as np
import pytest
import torch

from paper_2506_14097_gb300 import scenes

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if b.size == 0:
        return 0.0
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def cfg_pair(R, orc, sc, dynamics, precision, dt=None, **kw):
    amin = float(sc.axes.min())
    dt = sc.dt if dt is None else dt
    base = dict(dynamics=dynamics, dt=dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
    base.update(kw)
    ocfg = orc.Config(**{k: v for k, v in base.items() if k in orc.Config.__dataclass_fields__})
    gkw = dict(base)
    gkw["precision"] = precision
    gkw["length_scale"] = amin
    gcfg = R.make_config(**gkw)
    return ocfg, gcfg


# ---------------------------------------------------------------------------
# broad phase
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,side,skin", [(0, 10.0, 0.1), (1, 10.0, 0.1), (300, 12.0, 0.05), (5000, 40.0, 0.04),
                                         (20000, 55.0, 0.05), (32768, 30.0, 0.05)])
def test_broadphase_bitexact(relcp_gpu, orc, n, side, skin):
    R = relcp_gpu
    rng = np.random.default_rng(100 + n)
    x = rng.random((n, 3)) * side
    rb = rng.uniform(0.4, 1.0, n)
    box = np.array([side] * 3)
    ref = orc.candidate_pairs(x, rb, box, skin)
    got = R.relcp_broadphase(dev(x), dev(rb), box, skin).cpu().numpy()
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_broadphase_open_box_and_threshold(relcp_gpu, orc):
    R = relcp_gpu
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 3.0000001, 0.0], [0.1, 0.2, 1.5]])
    rb = np.array([0.75, 0.75, 0.75, 0.5])
    ref = orc.candidate_pairs(x, rb, np.zeros(3), 0.5)
    got = R.relcp_broadphase(dev(x), dev(rb), np.zeros(3), 0.5).cpu().numpy()
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# SNSD
# ---------------------------------------------------------------------------
def random_pairs_scene(rng, n, side):
    x = rng.random((n, 3)) * side
    q = scenes.random_quaternions(rng, n)
    axes = rng.uniform(0.4, 1.0, (n, 3))
    return x, q, axes


@pytest.mark.parametrize("precision,tol,vtol", [(0, 1e-10, 1e-7), (1, 1e-9, 1e-5)])
def test_snsd_parity(relcp_gpu, orc, precision, tol, vtol):
    """FP64: Phi, n and the lever arms to FP64 accuracy.  Mixed: n and the
    lever arms at FP32 Newton accuracy (relative 1e-5), Phi still to 1e-9
    because the FP64 polish evaluates G at the FP32 maximiser, where G is
    stationary."""
    R = relcp_gpu
    rng = np.random.default_rng(7)
    x, q, axes = random_pairs_scene(rng, 400, 9.0)
    box = np.array([9.0] * 3)
    pairs = orc.candidate_pairs(x, axes.max(axis=1), box, 0.3)
    assert pairs.shape[0] > 200
    phi, n, ra, rb, fl = orc.snsd(pairs, x, q, axes, box)
    assert fl.max() == 0
    out, iters = R.relcp_snsd_eval(dev(pairs, torch.int32), dev(x), dev(q), dev(axes), box, precision)
    out = out.cpu().numpy()
    assert (iters.cpu().numpy() >= 0).all()
    assert np.abs(out[:, 0] - phi).max() <= tol * (1 + np.abs(phi).max())
    assert np.abs(out[:, 1:4] - n).max() <= vtol
    assert np.abs(out[:, 4:7] - ra).max() <= vtol
    assert np.abs(out[:, 7:10] - rb).max() <= vtol
    # overlapping pairs are present and agree in sign
    assert (phi < 0).sum() > 10
    assert np.array_equal(out[:, 0] < 0, phi < 0)


def test_snsd_spheres_closed_form(relcp_gpu):
    R = relcp_gpu
    rng = np.random.default_rng(8)
    n = 200
    x = rng.random((n, 3)) * 6.0
    r = rng.uniform(0.3, 1.0, n)
    axes = np.repeat(r[:, None], 3, axis=1)
    q = scenes.random_quaternions(rng, n)
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, n)][:3000], dtype=np.int32)
    out, _ = R.relcp_snsd_eval(dev(pairs, torch.int32), dev(x), dev(q), dev(axes), np.zeros(3), 0)
    out = out.cpu().numpy()
    d = x[pairs[:, 1]] - x[pairs[:, 0]]
    L = np.linalg.norm(d, axis=1)
    assert np.abs(out[:, 0] - (L - r[pairs[:, 0]] - r[pairs[:, 1]])).max() < 1e-12 * (1 + L.max())


# ---------------------------------------------------------------------------
# one LCP from identical rows
# ---------------------------------------------------------------------------
def contact_rows_from_scene(orc, sc, dt, dynamics):
    """A_0 rows of a scene built with the oracle, with K and q."""
    amin = float(sc.axes.min())
    box = np.asarray(sc.box)
    kt, Kr = orc.operator_K(dynamics, dt, sc.q, sc.axes)
    pairs = orc.candidate_pairs(sc.x, sc.axes.max(axis=1), box, 0.1 * amin)
    phi, n, ra, rb, _ = orc.snsd(pairs, sc.x, sc.q, sc.axes, box)
    keep = phi <= 0.1 * amin
    ia, ib = pairs[keep, 0].astype(np.int64), pairs[keep, 1].astype(np.int64)
    nn = n[keep]
    ta, tb = np.cross(ra[keep], nn), np.cross(rb[keep], nn)
    U = orc.free_velocity(orc.Config(dynamics=dynamics, dt=dt, box=tuple(box)), sc.x, sc.vel, sc.fext, kt, Kr, box)
    qv = phi[keep] + dt * orc.rows_dot_U(ia, ib, nn, ta, tb, U)
    K7 = np.stack([kt, Kr[:, 0, 0], Kr[:, 1, 1], Kr[:, 2, 2], Kr[:, 0, 1], Kr[:, 0, 2], Kr[:, 1, 2]], axis=1)
    return ia, ib, nn, ta, tb, qv, kt, Kr, K7


@pytest.mark.parametrize("precision", [0, 1])
def test_lcp_parity(relcp_gpu, orc, precision):
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=3, n=125, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    dt = 1e-2
    ia, ib, nn, ta, tb, qv, kt, Kr, K7 = contact_rows_from_scene(orc, sc, dt, orc.INERTIAL)
    m = ia.size
    assert m > 20
    A = orc.dense_A(dt, kt, Kr, ia, ib, nn, ta, tb)
    gam_ref, w, st, _ = orc.lemke(A, qv)
    assert st == 0
    Uc_ref = orc.apply_K(kt, Kr, orc.wrench(sc.n, ia, ib, nn, ta, tb, gam_ref))
    geom = np.concatenate([nn, ta, tb], axis=1)
    tol = 1e-13 if precision == 0 else 1e-8
    gam, uc, info = R.relcp_lcp_solve(dev(ia, torch.int32), dev(ib, torch.int32), dev(geom), dev(qv), dev(K7), dt,
                                      precision=precision, tol=tol, max_iter=200000)
    gam, uc = gam.cpu().numpy(), uc.cpu().numpy()
    assert info.status == 0, (info.iterations, info.residual)
    bound = 1e-9 if precision == 0 else 1e-5
    assert rel_err(uc, Uc_ref) <= bound, (rel_err(uc, Uc_ref), info.iterations)
    # gamma is unique here (A positive definite on this instance)
    if np.linalg.eigvalsh(A).min() > 1e-8 * np.abs(A).max():
        assert rel_err(gam, gam_ref) <= bound
    # complementarity of the GPU result, checked with the oracle's A
    g = A @ gam + qv
    assert gam.min() >= 0 and g.min() >= -10 * tol


@pytest.mark.parametrize("nb", [30000, 60000])
def test_lcp_large_random_complementarity(relcp_gpu, nb):
    """A random contact LCP with 3 rows per body, solved on the mixed path at a
    size where every row has its own thread (30,000 bodies, 90,000 rows: the
    iterations with one grid barrier) and one where rows outnumber the threads
    (60,000 bodies, 180,000 rows: the two-barrier iterations).  Too large for
    the oracle's Lemke: checked by the properties of the solution, in FP64 on
    the host: gamma >= 0, g = q + A gamma >= -tol, complementarity within the
    tolerance, and the returned contact velocity equal to K D^T gamma."""
    import scipy.sparse as sp

    R = relcp_gpu
    rng = np.random.default_rng(nb)
    m = 3 * nb
    ia = np.repeat(np.arange(nb), 3)
    ib = (ia + rng.integers(1, nb, size=m)) % nb
    nn = rng.standard_normal((m, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    ta = np.cross(0.5 * rng.standard_normal((m, 3)), nn)
    tb = np.cross(0.5 * rng.standard_normal((m, 3)), nn)
    kt, kr, c = 1.0, 12.0, 1e-2
    qv = rng.uniform(-0.02, 0.05, m)
    K7 = np.tile(np.array([kt, kr, kr, kr, 0.0, 0.0, 0.0]), (nb, 1))
    tol = 1e-6
    geom = np.concatenate([nn, ta, tb], axis=1)
    gam, uc, info = R.relcp_lcp_solve(dev(ia, torch.int32), dev(ib, torch.int32), dev(geom), dev(qv), dev(K7), c,
                                      precision=R.RELCP_MIXED, tol=tol, max_iter=20000)
    gam, uc = gam.cpu().numpy(), uc.cpu().numpy()
    assert info.status == 0, (info.iterations, info.residual)
    # the path taken: one grid barrier per iteration exactly when every row
    # has a thread of its own (152 SMs x 640 threads = 97,280 slots on GB300)
    assert info.one_barrier == int(m <= info.grid_blocks * 640)
    if torch.cuda.get_device_properties(0).multi_processor_count >= 152:
        assert info.one_barrier == (1 if nb == 30000 else 0)
    rows = np.repeat(np.arange(m), 12)
    cols = np.concatenate([6 * ia[:, None] + np.arange(6), 6 * ib[:, None] + np.arange(6)], 1).ravel()
    D = sp.csr_matrix((np.concatenate([-nn, -ta, nn, tb], 1).ravel(), (rows, cols)), shape=(m, 6 * nb))
    Kd = np.tile(np.array([kt, kt, kt, kr, kr, kr]), nb)
    U = Kd * (D.T @ gam)
    g = qv + c * (D @ U)
    Aaa = c * (2 * kt + kr * (ta ** 2).sum(1) + kr * (tb ** 2).sum(1))
    assert gam.min() >= 0.0
    assert g.min() >= -10 * tol
    assert np.abs(np.minimum(Aaa * gam, g)).max() <= 10 * tol
    assert rel_err(uc, U.reshape(nb, 6)) <= 1e-5


def test_lcp_empty_and_zero_rows(relcp_gpu):
    R = relcp_gpu
    K7 = dev(np.ones((3, 7)))
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    gam, uc, info = R.relcp_lcp_solve(e, e, torch.zeros((0, 9), dtype=torch.float64, device="cuda"),
                                      torch.zeros(0, dtype=torch.float64, device="cuda"), K7, 1e-3)
    assert gam.numel() == 0 and float(uc.abs().max()) == 0.0 and info.iterations == 0


# ---------------------------------------------------------------------------
# full steps from identical states
# ---------------------------------------------------------------------------
def compare_step(R, orc, sc, ocfg, gcfg, vel=None, fext=None, bound=1e-9):
    ref = orc.step(ocfg, sc.x, sc.q, sc.axes, vel, fext)
    assert ref.ambiguous == 0 and ref.status == 0
    sim = R.Simulation(gcfg)
    sim.set_bodies(np.ascontiguousarray(sc.x), np.ascontiguousarray(sc.q), np.ascontiguousarray(sc.axes),
                   None if vel is None else np.ascontiguousarray(vel),
                   None if fext is None else np.ascontiguousarray(fext))
    st = sim.step(1)
    assert st == 0
    stats = sim.stats()
    pairs, phi0 = R.relcp_get_pairs(sim.ctx)
    assert np.array_equal(pairs, ref.pairs)
    assert np.abs(phi0 - ref.phi0).max() <= 1e-10 * (1 + np.abs(ref.phi0).max()) if ref.phi0.size else True
    ids, geom, gam = R.relcp_get_rows(sim.ctx)
    assert stats.depth == ref.depth
    ref_ids = np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1)
    assert np.array_equal(ids, ref_ids)
    x, q, v = sim.bodies()
    assert rel_err(v, ref.vel) <= bound, rel_err(v, ref.vel)
    dx = orc.min_image(x - ref.x, np.asarray(ref.box))
    assert np.abs(dx).max() <= bound * (1 + np.abs(ref.x).max())
    qs = np.sign(np.sum(q * ref.q, axis=1))[:, None]
    assert np.abs(q - qs * ref.q).max() <= bound
    if ref.gamma.size:
        uc = R.relcp_get_contact_velocity(sim.ctx, sc.n)
        assert rel_err(uc, ref.U_contact) <= bound
    assert stats.max_overlap <= ocfg.eps_ncp
    sim.close()
    return ref, stats


@pytest.mark.parametrize("precision,bound", [(0, 1e-9), (1, 1e-5)])
def test_step_parity_inertial_with_recursion(relcp_gpu, orc, precision, bound):
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=2, n=64, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    ocfg, gcfg = cfg_pair(R, orc, sc, orc.INERTIAL, precision)
    x, q, v = sc.x, sc.q, sc.vel
    depths = []
    for k in range(12):
        sck = scenes.Scene(x=x, q=q, axes=sc.axes, vel=v, fext=sc.fext, box=sc.box, dt=sc.dt)
        ref, stats = compare_step(R, orc, sck, ocfg, gcfg, vel=v, bound=bound)
        depths.append(ref.depth)
        x, q, v = ref.x, ref.q, ref.vel
    assert max(depths) >= 1


def test_step_parity_overdamped_two_ellipsoids(relcp_gpu, orc):
    R = relcp_gpu
    sc = scenes.two_ellipsoid_scene(offset_y=4.2)
    ocfg = orc.Config(dynamics=orc.OVERDAMPED, dt=0.1, eps_ncp=1e-5, box=(0, 0, 0), skin=0.5)
    gcfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, dt=0.1, eps_ncp=1e-5, box=(0, 0, 0), skin=0.5,
                         length_scale=1.0)
    x, q = sc.x, sc.q
    for k in range(40):
        r = orc.step(ocfg, x, q, sc.axes, None, sc.fext)
        if k >= 22:
            sck = scenes.Scene(x=x, q=q, axes=sc.axes, vel=np.zeros((2, 6)), fext=sc.fext, box=sc.box, dt=0.1)
            ref, stats = compare_step(R, orc, sck, ocfg, gcfg, fext=sc.fext)
        x, q = r.x, r.q
    assert stats.depth >= 1


def test_step_parity_compacting_suspension(relcp_gpu, orc):
    R = relcp_gpu
    sc = scenes.suspension_scene(seed=1, n=256, phi=0.1, steps=300, dt=5e-3)
    amin = float(sc.axes.min())
    rate = sc.meta["strain_rate"]
    ocfg = orc.Config(dynamics=orc.OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin,
                      strain_rate=rate)
    x, q, box = sc.x, sc.q, np.asarray(sc.box)
    # advance with the oracle to a dense state, then compare single steps
    for k in range(260):
        r = orc.step(orc.Config(**{**ocfg.__dict__, "box": tuple(box)}), x, q, sc.axes)
        x, q, box = r.x, r.q, r.box
    for k in range(3):
        oc = orc.Config(**{**ocfg.__dict__, "box": tuple(box)})
        gcfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(box),
                             skin=0.1 * amin, strain_rate=rate, length_scale=amin)
        sck = scenes.Scene(x=x, q=q, axes=sc.axes, vel=np.zeros((sc.n, 6)), fext=np.zeros((sc.n, 6)), box=box,
                           dt=sc.dt)
        ref, stats = compare_step(R, orc, sck, oc, gcfg)
        assert ref.rows_ia.size > 100
        x, q, box = ref.x, ref.q, ref.box
    # the same state translated by s and wrapped into the box: the wrapped
    # bodies' background velocities change by multiples of strain_rate x L,
    # which the minimum-image offsets of their pairs must cancel; the GPU step
    # matches the oracle's from the shifted state, and its gamma per row and
    # contact velocities equal those of the unshifted state
    oc = orc.Config(**{**ocfg.__dict__, "box": tuple(box)})
    gcfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(box),
                         skin=0.1 * amin, strain_rate=rate, length_scale=amin)
    out = []
    for s_ in (np.zeros(3), np.array([0.37, 0.61, 0.5]) * box):
        xs = x + s_
        xs -= box * np.floor(xs / box)
        sck = scenes.Scene(x=xs, q=q, axes=sc.axes, vel=np.zeros((sc.n, 6)), fext=np.zeros((sc.n, 6)), box=box,
                           dt=sc.dt)
        ref, stats = compare_step(R, orc, sck, oc, gcfg)
        sim = R.Simulation(gcfg)
        sim.set_bodies(np.ascontiguousarray(xs), np.ascontiguousarray(q), np.ascontiguousarray(sc.axes))
        sim.step(1)
        ids, _, gam = R.relcp_get_rows(sim.ctx)
        out.append((ids, gam, R.relcp_get_contact_velocity(sim.ctx, sc.n), sim.bodies()[0], s_))
        sim.close()
    (ids0, g0, u0, x0, _), (ids1, g1, u1, x1, s1) = out
    assert np.array_equal(ids0, ids1)
    assert rel_err(g1, g0) <= 1e-9 and rel_err(u1, u0) <= 1e-9
    box1 = box * (1 + rate * sc.dt)
    d = x1 - s1 * (1 + rate * sc.dt) - x0
    d -= box1 * np.rint(d / box1)
    assert np.abs(d).max() <= 1e-12 * box1.max()


def test_cached_pair_list_bitexact_over_steps(relcp_gpu, orc):
    """Every step's candidate pairs (served from the cached Verlet list with
    its displacement bound, rebuilt when needed) equal the oracle's brute
    force on the same positions, bit for bit, across a fast compaction."""
    R = relcp_gpu
    sc = scenes.suspension_scene(seed=4, n=3000, phi=0.1, phi_final=0.5, steps=120, dt=5e-3)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, dt=sc.dt, eps_ncp=1e-3 * amin,
                        box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"], length_scale=amin)
    sim = R.Simulation(cfg)
    sim.set_bodies(sc.x, sc.q, sc.axes)
    rb = sc.axes.max(axis=1)
    rebuilt = 0
    for k in range(100):
        x, q, _ = sim.bodies()
        box = R.relcp_get_box(sim.ctx)
        sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        rebuilt += sim.stats().pair_list_rebuilt
        pairs, _ = R.relcp_get_pairs(sim.ctx)
        ref = orc.candidate_pairs(x, rb, box, 0.1 * amin)
        assert np.array_equal(pairs, ref), k
    assert 1 <= rebuilt < 100
    sim.close()


def test_cached_pair_list_bitexact_32k(relcp_gpu, orc):
    """At the benchmark's size and density the cached list's fused filter and
    compaction runs over more than 32 look-back tiles of 1024 entries (several
    look-back windows); its pairs equal the oracle's brute force on the same
    positions, bit for bit."""
    R = relcp_gpu
    sc = scenes.suspension_scene(seed=23, n=32768, phi=0.1, phi_final=0.45, steps=60, dt=5e-3)
    amin = float(sc.axes.min())
    # (a strain of 1% per step: FP32 iterates stall above the overdamped
    # default stop of 1e-8 a_min; the pairs, not the LCP, are tested here)
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, dt=sc.dt, eps_ncp=1e-3 * amin,
                        box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"], length_scale=amin,
                        lcp_tol=1e-7 * amin)
    sim = R.Simulation(cfg)
    sim.set_bodies(sc.x, sc.q, sc.axes)
    sim.step(57, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    # hold the box from here on, so that the following steps serve their
    # pairs from the cached list (the first one after the change re-checks it)
    box = R.relcp_get_box(sim.ctx)
    for k in range(3):
        cfg.box[k] = box[k]
    cfg.strain_rate = 0.0
    R.relcp_set_config(sim.ctx, cfg)
    sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    rb = sc.axes.max(axis=1)
    cached = 0
    for _ in range(2):
        x, q, _ = sim.bodies()
        box = R.relcp_get_box(sim.ctx)
        sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        cached += sim.stats().pair_list_rebuilt == 0
        pairs, _ = R.relcp_get_pairs(sim.ctx)
        ref = orc.candidate_pairs(x, rb, box, 0.1 * amin)
        assert ref.shape[0] > 40 * 1024
        assert np.array_equal(pairs, ref)
    assert cached >= 1
    sim.close()


# ---------------------------------------------------------------------------
# edge cases and error paths
# ---------------------------------------------------------------------------
def test_empty_and_single_body(relcp_gpu):
    R = relcp_gpu
    cfg = R.make_config(dt=1e-3, eps_ncp=1e-3, box=(10, 10, 10), skin=0.05)
    sim = R.Simulation(cfg)
    sim.set_bodies(np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 3)))
    assert sim.step(3) == 0
    sim.set_bodies(np.array([[1.0, 2.0, 3.0]]), np.array([[1.0, 0, 0, 0]]), np.array([[0.5, 0.6, 0.7]]),
                   np.array([[1.0, 0, 0, 0, 0, 0]]))
    assert sim.step(1) == 0
    x, q, v = sim.bodies()
    assert abs(x[0, 0] - 1.001) < 1e-15 and sim.stats().n_pairs == 0
    sim.close()


@pytest.mark.parametrize("staging", [False, True], ids=["in_place", "pinned_staging"])
def test_invalid_arguments_rejected(relcp_gpu, staging):
    R = relcp_gpu
    cfg = R.make_config(dt=1e-3, eps_ncp=1e-3, box=(10, 10, 10), skin=0.05,
                        flags=R.RELCP_FLAG_HOST_STAGING if staging else 0)
    sim = R.Simulation(cfg)
    x = np.array([[1.0, 2.0, 3.0]])
    with pytest.raises(R.RelcpError) as e:
        sim.set_bodies(x, np.array([[2.0, 0, 0, 0]]), np.array([[0.5, 0.6, 0.7]]))
    assert e.value.status == R.RELCP_ERR_INVALID_ARG
    with pytest.raises(R.RelcpError):
        sim.set_bodies(np.array([[np.nan, 0, 0]]), np.array([[1.0, 0, 0, 0]]), np.array([[0.5, 0.6, 0.7]]))
    with pytest.raises(R.RelcpError):
        sim.set_bodies(x, np.array([[1.0, 0, 0, 0]]), np.array([[0.5, -0.6, 0.7]]))
    bad = R.make_config(dt=-1.0)
    with pytest.raises(R.RelcpError):
        R.relcp_create(bad)
    sim2 = R.Simulation(cfg)
    with pytest.raises(R.RelcpError) as e:
        sim2.step(1)
    assert e.value.status == R.RELCP_ERR_STATE
    sim.close()
    sim2.close()


@pytest.mark.parametrize("staging", [False, True], ids=["in_place", "pinned_staging"])
def test_rejected_bodies_leave_state_untouched(relcp_gpu, staging):
    """Invalid body input names the first invalid body and changes nothing:
    stepping on afterwards is bit for bit stepping without the call."""
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=4, n=512, spacing=1.9, dt=1e-2, vel_sigma=2.0, omega_sigma=1.0)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box),
                        skin=0.1 * amin, length_scale=amin, flags=R.RELCP_FLAG_HOST_STAGING if staging else 0)
    a, b = R.Simulation(cfg), R.Simulation(cfg)
    for s_ in (a, b):
        s_.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        s_.step(3)
    cases = []
    q = sc.q.copy()
    q[300] *= 1.5
    q[450] *= 2.0
    cases.append(((sc.x, q, sc.axes, sc.vel), "body 300: quaternion"))
    x = sc.x.copy()
    x[77, 1] = np.inf
    cases.append(((x, sc.q, sc.axes, sc.vel), "body 77: position"))
    ax = sc.axes.copy()
    ax[200, 2] = 0.0
    x2 = sc.x.copy()
    x2[201, 0] = np.nan
    cases.append(((x2, sc.q, ax, sc.vel), "body 200: semi-axes"))
    v = sc.vel.copy()
    v[5, 4] = np.nan
    cases.append(((sc.x, sc.q, sc.axes, v), "body 5: velocity"))
    for args, msg in cases:
        with pytest.raises(R.RelcpError) as e:
            b.set_bodies(*args)
        assert e.value.status == R.RELCP_ERR_INVALID_ARG and msg in str(e.value)
    a.step(3)
    b.step(3)
    for u, w in zip(a.bodies(), b.bodies()):
        assert np.array_equal(u, w)
    a.close()
    b.close()


def test_device_body_io_matches_host(relcp_gpu):
    """Body state given and read back as device arrays steps bit for bit as
    the same state given and read back as host arrays."""
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=6, n=700, spacing=1.9, dt=1e-2, vel_sigma=2.0, omega_sigma=1.0)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box),
                        skin=0.1 * amin, length_scale=amin)
    a, b = R.Simulation(cfg), R.Simulation(cfg)
    a.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
    R.relcp_set_bodies(b.ctx, dev(sc.x), dev(sc.q), dev(sc.axes), dev(sc.vel))
    b.n = sc.x.shape[0]
    a.step(4)
    b.step(4)
    xd = torch.zeros((b.n, 3), dtype=torch.float64, device="cuda")
    qd = torch.zeros((b.n, 4), dtype=torch.float64, device="cuda")
    vd = torch.zeros((b.n, 6), dtype=torch.float64, device="cuda")
    R.relcp_get_bodies(b.ctx, xd, qd, vd)
    for u, w in zip(a.bodies(), (xd, qd, vd)):
        assert np.array_equal(u, w.cpu().numpy())
    a.close()
    b.close()


def test_fault_injection_and_caps(relcp_gpu, orc):
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=2, n=64, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    amin = float(sc.axes.min())
    base = dict(dynamics=R.RELCP_INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin,
                length_scale=amin)
    for fault, expect in ((R.RELCP_FAULT_ROW_CAPACITY, R.RELCP_ERR_CAPACITY),
                          (R.RELCP_FAULT_LCP_ITERS, R.RELCP_ERR_NOT_CONVERGED)):
        sim = R.Simulation(R.make_config(fault_inject=fault, **base))
        sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        assert sim.step(1, allow=(expect,)) == expect
        sim.close()
    # recursion cap 0 reports the limit when the full method would augment
    x, q, v = sc.x, sc.q, sc.vel
    ocfg = orc.Config(dynamics=orc.INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
    while True:
        r = orc.step(ocfg, x, q, sc.axes, v)
        if r.depth >= 1:
            break
        x, q, v = r.x, r.q, r.vel
    sim = R.Simulation(R.make_config(max_recursion=0, **base))
    sim.set_bodies(x, q, sc.axes, v)
    assert sim.step(1, allow=(R.RELCP_ERR_RECURSION_LIMIT,)) == R.RELCP_ERR_RECURSION_LIMIT
    ids, geom, gam = R.relcp_get_rows(sim.ctx)
    assert (ids[:, 2] == 0).all()
    sim.close()


def test_device_wait_timeout_reported(relcp_gpu, orc):
    """A block of the persistent LCP launch that never arrives at the grid
    barrier (host-set fault RELCP_FAULT_LCP_TIMEOUT: the launch's waits give
    up after 2 ms and its last block leaves before its first arrival): every
    other block's bounded wait runs out, the launch ends, and the step returns
    RELCP_ERR_TIMEOUT promptly.  The context stays usable: with the fault
    cleared the same state steps like the oracle, on both precision paths."""
    import time

    R = relcp_gpu
    sc = scenes.lattice_scene(seed=4, n=4096, spacing=1.9, dt=1e-2, vel_sigma=2.0, omega_sigma=1.0)
    for precision, bound in ((R.RELCP_FP64, 1e-9), (R.RELCP_MIXED, 1e-5)):
        ocfg, gcfg = cfg_pair(R, orc, sc, orc.INERTIAL, precision, fault_inject=R.RELCP_FAULT_LCP_TIMEOUT)
        sim = R.Simulation(gcfg)
        sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        t0 = time.perf_counter()
        st = sim.step(1, allow=(R.RELCP_ERR_TIMEOUT,))
        assert st == R.RELCP_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        assert "timed out" in R.last_error()
        gcfg.fault_inject = 0
        R.relcp_set_config(sim.ctx, gcfg)
        sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        assert sim.step(1) == R.RELCP_OK
        ref = orc.step(ocfg, sc.x, sc.q, sc.axes, sc.vel)
        assert ref.status == 0 and ref.rows_ia.size > 100
        ids, _, _ = R.relcp_get_rows(sim.ctx)
        assert np.array_equal(ids, np.stack([ref.rows_ia, ref.rows_ib, ref.rows_rec, ref.rows_pair], axis=1))
        x, q, v = sim.bodies()
        assert rel_err(v, ref.vel) <= bound
        sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_newton_failure_reported(relcp_gpu, precision):
    """With every SNSD Newton phase capped at one iteration (host-set fault
    RELCP_FAULT_NEWTON_ITERS) the pairs whose start is not already stationary
    do not converge: the step completes and reports RELCP_ERR_NEWTON; with the
    cap lifted the same state steps without error."""
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=2, n=64, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_INERTIAL, precision=precision, dt=1e-2, eps_ncp=1e-3 * amin,
                        box=tuple(sc.box), skin=0.1 * amin, length_scale=amin,
                        fault_inject=R.RELCP_FAULT_NEWTON_ITERS)
    sim = R.Simulation(cfg)
    sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
    assert sim.step(1, allow=(R.RELCP_ERR_NEWTON,)) == R.RELCP_ERR_NEWTON
    assert sim.stats().status == R.RELCP_ERR_NEWTON
    cfg.fault_inject = 0
    R.relcp_set_config(sim.ctx, cfg)
    sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
    assert sim.step(1) == R.RELCP_OK
    sim.close()


def test_deterministic_bitwise(relcp_gpu):
    R = relcp_gpu
    sc = scenes.lattice_scene(seed=2, n=64, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    amin = float(sc.axes.min())
    outs = []
    for rep in range(2):
        sim = R.Simulation(R.make_config(dynamics=R.RELCP_INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box),
                                         skin=0.1 * amin, length_scale=amin))
        sim.set_bodies(sc.x, sc.q, sc.axes, sc.vel)
        sim.step(10)
        outs.append(sim.bodies())
        sim.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_carried_c0_values_match_fresh_evaluation(relcp_gpu):
    """From the second step on a pair that was a candidate in the previous step
    takes its SNSD at C^k from that step's last overlap test, which evaluated
    it at the configuration the step accepted, and its warm-start gamma from
    the memo of the cached candidate list (carried across list rebuilds).
    Against evaluating every pair afresh (RELCP_FLAG_NO_SNSD_REUSE) the
    trajectory, the pair lists and the C^k signed distances agree within each
    path's tolerance; the warm start cuts the LCP iterations."""
    R = relcp_gpu
    sc = scenes.suspension_scene(seed=5, n=2048, phi=0.1, phi_final=0.45, steps=60, dt=5e-3)
    amin = float(sc.axes.min())
    # mixed: the relative 1e-5 of that path, on lengths scaled by the smallest semi-axis
    for prec, xtol, ptol in ((R.RELCP_FP64, 1e-9, 1e-10), (R.RELCP_MIXED, 1e-5 * amin, 1e-5 * amin)):
        outs = {}
        for flags in (0, R.RELCP_FLAG_NO_SNSD_REUSE, R.RELCP_FLAG_NO_WARM_START):
            cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=prec, dt=sc.dt, eps_ncp=1e-3 * amin,
                                box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"],
                                length_scale=amin, flags=flags)
            sim = R.Simulation(cfg)
            sim.set_bodies(sc.x, sc.q, sc.axes)
            ev, rebuilt, iters = [], 0, 0
            for _ in range(40):
                sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
                st = sim.stats()
                ev.append((st.snsd_c0_evaluated, st.n_pairs))
                rebuilt += st.pair_list_rebuilt
                iters += st.lcp_iters_total
            x, q, v = sim.bodies()
            box = np.asarray(R.relcp_get_box(sim.ctx))
            pairs, phi0 = R.relcp_get_pairs(sim.ctx)
            outs[flags] = (x, q, ev, rebuilt, iters, pairs, phi0)
            sim.close()
        (x0, q0, ev0, rb0, it0, p0, f0) = outs[0]
        (x1, q1, ev1, rb1, it1, p1, f1) = outs[R.RELCP_FLAG_NO_SNSD_REUSE]
        assert ev0[0][0] == ev0[0][1] and all(e == n for e, n in ev1)
        assert sum(e for e, _ in ev0[1:]) < 0.2 * sum(n for _, n in ev0[1:])
        assert rb0 >= 1  # the memo crossed at least one rebuild of the cached list
        dx = x0 - x1
        dx -= box * np.round(dx / box)
        assert np.abs(dx).max() <= xtol and np.abs(q0 - q1).max() <= xtol
        k0 = {tuple(p): f for p, f in zip(p0, f0)}
        common = [(k0[tuple(p)], f) for p, f in zip(p1, f1) if tuple(p) in k0]
        assert len(common) >= 0.99 * max(len(p0), len(p1))
        a, b = np.array(common).T
        assert np.abs(a - b).max() <= ptol
        assert it0 < outs[R.RELCP_FLAG_NO_WARM_START][4]


@pytest.mark.parametrize("learned_start", [False, True])
def test_graph_replay_matches_direct_launches(relcp_gpu, learned_start):
    """From the third steady step on, the first level of a step (broad-phase
    filter through the overlap test) is replayed from a captured CUDA graph
    whose kernels read the per-step box and stamp from device memory; the
    results equal, bit for bit, those of launching every kernel from the host
    (without RELCP_FLAG_GRAPH), and the replayed kernels are counted."""
    R = relcp_gpu
    from paper_2506_14097_gb300 import learned

    # a slow compaction: the cached pair list is rarely rebuilt, so most steps replay
    sc = scenes.suspension_scene(seed=6, n=2048, phi=0.15, phi_final=0.5, steps=2000, dt=5e-3)
    amin = float(sc.axes.min())
    params = learned.init_params(seed=3) if learned_start else None
    outs, launches = [], []
    replayed = []
    for flags in (R.RELCP_FLAG_GRAPH, 0):
        cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, dt=sc.dt, eps_ncp=1e-3 * amin,
                            box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"],
                            length_scale=amin, flags=flags | R.RELCP_FLAG_LCP_TIMING,
                            guess=R.RELCP_GUESS_MLP if learned_start else R.RELCP_GUESS_COLD)
        stream = torch.cuda.Stream()  # a capturable stream (not the legacy default stream)
        sim = R.Simulation(cfg, stream.cuda_stream)
        if learned_start:
            R.relcp_load_mlp(sim.ctx, params)
        sim.set_bodies(sc.x, sc.q, sc.axes)
        l0 = R.relcp_kernel_launches()
        ms = 0.0
        rep = 0
        for _ in range(40):
            sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
            ms += sim.stats().ms_lcp_kernel
            rep += sim.stats().graph_replayed
        replayed.append(rep)
        launches.append(R.relcp_kernel_launches() - l0)
        outs.append(sim.bodies() + (R.relcp_get_pairs(sim.ctx)[1],))
        assert ms > 0.0  # the LCP kernel events are recorded by the replayed graph too
        sim.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    assert launches[0] == launches[1]
    assert replayed[0] >= 10 and replayed[1] == 0


@pytest.mark.parametrize("staging", [False, True], ids=["in_place", "pinned_staging"])
def test_host_roundtrip_keeps_carried_state(relcp_gpu, staging):
    """relcp_set_bodies with the state relcp_get_bodies returned (and an
    unchanged config) keeps everything a step carries to the next: the
    trajectory is bit for bit that of stepping without the round trip and the
    carried SNSD values stay in use.  Moving one body drops the carried SNSD
    values; changing a semi-axis drops the cached pair list too."""
    R = relcp_gpu
    sc = scenes.suspension_scene(seed=7, n=2048, phi=0.15, phi_final=0.45, steps=200, dt=5e-3)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, dt=sc.dt, eps_ncp=1e-3 * amin,
                        box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"], length_scale=amin,
                        flags=R.RELCP_FLAG_HOST_STAGING if staging else 0)
    a = R.Simulation(cfg)
    a.set_bodies(sc.x, sc.q, sc.axes)
    for _ in range(20):
        a.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    b = R.Simulation(cfg)
    b.set_bodies(sc.x, sc.q, sc.axes)
    evals = []
    for _ in range(20):
        b.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        st = b.stats()
        evals.append((st.snsd_c0_evaluated, st.n_pairs))
        x, q, v = b.bodies()
        box = R.relcp_get_box(b.ctx)
        for k in range(3):
            cfg.box[k] = box[k]
        R.relcp_set_config(b.ctx, cfg)
        b.set_bodies(x, q, sc.axes)
    for u, w in zip(a.bodies()[:2], b.bodies()[:2]):
        assert np.array_equal(u, w)
    assert sum(e for e, _ in evals[1:]) < 0.2 * sum(n for _, n in evals[1:])
    # a moved body: the next C^k evaluates every pair again, while the cached
    # pair list (checked by its displacement bound) survives most such moves
    rebuilt = 0
    for _ in range(6):
        x, q, _ = b.bodies()
        x[0, 0] += 1e-9
        b.set_bodies(x, q, sc.axes)
        b.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
        st = b.stats()
        assert st.snsd_c0_evaluated == st.n_pairs
        rebuilt += st.pair_list_rebuilt
    assert rebuilt <= 2
    # a changed shape: the cached pair list is rebuilt
    x, q, _ = b.bodies()
    ax = sc.axes.copy()
    ax[0, 0] *= 1.01
    b.set_bodies(x, q, ax)
    b.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    assert b.stats().pair_list_rebuilt == 1
    a.close()
    b.close()


@pytest.mark.parametrize("precision,bound,tol", [(0, 1e-9, None), (1, 1e-5, 1e-8)])
def test_step_parity_spherocylinders(relcp_gpu, orc, precision, bound, tol):
    """Spherocylinders (the colony cells of Sec. 5.4) in a periodic box, pulled
    towards the box centre by a linear force (overdamped): one step from the
    same state on the GPU and in the oracle at each of 12 states along the
    oracle's trajectory (the recursion reaches depth 6), with pairs and
    constraint ids bit for bit.  Rows appended to pairs of flat-sided bodies
    nearly repeat earlier rows, so the LCP is close to singular: the FP64 path
    needs up to ~6x10^4 projected-gradient iterations, and plain FP32 iterates
    stall near a residual of 1e-7 (the pull towards the centre makes the
    contact velocities large against their differences); the mixed path's
    iterative refinement reaches a stop of 1e-8 and the mixed bound 1e-5."""
    R = relcp_gpu
    rng = np.random.default_rng(61)
    n, side = 80, 11.0
    rho = rng.uniform(0.3, 0.5, n)
    h = rng.uniform(0.2, 0.9, n)
    axes = np.stack([h + rho, rho, rho], axis=1)
    x = scenes._rsa_positions(rng, axes[:, 0], side, max_attempts=500 * n)
    q = scenes.random_quaternions(rng, n)
    box = np.full(3, side)
    fext = np.zeros((n, 6))
    fext[:, :3] = -(x - side / 2) * 2.0
    amin = float(rho.min())
    ocfg = orc.Config(dynamics=orc.OVERDAMPED, dt=0.05, eps_ncp=1e-3 * amin, box=tuple(box), skin=0.1 * amin,
                      shape=orc.SHAPE_SPHEROCYLINDER)
    gcfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=precision, dt=0.05, eps_ncp=1e-3 * amin,
                         box=tuple(box), skin=0.1 * amin, length_scale=amin, shape=R.RELCP_SHAPE_SPHEROCYLINDER,
                         lcp_tol=tol, lcp_max_iter=200000)
    rows, depth = 0, 0
    for k in range(12):
        sck = scenes.Scene(x=x, q=q, axes=axes, vel=np.zeros((n, 6)), fext=fext, box=box, dt=0.05)
        ref, stats = compare_step(R, orc, sck, ocfg, gcfg, fext=fext, bound=bound)
        rows += ref.rows_ia.size
        depth = max(depth, ref.depth)
        x, q = ref.x, ref.q
    assert rows > 500 and depth >= 3  # the flat sides make the recursion append rows
