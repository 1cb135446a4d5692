"""Pins of the oracle's time step (Algorithm 1, Eq. relcp, Eq. relcp_inertial)
against what the paper and mechanics fix:

* sphere-only scenes never augment (orthogonal motion cannot create overlap
  between spheres, Sec. 2.1.4; the true gap of two spheres is never below the
  linearised gap);
* the recursion collapses to the single-constraint SNSD-LCP as dt -> 0
  (Corollary "reduction to single-constraint SNSD-LCP"; Sec. 5.2);
* W_n = gamma_n^T A_n gamma_n is nondecreasing over the recursion (proof of
  the finite-termination theorem);
* after acceptance the maximum overlap is at most eps_NCP (Eq.
  gap_stopping_rule) and every LCP is complementary;
* contact impulses conserve linear momentum exactly and angular momentum up
  to the SNSD accuracy (y_b - y_a = Phi n);
* head-on equal spheres: perfectly inelastic closed form (Sec. 2.1.4);
* overdamped balanced pair: gamma equals the applied force;
* the linearised separation of a row predicts the true separation at the
  trial configuration with an O(dt^2) error (Eq. linear_sep);
* recursion capped at 0 equals the LCP-SNSD solve;
* a row appended at recursion j is the linearisation of Phi at C_j pulled
  back to C^k (Sec. 3.1.3): its modelled gap equals Phi(C_j) at the solve
  that produced C_j and follows the true Phi to first order along the later
  solves;
* the affine compaction of a periodic box has no preferred origin: a common
  translation with wrapping changes nothing but the positions, and free
  bodies scale with the box;
* quaternion update and mass properties against exact rotation and Monte
  Carlo integration.
"""
import itertools

import numpy as np
import pytest

from paper_2506_14097_gb300 import scenes


def enum_solver(A, q):
    n = q.shape[0]
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            z = np.zeros(n)
            if S:
                zS = np.linalg.lstsq(A[np.ix_(S, S)], -q[S], rcond=None)[0]
                if np.linalg.norm(A[np.ix_(S, S)] @ zS + q[S]) > 1e-10 * (1 + abs(q).max()) or zS.min() < -1e-12:
                    continue
                z[S] = np.maximum(zS, 0)
            if (A @ z + q).min() >= -1e-11 * (1 + abs(q).max()):
                return z
    raise AssertionError("no LCP solution found by enumeration")


def cfg_for(orc, sc, dynamics, **kw):
    amin = float(sc.axes.min())
    base = dict(dynamics=dynamics, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
    base.update(kw)
    return orc.Config(**base)


def test_spheres_never_augment(orc):
    sc = scenes.sphere_scene(seed=3, n=120, side=9.0, vel_sigma=3.0)
    cfg = cfg_for(orc, sc, orc.INERTIAL, dt=5e-3)
    x, q, v = sc.x, sc.q, sc.vel
    nrows = 0
    for _ in range(40):
        r = orc.step(cfg, x, q, sc.axes, v)
        assert r.depth == 0 and r.status == 0
        nrows += r.rows_ia.size
        x, q, v = r.x, r.q, r.vel
    assert nrows > 50  # contacts did occur


def test_depth_vanishes_as_dt_goes_to_zero(orc):
    sc = scenes.two_ellipsoid_scene(offset_y=4.2)
    depth = {}
    for dt, nsteps in ((0.1, 150), (0.01, 1500)):
        cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=dt, eps_ncp=1e-5, box=(0, 0, 0), skin=0.5)
        x, q = sc.x, sc.q
        ds = []
        for _ in range(nsteps):
            r = orc.step(cfg, x, q, sc.axes, None, sc.fext)
            assert r.status == 0
            assert r.max_overlap <= 1e-5
            ds.append(r.depth)
            if r.depth:
                w = np.array(r.W)
                assert np.all(np.diff(w) >= -1e-12 * max(1.0, w.max()))
            x, q = r.x, r.q
        depth[dt] = np.array(ds)
    assert depth[0.1].max() >= 1
    assert depth[0.01].max() == 0


def test_recursion_invariants_dense_scene(orc):
    """Dense overdamped suspension at a large step: every LCP complementary,
    W_n nondecreasing, stopping rule met, enumeration == Lemke on small
    instances."""
    sc = scenes.lattice_scene(seed=5, n=27, spacing=1.55, axes_range=(0.45, 0.8), vel_sigma=0.0, omega_sigma=0.0)
    rng = np.random.default_rng(5)
    fext = np.concatenate([-(sc.x - sc.box / 2) * 4.0, rng.normal(0, 0.5, (sc.n, 3))], axis=1)
    cfg = cfg_for(orc, sc, orc.OVERDAMPED, dt=0.05)
    x, q = sc.x, sc.q
    saw_depth = False
    for k in range(25):
        r = orc.step(cfg, x, q, sc.axes, None, fext)
        assert r.status == 0
        assert r.max_overlap <= cfg.eps_ncp
        for gam, g in zip(r.gammas, r.gs):
            if gam.size:
                sc_ = 1 + np.abs(g).max()
                assert gam.min() >= 0 and g.min() >= -1e-11 * sc_
                assert np.abs(gam * g).max() <= 1e-11 * sc_ * (1 + gam.max())
        w = np.array(r.W)
        assert np.all(np.diff(w) >= -1e-10 * max(1.0, w.max()))
        if r.depth:
            saw_depth = True
        if r.rows_ia.size and r.rows_ia.size <= 10:
            r2 = orc.step(cfg, x, q, sc.axes, None, fext, lcp_solver=enum_solver)
            assert r2.depth == r.depth
            assert np.allclose(r2.x, r.x, atol=1e-10) and np.allclose(r2.vel, r.vel, atol=1e-8)
        x, q = r.x, r.q
    assert saw_depth


def test_contact_impulse_conserves_momentum(orc):
    """Linear momentum of the whole contact impulse is conserved exactly.
    Angular momentum about the origin is conserved by the rows generated at
    C^k (their lever arms satisfy y_b - y_a = Phi n at C^k); rows appended at
    a trial configuration are frozen there, so only their linear part is
    checked here."""
    sc = scenes.sphere_scene(seed=7, n=40, side=7.0, vel_sigma=4.0)
    rng = np.random.default_rng(7)
    axes = sc.axes * rng.uniform(0.7, 1.0, sc.axes.shape)
    cfg = orc.Config(dynamics=orc.INERTIAL, dt=1e-2, eps_ncp=1e-4, box=(0, 0, 0), skin=0.1)
    x, q, v = sc.x, sc.q, sc.vel
    checked = 0
    for _ in range(30):
        r = orc.step(cfg, x, q, axes, v)
        assert r.status == 0
        m, I = orc.mass_properties(axes)
        Uc = r.U_contact  # = dt M^-1 D gamma
        P = np.sum(m[:, None] * Uc[:, :3], axis=0)
        scale = 1 + np.abs(m[:, None] * Uc[:, :3]).sum()
        assert np.abs(P).max() <= 1e-12 * scale
        sel = r.rows_rec == 0
        if r.gamma.size and sel.any():
            W0 = orc.wrench(x.shape[0], r.rows_ia[sel], r.rows_ib[sel], r.rows_n[sel], r.rows_ta[sel],
                            r.rows_tb[sel], r.gamma[sel])
            L = np.sum(np.cross(x, W0[:, :3]) + W0[:, 3:], axis=0)
            assert np.abs(L).max() <= 1e-10 * (1 + np.abs(W0).sum()) * (1 + np.abs(x).max())
            if r.gamma[sel].max() > 0:
                checked += 1
        x, q, v = r.x, r.q, r.vel
    assert checked > 3


def test_head_on_equal_spheres_inelastic(orc):
    r0, dt, u = 0.5, 1e-2, 1.0
    for gap in (0.0, 0.004):
        x = np.array([[0.0, 0.0, 0.0], [2 * r0 + gap, 0.0, 0.0]])
        q = np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]])
        axes = np.full((2, 3), r0)
        v = np.array([[u, 0, 0, 0, 0, 0], [-u, 0, 0, 0, 0, 0]], dtype=float)
        cfg = orc.Config(dynamics=orc.INERTIAL, dt=dt, eps_ncp=1e-6, box=(0, 0, 0), skin=0.1)
        r = orc.step(cfg, x, q, axes, v)
        # the gap closes exactly: relative velocity -gap/dt, split symmetrically
        assert abs(r.vel[0, 0] - gap / (2 * dt)) < 1e-12
        assert abs(r.vel[1, 0] + gap / (2 * dt)) < 1e-12
        assert abs(r.vel[0, 0] + r.vel[1, 0]) < 1e-14
        assert r.depth == 0


def test_overdamped_balanced_pair(orc):
    x = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    q = np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]])
    axes = np.array([[0.75] * 3, [0.75] * 3])
    F = 2.5
    fext = np.array([[F, 0, 0, 0, 0, 0], [-F, 0, 0, 0, 0, 0]], dtype=float)
    cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=1e-2, eps_ncp=1e-6, box=(0, 0, 0), skin=0.1, drag_xi=3.0)
    r = orc.step(cfg, x, q, axes, None, fext)
    assert r.gamma.size == 1 and abs(r.gamma[0] - F) < 1e-12
    assert np.abs(r.vel).max() < 1e-13
    # approaching pair at a gap: it closes exactly in one step
    x[1, 0] = 1.5 + 0.01
    r = orc.step(cfg, x, q, axes, None, fext)
    kt = 1.0 / (3.0 * 1.5)  # 1/(xi L), L = 2 x semi-axis
    # relative velocity -gap/dt = 2 kt (F - gamma)  ->  gamma = F - gap/(2 dt kt)
    assert abs(r.gamma[0] - (F - 0.01 / (2 * 1e-2 * kt))) < 1e-10


def test_linearised_separation_is_second_order(orc):
    """Phi(C + dt G U) - (Phi(C) + dt d^T U) = O(dt^2) for the Jacobian row
    [-n, -(r_a x n), n, (r_b x n)]."""
    rng = np.random.default_rng(31)
    for _ in range(10):
        x = np.array([[0.0, 0, 0], rng.normal(size=3)])
        x[1] = x[1] / np.linalg.norm(x[1]) * 1.6
        q = scenes.random_quaternions(rng, 2)
        axes = rng.uniform(0.5, 1.0, (2, 3))
        U = rng.normal(size=(2, 6))
        pairs = np.array([[0, 1]], dtype=np.int32)
        phi, n, ra, rb, _ = orc.snsd(pairs, x, q, axes, np.zeros(3))
        ta, tb = np.cross(ra, n), np.cross(rb, n)
        rate = orc.rows_dot_U(np.array([0]), np.array([1]), n, ta, tb, U)[0]
        errs = []
        for dt in (1e-2, 5e-3, 2.5e-3):
            x1 = x + dt * U[:, :3]
            q1 = orc.quat_step(q, U[:, 3:], dt)
            p1 = orc.snsd(pairs, x1, q1, axes, np.zeros(3))[0][0]
            errs.append(abs(p1 - (phi[0] + dt * rate)))
        assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_recursion_zero_is_lcp_snsd(orc):
    sc = scenes.two_ellipsoid_scene(offset_y=4.2)
    cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=0.1, eps_ncp=1e-5, box=(0, 0, 0), skin=0.5)
    x, q = sc.x, sc.q
    for _ in range(30):
        r = orc.step(cfg, x, q, sc.axes, None, sc.fext)
        x, q = r.x, r.q
    assert r.depth >= 1
    cfg0 = orc.Config(**{**cfg.__dict__, "max_recursion": 0})
    x0, q0 = x, q
    r_full = orc.step(cfg, x0, q0, sc.axes, None, sc.fext)
    r_zero = orc.step(cfg0, x0, q0, sc.axes, None, sc.fext)
    assert r_zero.status == 5  # recursion limit reported
    assert np.all(r_zero.rows_rec == 0)
    assert np.allclose(r_zero.gamma, r_full.gammas[0], rtol=0, atol=0)


def test_quaternion_update_vs_exact_rotation(orc):
    rng = np.random.default_rng(33)
    q = scenes.random_quaternions(rng, 50)
    w = rng.normal(size=(50, 3))
    for dt in (1e-2, 1e-3):
        q1 = orc.quat_step(q, w, dt)
        th = np.linalg.norm(w, axis=1) * dt
        ax = w / np.linalg.norm(w, axis=1, keepdims=True)
        dq = np.concatenate([np.cos(th / 2)[:, None], np.sin(th / 2)[:, None] * ax], axis=1)
        qe = orc.quat_mul(dq, q)
        err = np.minimum(np.linalg.norm(q1 - qe, axis=1), np.linalg.norm(q1 + qe, axis=1))
        assert err.max() < 0.1 * (np.linalg.norm(w, axis=1).max() * dt) ** 3


def test_mass_properties_monte_carlo(orc):
    rng = np.random.default_rng(34)
    axes = np.array([[0.5, 0.8, 1.1]])
    m, I = orc.mass_properties(axes)
    N = 2_000_000
    pts = (rng.random((N, 3)) * 2 - 1) * axes[0]
    inside = np.sum((pts / axes[0]) ** 2, axis=1) <= 1
    boxvol = np.prod(2 * axes[0])
    mc_m = boxvol * inside.mean()
    p = pts[inside]
    mc_I = boxvol / N * np.array([np.sum(p[:, 1] ** 2 + p[:, 2] ** 2), np.sum(p[:, 0] ** 2 + p[:, 2] ** 2),
                                  np.sum(p[:, 0] ** 2 + p[:, 1] ** 2)])
    assert abs(mc_m - m[0]) / m[0] < 5e-3
    assert np.allclose(mc_I, I[0], rtol=1e-2)


def test_rotation_matrix_matches_sandwich_product(orc):
    rng = np.random.default_rng(35)
    q = scenes.random_quaternions(rng, 20)
    R = orc.quat_rot(q)
    for k in range(20):
        for e in np.eye(3):
            v = orc.quat_mul(orc.quat_mul(q[k], np.array([0.0, *e])), q[k] * np.array([1, -1, -1, -1]))
            assert np.allclose(R[k] @ e, v[1:], atol=1e-14)


# ---------------------------------------------------------------------------
# pull-back of appended rows (Sec. 3.1.3) and the periodic affine background
# ---------------------------------------------------------------------------
def _trial_phi(orc, cfg, x, q, axes, U_free, kt, Kr, rows, gamma, pairs, box1):
    """True SNSD of `pairs` at the trial configuration C^k + dt G^k (U_free +
    K D gamma) of a given gamma over the given rows."""
    ia, ib, nrm, ta, tb = rows
    U = U_free + orc.apply_K(kt, Kr, orc.wrench(x.shape[0], ia, ib, nrm, ta, tb, gamma))
    return orc.snsd(pairs, x + cfg.dt * U[:, :3], orc.quat_step(q, U[:, 3:], cfg.dt), axes, box1)[0]


def _check_pullback(orc, cfg, x, q, axes, vel, fext):
    """For every row appended at recursion j >= 1, its modelled gap
    g_a(gamma) = q_a + (A gamma)_a is the linearisation of the true SNSD at
    the configuration C_j where the row was found, pulled back to C^k:
      (i)  at the gamma that produced C_j it equals Phi_a(C_j) exactly;
      (ii) along the segment from that gamma to the final one it follows the
           true Phi_a of the trial configuration to first order: the
           mismatch is a small fraction (1%) of the modelled change, which
           also pins the frozen row (n, r_a x n, r_b x n) taken at C_j.
    Dropping, flipping or widening (U instead of K D gamma) the pulled-back
    term breaks (i) by a first-order amount."""
    r = orc.step(cfg, x, q, axes, vel, fext)
    if r.depth == 0:
        return 0, 0.0
    n = x.shape[0]
    qn = q / np.linalg.norm(q, axis=1, keepdims=True)
    kt, Kr = orc.operator_K(cfg.dynamics, cfg.dt, qn, axes, cfg.density, cfg.drag_xi)
    box0 = np.asarray(cfg.box, dtype=float)
    box1 = np.where(box0 > 0, box0 * (1 + cfg.strain_rate * cfg.dt), 0.0)
    U_free = orc.free_velocity(cfg, x, np.zeros((n, 6)) if vel is None else vel,
                               np.zeros((n, 6)) if fext is None else fext, kt, Kr, box0)
    m = r.rows_ia.size
    A = orc.dense_A(cfg.dt, kt, Kr, r.rows_ia, r.rows_ib, r.rows_n, r.rows_ta, r.rows_tb)
    rows = (r.rows_ia, r.rows_ib, r.rows_n, r.rows_ta, r.rows_tb)
    checked, pulled = 0, 0.0
    for j in range(1, r.depth + 1):
        sel = np.nonzero(r.rows_rec == j)[0]
        g_prev = np.zeros(m)
        g_prev[:r.gammas[j - 1].size] = r.gammas[j - 1]
        pulled = max(pulled, float(np.abs((A @ g_prev)[sel]).max()))  # c d^T K D gamma_{j-1}
        model0 = r.rows_q[sel] + (A @ g_prev)[sel]
        true0 = r.trial_phi[j - 1][r.rows_pair[sel]]
        assert np.abs(model0 - true0).max() <= 1e-12 * (1 + np.abs(true0).max())
        pairs = r.pairs[r.rows_pair[sel]]
        for t in (1.0, 0.5, 0.25):
            gt = g_prev + t * (r.gamma - g_prev)
            change = np.abs((A @ (gt - g_prev))[sel]).max()
            model = r.rows_q[sel] + (A @ gt)[sel]
            true = _trial_phi(orc, cfg, x, qn, axes, U_free, kt, Kr, rows, gt, pairs, box1)
            # the mismatch is the curvature of Phi plus the difference between
            # the linear kinematic map at C^k and rigid motion at C_j (relative
            # O(dt |omega|)): measured below 0.4% of the modelled change here
            assert np.abs(model - true).max() <= 1e-2 * change + 1e-12, (t, np.abs(model - true).max(), change)
        checked += sel.size
    return checked, pulled


def test_pullback_offset_of_appended_rows(orc):
    """Overdamped two-ellipsoid collision (Sec. 5.2) at dt = 0.1, where the
    recursion appends rows, and a dense inertial lattice."""
    sc = scenes.two_ellipsoid_scene(offset_y=4.2)
    cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=0.1, eps_ncp=1e-5, box=(0, 0, 0), skin=0.5)
    x, q = sc.x, sc.q
    checked, pulled = 0, 0.0
    for _ in range(40):
        c_, p_ = _check_pullback(orc, cfg, x, q, sc.axes, None, sc.fext)
        checked, pulled = checked + c_, max(pulled, p_)
        r = orc.step(cfg, x, q, sc.axes, None, sc.fext)
        x, q = r.x, r.q
    # the pulled-back term is a first-order amount, far above eps_NCP: leaving
    # it out could not pass (i)
    assert checked >= 3 and pulled > 100 * cfg.eps_ncp
    sc = scenes.lattice_scene(seed=2, n=64, spacing=1.8, dt=1e-2, vel_sigma=3.0, omega_sigma=1.5)
    amin = float(sc.axes.min())
    cfg = orc.Config(dynamics=orc.INERTIAL, dt=1e-2, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
    x, q, v = sc.x, sc.q, sc.vel
    checked, pulled = 0, 0.0
    for _ in range(12):
        c_, p_ = _check_pullback(orc, cfg, x, q, sc.axes, v, None)
        checked, pulled = checked + c_, max(pulled, p_)
        r = orc.step(cfg, x, q, sc.axes, v)
        x, q, v = r.x, r.q, r.vel
    assert checked >= 1 and pulled > cfg.eps_ncp


def _compacted_state(orc, n=256, steps=200, seed=1):
    sc = scenes.suspension_scene(seed=seed, n=n, phi=0.1, steps=300, dt=5e-3)
    amin = float(sc.axes.min())
    rate = sc.meta["strain_rate"]
    cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin,
                     strain_rate=rate)
    x, q, box = sc.x, sc.q, np.asarray(sc.box)
    for _ in range(steps):
        r = orc.step(orc.Config(**{**cfg.__dict__, "box": tuple(box)}), x, q, sc.axes)
        x, q, box = r.x, r.q, r.box
    return orc.Config(**{**cfg.__dict__, "box": tuple(box)}), x, q, sc.axes


def test_affine_compaction_is_translation_invariant(orc):
    """A periodic box compacted affinely has no preferred origin: translating
    every body by s and wrapping it into the box changes the background
    velocity of the wrapped bodies by a multiple of strain_rate x L, which the
    minimum-image offset of each pair must cancel.  The step from the shifted
    state therefore has the same pairs, rows and gamma, the same contact
    velocities, and its accepted configuration is the original one shifted by
    s (1 + strain_rate dt), modulo the new box.  Several shifts move different
    pairs across the boundary."""
    cfg, x, q, axes = _compacted_state(orc)
    rate = cfg.strain_rate
    box = np.asarray(cfg.box)
    r0 = orc.step(cfg, x, q, axes)
    assert r0.rows_ia.size > 100 and r0.gamma.max() > 0
    rng = np.random.default_rng(0)
    straddled = 0
    for s in (rng.uniform(0.2, 0.8, 3) * box, np.array([0.5, 0.0, 0.0]) * box, rng.uniform(0, 1, 3) * box):
        xs = x + s
        xs -= box * np.floor(xs / box)
        raw0 = x[r0.rows_ib] - x[r0.rows_ia]
        raws = xs[r0.rows_ib] - xs[r0.rows_ia]
        straddled += int(np.sum(np.any(np.abs(raw0 - raws) > 0.5 * box, axis=1)))
        r1 = orc.step(cfg, xs, q, axes)
        assert np.array_equal(r0.pairs, r1.pairs)
        ids0 = np.stack([r0.rows_ia, r0.rows_ib, r0.rows_rec, r0.rows_pair])
        ids1 = np.stack([r1.rows_ia, r1.rows_ib, r1.rows_rec, r1.rows_pair])
        assert np.array_equal(ids0, ids1)
        assert np.abs(r0.gamma - r1.gamma).max() <= 1e-9 * np.abs(r0.gamma).max()
        assert np.abs(r0.U_contact - r1.U_contact).max() <= 1e-9 * np.abs(r0.U_contact).max()
        box1 = np.asarray(r0.box)
        d = r1.x - s * (1 + rate * cfg.dt) - r0.x
        d -= box1 * np.rint(d / box1)
        assert np.abs(d).max() <= 1e-12 * box1.max()
    assert straddled > 10  # rows whose bodies the shifts moved across the boundary


def test_affine_compaction_scales_free_bodies_with_the_box(orc):
    """Without contacts the background velocity strain_rate (x - L/2) scales
    every body about the box centre by the factor the box side takes:
    x' - L/2 = (1 + strain_rate dt)(x - L/2) with L' = L (1 + strain_rate dt),
    for compaction and for dilation (a uniform drift of the centre relative to
    the new box, (L - L')/2, is a translation of the periodic system)."""
    rng = np.random.default_rng(4)
    n, L = 20, 50.0
    x = rng.uniform(0, L, (n, 3))
    q = scenes.random_quaternions(rng, n)
    axes = np.full((n, 3), 0.3)
    for rate in (-0.8, 0.5):
        cfg = orc.Config(dynamics=orc.OVERDAMPED, dt=1e-2, eps_ncp=1e-4, box=(L, L, L), skin=0.03, strain_rate=rate)
        r = orc.step(cfg, x, q, axes)
        assert r.rows_ia.size == 0
        L1 = np.asarray(r.box)
        assert np.allclose(L1, L * (1 + rate * 1e-2), rtol=1e-15)
        f = 1 + rate * 1e-2
        d = r.x - 0.5 * L - f * (x - 0.5 * L)
        d -= L1 * np.rint(d / L1)  # accepted positions are wrapped into the new box
        assert np.abs(d).max() <= 1e-12
        assert np.abs(r.vel[:, :3] - rate * (x - 0.5 * L)).max() <= 1e-13
