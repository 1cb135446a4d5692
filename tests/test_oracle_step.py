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
