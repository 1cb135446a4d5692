"""Pins of the oracle's planar dynamics (OVERDAMPED_2D) used by the growing
colony (Sec. 5.4 restated with ellipsoidal cells in the z = 0 plane):

* the LCP operator of the embedded six-DOF rows equals c D3^T M3 D3 built
  directly on the three planar DOFs (u_x, u_y, omega_z) with the mobility
  diag(1/(xi L), 1/(xi L), 12/(xi L^3)) of Eq. ellipsoid_mobility;
* a balanced pair of touching cells pushed together carries gamma = F and does
  not move (overdamped force balance);
* a colony grown through several divisions stays in the plane exactly
  (z = 0, rotations about z only), meets the stopping rule every step, and its
  recursion invariants hold;
* the colony model is deterministic in its seed.
"""
import numpy as np

from paper_2506_14097_gb300 import scenes


def colony_cfg(orc, dt=0.05):
    return orc.Config(dynamics=orc.OVERDAMPED_2D, dt=dt, eps_ncp=5e-4, box=(0, 0, 0), skin=0.05)


def grow(orc, col, steps, cfg, check=None):
    for _ in range(steps):
        r = orc.step(cfg, col.x, col.q(), col.axes())
        assert r.status == 0
        if check:
            check(r)
        col.advance(r.x, r.q)
    return col


def test_planar_operator_is_three_dof_assembly(orc):
    col = scenes.Colony(seed=3, rate=0.1)
    grow(orc, col, 900, colony_cfg(orc))
    assert col.n >= 8
    cfg = colony_cfg(orc)
    x, q, axes = col.x, col.q(), col.axes()
    r = orc.step(cfg, x, q, axes)
    m = r.rows_ia.size
    assert m >= 6
    kt, Kr = orc.operator_K(cfg.dynamics, cfg.dt, q, axes)
    A6 = orc.dense_A(cfg.dt, kt, Kr, r.rows_ia, r.rows_ib, r.rows_n, r.rows_ta, r.rows_tb)
    # three-DOF assembly from the SNSD geometry of the same rows
    phi, n, ra, rb, _ = orc.snsd(r.pairs, x, q, axes, np.zeros(3))
    N = col.n
    L = 2.0 * axes.max(axis=1)
    M3 = np.zeros(3 * N)
    M3[0::3] = 1.0 / L
    M3[1::3] = 1.0 / L
    M3[2::3] = 12.0 / L ** 3
    D3 = np.zeros((m, 3 * N))
    for k in range(m):
        p = r.rows_pair[k]
        a, b = r.pairs[p]
        nn, rA, rB = n[p], ra[p], rb[p]
        D3[k, 3 * a:3 * a + 2] = -nn[:2]
        D3[k, 3 * a + 2] = -(rA[0] * nn[1] - rA[1] * nn[0])
        D3[k, 3 * b:3 * b + 2] = nn[:2]
        D3[k, 3 * b + 2] = rB[0] * nn[1] - rB[1] * nn[0]
    A3 = cfg.dt * D3 @ np.diag(M3) @ D3.T
    assert np.all(r.rows_rec == 0)
    assert np.abs(A6 - A3).max() <= 1e-13 * np.abs(A3).max()


def test_planar_balanced_pair(orc):
    F = 1.5
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = scenes.planar_quaternions(np.array([0.0, 0.0]))
    axes = np.full((2, 3), 0.5)
    fext = np.array([[F, 0, 0, 0, 0, 0], [-F, 0, 0, 0, 0, 0]], dtype=float)
    r = orc.step(colony_cfg(orc), x, q, axes, None, fext)
    assert r.gamma.size == 1 and abs(r.gamma[0] - F) < 1e-12
    assert np.abs(r.vel).max() < 1e-13


def test_colony_stays_planar_and_meets_the_stopping_rule(orc):
    col = scenes.Colony(seed=5, rate=0.1)
    cfg = colony_cfg(orc)
    seen = {"rows": 0, "depth": 0}

    def check(r):
        assert np.all(r.x[:, 2] == 0.0)
        assert np.all(r.q[:, 1] == 0.0) and np.all(r.q[:, 2] == 0.0)
        assert np.all(r.vel[:, 2] == 0.0) and np.all(r.vel[:, 3:5] == 0.0)
        assert r.max_overlap <= cfg.eps_ncp
        w = np.array(r.W)
        assert np.all(np.diff(w) >= -1e-10 * max(1.0, w.max()))
        seen["rows"] += r.rows_ia.size
        seen["depth"] = max(seen["depth"], r.depth)

    grow(orc, col, 1200, cfg, check)
    assert col.n >= 12 and col.divisions >= 11 and seen["rows"] > 100


def test_colony_model_deterministic():
    a, b = scenes.Colony(seed=9, rate=0.05), scenes.Colony(seed=9, rate=0.05)
    for _ in range(500):
        a.advance(a.x + 0.001, a.q())
        b.advance(b.x + 0.001, b.q())
    assert a.n == b.n and np.array_equal(a.x, b.x) and np.array_equal(a.theta, b.theta) and np.array_equal(a.L, b.L)
