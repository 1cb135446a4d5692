"""Pins of the oracle's spherocylinder SNSD (the colony cells of Sec. 5.4):
a segment of half-length h along the body x axis swept by a ball of radius
rho, semi-axes row (h + rho, rho, rho).

* h = 0 reduces to spheres: Phi = |d| - rho_a - rho_b;
* perpendicular skew segments: closest points and Phi in closed form;
* the closest-point parameters minimise |w + t v - s u|^2 over the rectangle
  (a 401 x 401 grid search plus local refinement never finds lower);
* Phi is the maximum over unit n of the support-function gap
  G(n) = n.d - h_a |u.n| - rho_a - h_b |v.n| - rho_b (separated pairs; 40k
  sampled directions never exceed it, and G at the returned normal equals it);
* the support points lie on the surfaces, with y_b - y_a = Phi n;
* a planar spherocylinder colony meets the stopping rule and stays planar.
"""
import numpy as np

from paper_2506_14097_gb300 import scenes


def pair_state(rng, separated=True):
    q = scenes.random_quaternions(rng, 2)
    rho = rng.uniform(0.2, 0.6, 2)
    h = rng.uniform(0.0, 1.5, 2)
    axes = np.stack([h + rho, rho, rho], axis=1)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    dist = (h.sum() + rho.sum() + rng.uniform(0.05, 0.5)) if separated else rng.uniform(0.3, 1.0) * (h.sum() + rho.sum())
    x = np.stack([np.zeros(3), dist * d])
    return x, q, axes


def test_sphere_limit(orc):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 4, (40, 3))
    r = rng.uniform(0.2, 0.7, 40)
    axes = np.stack([r, r, r], axis=1)
    q = scenes.random_quaternions(rng, 40)
    pairs = np.array([(i, j) for i in range(40) for j in range(i + 1, 40)])
    phi, n, ra, rb, fl = orc.snsd_capsules(pairs, x, q, axes, np.zeros(3))
    d = np.linalg.norm(x[pairs[:, 1]] - x[pairs[:, 0]], axis=1)
    assert fl.max() == 0
    assert np.abs(phi - (d - r[pairs[:, 0]] - r[pairs[:, 1]])).max() < 1e-13


def test_perpendicular_skew_segments(orc):
    # a along x (h = 1, rho = 0.3) at the origin; b along y (h = 1, rho = 0.2) at (0.2, 0.5, 1.5)
    qa = np.array([1.0, 0, 0, 0])
    qb = np.array([np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)])  # body x -> world y
    x = np.array([[0.0, 0, 0], [0.2, 0.5, 1.5]])
    axes = np.array([[1.3, 0.3, 0.3], [1.2, 0.2, 0.2]])
    phi, n, ra, rb, fl = orc.snsd_capsules(np.array([[0, 1]]), x, np.stack([qa, qb]), axes, np.zeros(3))
    assert abs(phi[0] - 1.0) < 1e-14
    assert np.abs(n[0] - [0, 0, 1]).max() < 1e-14
    assert np.abs(ra[0] - [0.2, 0, 0.3]).max() < 1e-14   # s = 0.2 on a, plus rho_a n
    assert np.abs(rb[0] - [0, -0.5, -0.2]).max() < 1e-14  # t = -0.5 on b, minus rho_b n


def test_closest_points_minimise_over_the_rectangle(orc):
    rng = np.random.default_rng(2)
    for _ in range(60):
        u, v = rng.normal(size=3), rng.normal(size=3)
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        w = rng.normal(size=3) * 1.5
        ha, hb = rng.uniform(0, 1.5, 2)
        s_, t_ = orc.segment_closest_params(w, u, ha, v, hb)
        f = np.sum((w + t_ * v - s_ * u) ** 2)
        S, T = np.meshgrid(np.linspace(-ha, ha, 401), np.linspace(-hb, hb, 401), indexing="ij")
        F = np.sum((w[None, None] + T[..., None] * v - S[..., None] * u) ** 2, axis=-1)
        k = np.unravel_index(np.argmin(F), F.shape)
        # local refinement of the grid minimum by projected coordinate descent
        s0, t0 = S[k], T[k]
        for _ in range(200):
            s0 = np.clip(w @ u + t0 * (u @ v), -ha, ha)
            t0 = np.clip(s0 * (u @ v) - w @ v, -hb, hb)
        f_ref = min(F[k], np.sum((w + t0 * v - s0 * u) ** 2))
        assert f <= f_ref + 1e-12


def test_phi_is_support_function_maximum(orc):
    rng = np.random.default_rng(3)
    dirs = rng.normal(size=(40000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for _ in range(20):
        x, q, axes = pair_state(rng, separated=True)
        phi, n, ra, rb, fl = orc.snsd_capsules(np.array([[0, 1]]), x, q, axes, np.zeros(3))
        u, h, rho = orc.capsule_geometry(q, axes)
        d = x[1] - x[0]

        def G(m):
            return m @ d - h[0] * np.abs(m @ u[0]) - rho[0] - h[1] * np.abs(m @ u[1]) - rho[1]

        assert G(dirs).max() <= phi[0] + 1e-12
        assert abs(G(n[0]) - phi[0]) <= 1e-12
        # support points on the surfaces, separated along n by Phi
        ya, yb = x[0] + ra[0], x[1] + rb[0]
        assert abs(np.linalg.norm(yb - ya) - abs(phi[0])) < 1e-12
        assert np.abs((yb - ya) - phi[0] * n[0]).max() < 1e-12


def test_capsule_colony_step_invariants(orc):
    # cells along x touching end to end and side by side, pushed together
    x = np.array([[0.0, 0, 0], [2.0, 0.05, 0], [1.0, 1.05, 0], [-1.0, 1.0, 0]])
    theta = np.array([0.0, 0.1, -0.05, 0.3])
    q = scenes.planar_quaternions(theta)
    axes = np.tile([1.0, 0.5, 0.5], (4, 1))  # h = 0.5, rho = 0.5
    fext = np.zeros((4, 6))
    fext[:, :2] = -x[:, :2]
    cfg = orc.Config(dynamics=orc.OVERDAMPED_2D, dt=0.05, eps_ncp=5e-4, box=(0, 0, 0), skin=0.05,
                     shape=orc.SHAPE_SPHEROCYLINDER)
    rows = 0
    for _ in range(60):
        r = orc.step(cfg, x, q, axes, None, fext)
        assert r.status == 0 and r.max_overlap <= cfg.eps_ncp
        assert np.all(r.x[:, 2] == 0.0) and np.all(r.q[:, 1:3] == 0.0)
        for gam, g in zip(r.gammas, r.gs):
            if gam.size:
                assert gam.min() >= 0 and g.min() >= -1e-11
        rows += r.rows_ia.size
        x, q = r.x, r.q
        fext[:, :2] = -x[:, :2]
    assert rows > 60
