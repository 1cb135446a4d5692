"""Pins of the oracle's shared-normal signed distance (SNSD) against facts the
paper and geometry fix, none of which reuse the oracle's own formula:

* spheres: Phi = |d| - r1 - r2 with n = d/|d| (textbook SNSD);
* separated, equally oriented ellipsoids offset along a principal axis:
  Phi = |d| - a1 - a2;
* the support points lie on the surfaces with outward normals n and -n
  (n_a = -n_b, Sec. 2.1.4) and y_b - y_a = Phi n (interior tangent-ball
  lemma, Sec. 4.2);
* sign agrees with the Perram-Wertheim overlap function (an independent
  published predicate), and translating b by -Phi n makes the bodies tangent
  (Perram-Wertheim F = 1);
* Phi is not below G(n) for any of 20k sampled directions;
* for separated bodies Phi equals the primal Euclidean distance (an
  SLSQP minimisation over surface points);
* the envelope property dPhi = row . dU along rigid motions (Sec. 2.1.3,
  linearised separation rate).
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar


def rand_rot_quat(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def rot(q):
    s, x, y, z = q / np.linalg.norm(q)
    # independent construction: rotate the basis vectors with the Hamilton
    # sandwich product v' = q v q*
    def qmul(a, b):
        return np.array([a[0] * b[0] - a[1:] @ b[1:], *(a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:]))])

    qq = np.array([s, x, y, z])
    qc = np.array([s, -x, -y, -z])
    cols = []
    for e in np.eye(3):
        v = qmul(qmul(qq, np.array([0.0, *e])), qc)
        cols.append(v[1:])
    return np.stack(cols, axis=1)


def shape(q, ax):
    R = rot(q)
    return R @ np.diag(np.asarray(ax) ** 2) @ R.T


def pw_F(d, Pa, Pb):
    """Perram-Wertheim contact function max_l l(1-l) d^T ((1-l)Pa + l Pb)^-1 d;
    < 1 overlap, = 1 external tangency, > 1 separated."""
    f = lambda l: -(l * (1 - l) * d @ np.linalg.solve((1 - l) * Pa + l * Pb, d))
    r = minimize_scalar(f, bounds=(0.0, 1.0), method="bounded", options={"xatol": 1e-13})
    return -r.fun


def fib_sphere(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def random_pair(rng, dist_scale=1.0):
    qa, qb = rand_rot_quat(rng, 2)
    aa = rng.uniform(0.4, 1.0, 3)
    ab = rng.uniform(0.4, 1.0, 3)
    d = rng.normal(size=3)
    d = d / np.linalg.norm(d) * rng.uniform(0.6, 2.4) * dist_scale
    return d, qa, aa, qb, ab


def test_spheres_closed_form(orc):
    rng = np.random.default_rng(11)
    for _ in range(200):
        r1, r2 = rng.uniform(0.3, 1.2, 2)
        d = rng.normal(size=3) * rng.uniform(0.2, 2.0)
        P1, P2 = r1 * r1 * np.eye(3), r2 * r2 * np.eye(3)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, P1, P2)
        L = np.linalg.norm(d)
        assert abs(phi - (L - r1 - r2)) <= 1e-13 * (1 + L)
        assert np.allclose(n, d / L, atol=1e-12)
        assert np.allclose(ra, r1 * d / L, atol=1e-12)
        assert np.allclose(rb, -r2 * d / L, atol=1e-12)


def test_coaxial_ellipsoids(orc):
    rng = np.random.default_rng(12)
    for _ in range(100):
        q = rand_rot_quat(rng, 1)[0]
        R = rot(q)
        aa, ab = rng.uniform(0.4, 1.0, 3), rng.uniform(0.4, 1.0, 3)
        k = rng.integers(3)
        # separated along a common principal axis: by the reflection symmetry
        # of both bodies the unique closest pair lies on that axis
        L = aa[k] + ab[k] + rng.uniform(1e-3, 2.0)
        d = R[:, k] * L
        phi, n, ra, rb, fl = orc.snsd_from_d(d, shape(q, aa), shape(q, ab))
        assert abs(phi - (L - aa[k] - ab[k])) <= 1e-12
        assert np.allclose(n, R[:, k], atol=1e-9)


def test_support_points_and_shared_normal(orc):
    rng = np.random.default_rng(13)
    for _ in range(300):
        d, qa, aa, qb, ab = random_pair(rng)
        Pa, Pb = shape(qa, aa), shape(qb, ab)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, Pa, Pb)
        assert fl == 0
        Ra, Rb = rot(qa), rot(qb)
        # on the surfaces
        assert abs(np.linalg.norm((Ra.T @ ra) / aa) - 1) < 1e-12
        assert abs(np.linalg.norm((Rb.T @ rb) / ab) - 1) < 1e-12
        # outward normals n at y_a and -n at y_b (gradients of the implicit
        # functions x^T P^-1 x)
        na = np.linalg.solve(Pa, ra)
        nb = np.linalg.solve(Pb, rb)
        assert np.allclose(na / np.linalg.norm(na), n, atol=1e-10)
        assert np.allclose(nb / np.linalg.norm(nb), -n, atol=1e-10)
        # y_b - y_a = Phi n
        yab = (d + rb) - ra
        assert np.allclose(yab, phi * n, atol=1e-11 * (1 + np.linalg.norm(d)))


def test_sign_and_tangency_vs_perram_wertheim(orc):
    rng = np.random.default_rng(14)
    checked = 0
    for _ in range(150):
        d, qa, aa, qb, ab = random_pair(rng)
        Pa, Pb = shape(qa, aa), shape(qb, ab)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, Pa, Pb)
        F = pw_F(d, Pa, Pb)
        if abs(F - 1) > 1e-3:
            assert (phi > 0) == (F > 1)
            checked += 1
        # translate b by -Phi n: tangent contact, F = 1
        F0 = pw_F(d - phi * n, Pa, Pb)
        assert abs(F0 - 1.0) < 1e-9, (phi, F0)
    assert checked > 100


def test_max_over_sampled_directions(orc):
    rng = np.random.default_rng(15)
    dirs = fib_sphere(20000)
    for _ in range(40):
        d, qa, aa, qb, ab = random_pair(rng)
        Pa, Pb = shape(qa, aa), shape(qb, ab)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, Pa, Pb)
        G = dirs @ d - np.sqrt(np.einsum("ij,jk,ik->i", dirs, Pa, dirs)) - np.sqrt(
            np.einsum("ij,jk,ik->i", dirs, Pb, dirs))
        assert phi >= G.max() - 1e-12
        assert phi - G.max() < 2e-3


def test_separated_equals_primal_distance(orc):
    rng = np.random.default_rng(16)
    done = 0
    while done < 15:
        d, qa, aa, qb, ab = random_pair(rng, dist_scale=1.5)
        Pa, Pb = shape(qa, aa), shape(qb, ab)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, Pa, Pb)
        if phi < 0.05:
            continue
        Ra, Rb = rot(qa), rot(qb)

        def f(z):
            ya = Ra @ (aa * z[:3])
            yb = d + Rb @ (ab * z[3:])
            return np.sum((ya - yb) ** 2)

        cons = [{"type": "ineq", "fun": lambda z: 1 - z[:3] @ z[:3]},
                {"type": "ineq", "fun": lambda z: 1 - z[3:] @ z[3:]}]
        best = np.inf
        for z0 in [np.concatenate([Ra.T @ (d / np.linalg.norm(d)) / aa * 0.5, -Rb.T @ (d / np.linalg.norm(d)) / ab * 0.5]),
                   np.zeros(6)]:
            r = minimize(f, z0, constraints=cons, method="SLSQP", options={"ftol": 1e-15, "maxiter": 500})
            best = min(best, r.fun)
        assert abs(math.sqrt(best) - phi) < 1e-6, (math.sqrt(best), phi)
        done += 1


def test_envelope_rate_equals_row_times_velocity(orc):
    """dPhi/dt along rigid motions = -n.u_a - (r_a x n).w_a + n.u_b + (r_b x n).w_b"""
    rng = np.random.default_rng(17)

    def qstep(q, w, h):
        wq = np.array([0.0, *w])
        s1, v1 = wq[0], wq[1:]
        s2, v2 = q[0], q[1:]
        prod = np.array([s1 * s2 - v1 @ v2, *(s1 * v2 + s2 * v1 + np.cross(v1, v2))])
        q1 = q + 0.5 * h * prod
        return q1 / np.linalg.norm(q1)

    for _ in range(60):
        d, qa, aa, qb, ab = random_pair(rng)
        phi, n, ra, rb, fl = orc.snsd_from_d(d, shape(qa, aa), shape(qb, ab))
        ua, wa, ub, wb = rng.normal(size=(4, 3))
        row = -n @ ua - np.cross(ra, n) @ wa + n @ ub + np.cross(rb, n) @ wb
        h = 1e-5
        vals = []
        for s in (+1, -1):
            dd = d + s * h * (ub - ua)
            qa1, qb1 = qstep(qa, wa, s * h), qstep(qb, wb, s * h)
            vals.append(orc.snsd_from_d(dd, shape(qa1, aa), shape(qb1, ab))[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - row) < 1e-6 * (1 + abs(row)), (fd, row)


def test_periodic_min_image(orc):
    rng = np.random.default_rng(18)
    box = np.array([10.0, 10.0, 10.0])
    x = np.array([[0.3, 5.0, 9.8], [9.5, 5.4, 0.4]])
    q = rand_rot_quat(rng, 2)
    axes = rng.uniform(0.4, 1.0, (2, 3))
    pairs = np.array([[0, 1]], dtype=np.int32)
    phi, n, ra, rb, fl = orc.snsd(pairs, x, q, axes, box)
    d = np.array([9.5 - 0.3 - 10.0, 0.4, 0.4 + 10.0 - 9.8])
    phi2, n2, *_ = orc.snsd_from_d(d, shape(q[0], axes[0]), shape(q[1], axes[1]))
    assert abs(phi[0] - phi2) < 1e-13 and np.allclose(n[0], n2)


def test_icosphere_seed_count(orc):
    import ctypes

    out = np.zeros((700, 3))
    k = orc.lib().orc_icosphere(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert k == 642
    assert np.allclose(np.linalg.norm(out[:k], axis=1), 1.0)
