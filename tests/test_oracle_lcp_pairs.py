"""Pins of the oracle's candidate pairs and its LCP solver.

Pairs: the brute-force definition is cross-checked by an independent cell
list written here.  LCP (Lemma "LCP <=> CQP", uniqueness lemma): Lemke's
method against brute-force 2^n active-set enumeration for n <= 12, the
complementarity invariants at larger n, CQP optimality against feasible
perturbations, and uniqueness of D gamma for positive semi-definite
A = D^T M D when gamma itself is not unique.
"""
import itertools

import numpy as np
import pytest


def enum_lcp(A, q):
    """All 2^n supports S: solve A_SS z_S = -q_S, accept z_S >= 0 and
    (A z + q) >= 0 off S.  Returns every solution found."""
    n = q.shape[0]
    sols = []
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            z = np.zeros(n)
            if S:
                AS = A[np.ix_(S, S)]
                try:
                    zS = np.linalg.lstsq(AS, -q[S], rcond=None)[0]
                except np.linalg.LinAlgError:
                    continue
                if np.linalg.norm(AS @ zS + q[S]) > 1e-9 * (1 + np.abs(q).max()):
                    continue
                if np.any(zS < -1e-11):
                    continue
                z[S] = np.maximum(zS, 0)
            w = A @ z + q
            if np.all(w >= -1e-10 * (1 + np.abs(q).max())):
                sols.append(z)
    return sols


def random_contact_lcp(rng, m, nbody, psd_extra=0):
    """A = D^T K D from random rigid-contact rows (the structure of the
    contact LCP), q random with both signs."""
    D = np.zeros((m, 6 * nbody))
    for r in range(m):
        a, b = rng.choice(nbody, 2, replace=False)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ra, rb = rng.normal(size=(2, 3)) * 0.5
        D[r, 6 * a:6 * a + 3] = -n
        D[r, 6 * a + 3:6 * a + 6] = -np.cross(ra, n)
        D[r, 6 * b:6 * b + 3] = n
        D[r, 6 * b + 3:6 * b + 6] = np.cross(rb, n)
    # duplicated rows make A singular (non-unique gamma)
    for _ in range(psd_extra):
        r = rng.integers(m)
        D = np.vstack([D, D[r]])
    kd = rng.uniform(0.5, 2.0, 6 * nbody)
    A = D @ np.diag(kd) @ D.T
    q = rng.normal(size=D.shape[0])
    return A, q, D, kd


def test_lemke_vs_enumeration_unique(orc):
    rng = np.random.default_rng(21)
    for trial in range(60):
        m = int(rng.integers(1, 11))
        A, q, D, kd = random_contact_lcp(rng, m, nbody=max(2, m))
        if np.linalg.eigvalsh(A).min() < 1e-6:
            continue
        z, w, st, piv = orc.lemke(A, q)
        assert st == 0
        sols = enum_lcp(A, q)
        assert len(sols) >= 1
        assert np.allclose(z, sols[0], atol=1e-10 * (1 + np.abs(sols[0]).max()))


def test_lemke_vs_enumeration_psd(orc):
    """Singular A: gamma not unique, but A gamma (hence D gamma) is."""
    rng = np.random.default_rng(22)
    done = 0
    for trial in range(80):
        m = int(rng.integers(2, 9))
        A, q, D, kd = random_contact_lcp(rng, m, nbody=3, psd_extra=int(rng.integers(1, 3)))
        sols = enum_lcp(A, q)
        if not sols:
            continue  # infeasible instance
        z, w, st, piv = orc.lemke(A, q)
        assert st == 0
        assert np.all(z >= 0)
        assert np.all(w >= -1e-10 * (1 + abs(q).max()))
        assert abs(z @ w) < 1e-9 * (1 + abs(q).max())
        Dz = (D.T @ z)
        Ds = D.T @ sols[0]
        assert np.allclose(Dz, Ds, atol=1e-8 * (1 + np.abs(Ds).max()))
        done += 1
    assert done > 20


def test_lemke_invariants_and_cqp_optimality(orc):
    rng = np.random.default_rng(23)
    for m in (50, 200):
        A, q, D, kd = random_contact_lcp(rng, m, nbody=m // 2)
        A += 1e-3 * np.eye(m)
        z, w, st, piv = orc.lemke(A, q)
        assert st == 0
        scale = 1 + abs(q).max()
        assert z.min() >= 0
        assert w.min() >= -1e-11 * scale
        assert np.max(np.minimum(z, np.abs(w)) * (z > 0)) < 1e-10 * scale
        f0 = 0.5 * z @ A @ z + q @ z
        for _ in range(50):
            y = np.maximum(z + rng.normal(size=m) * 1e-3, 0)
            assert 0.5 * y @ A @ y + q @ y >= f0 - 1e-12 * scale


def test_lemke_dgamma_unique_under_row_order(orc):
    rng = np.random.default_rng(24)
    A, q, D, kd = random_contact_lcp(rng, 30, nbody=6, psd_extra=5)
    z, w, st, _ = orc.lemke(A, q)
    if st != 0:
        pytest.skip("infeasible random instance")
    perm = rng.permutation(q.shape[0])
    z2, w2, st2, _ = orc.lemke(A[np.ix_(perm, perm)], q[perm])
    assert st2 == 0
    assert np.allclose(D.T @ z, D[perm].T @ z2, atol=1e-8 * (1 + np.abs(D.T @ z).max()))


def test_lemke_trivial_cases(orc):
    z, w, st, _ = orc.lemke(np.eye(3), np.array([1.0, 2.0, 3.0]))
    assert st == 0 and np.all(z == 0)
    z, w, st, _ = orc.lemke(np.zeros((0, 0)), np.zeros(0))
    assert st == 0 and z.size == 0
    # 1x1: z = -q/a when q < 0
    z, w, st, _ = orc.lemke(np.array([[2.0]]), np.array([-3.0]))
    assert st == 0 and abs(z[0] - 1.5) < 1e-15 and abs(w[0]) < 1e-15


def cell_list_pairs(x, rb, box, skin):
    """Independent cell-list construction of the same pair set."""
    n = x.shape[0]
    cut = 2 * rb.max() + skin
    nc = np.maximum((box // cut).astype(int), 1)
    cell = (np.floor(x / box * nc).astype(int)) % nc
    buckets = {}
    for i in range(n):
        buckets.setdefault(tuple(cell[i]), []).append(i)
    out = set()
    for i in range(n):
        for off in itertools.product((-1, 0, 1), repeat=3):
            key = tuple((cell[i] + np.array(off)) % nc)
            for j in buckets.get(key, ()):
                if j <= i:
                    continue
                d = x[j] - x[i]
                d = d - box * np.rint(d / box)
                if d @ d <= (rb[i] + rb[j] + skin) ** 2:
                    out.add((i, j))
    return out


def test_pairs_vs_cell_list(orc):
    rng = np.random.default_rng(25)
    for n, side in ((300, 12.0), (500, 15.0)):
        x = rng.random((n, 3)) * side
        rb = rng.uniform(0.4, 1.0, n)
        box = np.array([side] * 3)
        pairs = orc.candidate_pairs(x, rb, box, 0.05)
        # sorted i-major, j ascending
        keys = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
        assert np.all(np.diff(keys) > 0)
        assert set(map(tuple, pairs.tolist())) == cell_list_pairs(x, rb, box, 0.05)


def test_pairs_threshold_inclusive_and_open_axes(orc):
    # exactly at the cutoff: included (<=); beyond: excluded
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 3.0000001, 0.0]])
    rb = np.array([0.75, 0.75, 0.75])
    pairs = orc.candidate_pairs(x, rb, np.zeros(3), 0.5)
    assert pairs.tolist() == [[0, 1]]
    # periodic image across the boundary
    x = np.array([[0.1, 5.0, 5.0], [9.9, 5.0, 5.0]])
    pairs = orc.candidate_pairs(x, np.array([0.1, 0.1]), np.array([10.0, 10.0, 10.0]), 0.0)
    assert pairs.tolist() == [[0, 1]]
    pairs = orc.candidate_pairs(x, np.array([0.1, 0.1]), np.zeros(3), 0.0)
    assert pairs.tolist() == []
