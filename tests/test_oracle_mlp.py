"""Pins of the FP64 MLP reference: its backward pass against central finite
differences of its own loss (labels of the trust term held fixed), and its
features against the geometric definition (rotating the scene rigidly leaves
them unchanged; the target normal is the SNSD normal seen from body a)."""
import numpy as np

from oracle import mlp_oracle as M
from paper_2506_14097_gb300 import scenes


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = M.init_params(rng)
    p += rng.normal(0, 0.01, p.shape)  # nonzero biases
    X = rng.normal(size=(24, 16))
    T = rng.normal(size=(24, 4))
    for tol in (1e12, -1.0):  # all trust labels 1, then all 0: the loss is smooth
        L, g = M.loss_and_grad(p, X, T, 0.3, 0.2, tol)
        idx = rng.choice(np.nonzero(g)[0], 60, replace=False)
        h = 1e-6
        for k in idx:
            e = np.zeros_like(p)
            e[k] = h
            fd = (M.loss_and_grad(p + e, X, T, 0.3, 0.2, tol)[0] - M.loss_and_grad(p - e, X, T, 0.3, 0.2, tol)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * (1 + abs(g[k])), (k, fd, g[k])


def test_features_rigid_invariance_and_target(orc):
    rng = np.random.default_rng(4)
    n = 50
    x = rng.random((n, 3)) * 6
    q = scenes.random_quaternions(rng, n)
    axes = rng.uniform(0.4, 1.0, (n, 3))
    pairs = np.array([(i, i + 1) for i in range(n - 1)], dtype=np.int32)
    phi, nn, ra, rb, _ = orc.snsd(pairs, x, q, axes, np.zeros(3))
    out = np.concatenate([phi[:, None], nn, ra, rb], axis=1)
    f, t = M.features(pairs, x.copy(), q, axes, np.zeros(3), out)
    # a global rotation of the whole scene leaves the features and targets unchanged
    g = scenes.random_quaternions(rng, 1)[0]
    Rg = M.quat_rot(g[None])[0]
    x2 = x @ Rg.T
    qg = np.concatenate([[g[0] * q[:, 0] - q[:, 1:] @ g[1:]],
                         (g[0] * q[:, 1:] + q[:, :1] * g[1:] + np.cross(g[1:], q[:, 1:])).T]).T
    phi2, nn2, ra2, rb2, _ = orc.snsd(pairs, x2, qg, axes, np.zeros(3))
    out2 = np.concatenate([phi2[:, None], nn2, ra2, rb2], axis=1)
    f2, t2 = M.features(pairs, x2, qg, axes, np.zeros(3), out2)
    assert np.allclose(f, f2, atol=1e-9) and np.allclose(t, t2, atol=1e-8)
    # seed + target correction is the unit SNSD normal in a's frame
    assert np.allclose(np.linalg.norm(f[:, 13:16] + t[:, :3] / M.CORR_SCALE, axis=1), 1.0)
    assert np.allclose(np.linalg.norm(f[:, 13:16], axis=1), 1.0)
