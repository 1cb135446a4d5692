"""FP64 reference of the learned SNSD guess network: features, forward pass,
loss and backward pass (plain numpy).

TEST INFRASTRUCTURE ONLY: used by the tests to check the GPU kernels; the
library never imports it.  The network and loss are the library's own
definition (the paper has no learned component): 16 (13 used) -> 128 -> 128 ->
128 -> 8 (5 used), ReLU; loss per sample |o[0:3] - t|^2 + w_phi (o[3] - phi)^2
+ w_trust BCE(o[4], 1[|o[0:3] - t|^2 < trust_tol |t|^2]), averaged over the
batch, where t is the target correction from the analytic seed.
"""
import numpy as np

H, IN, OUT = 128, 16, 8
CORR_SCALE = 32.0  # the learned correction is scaled by this factor
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (OUT, H)), ("b4", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def init_params(rng, scale=1.0):
    """He-initialised parameters with the padded entries at zero."""
    p = np.zeros(NPARAMS)
    o = 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        if name.startswith("W"):
            w = rng.normal(0.0, scale * np.sqrt(2.0 / shape[1]), size=shape)
            if name == "W4":
                w[5:, :] = 0.0
            p[o:o + k] = w.ravel()
        o += k
    return p


def forward(p, X):
    w = unpack(p)
    acts = [np.asarray(X, dtype=np.float64)]
    h = acts[0]
    for l in (1, 2, 3):
        h = np.maximum(h @ w[f"W{l}"].T + w[f"b{l}"], 0.0)
        acts.append(h)
    o = h @ w["W4"].T + w["b4"]
    return o, acts


def loss_and_grad(p, X, T, w_phi=0.1, w_trust=0.1, trust_tol=0.01):
    w = unpack(p)
    o, acts = forward(p, X)
    B = X.shape[0]
    T = np.asarray(T, dtype=np.float64)
    r = o[:, :3] - T[:, :3]
    en = np.sum(r * r, axis=1)
    rp = o[:, 3] - T[:, 3]
    y = (en < trust_tol * np.sum(T[:, :3] ** 2, axis=1)).astype(np.float64)
    z = o[:, 4]
    bce = np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))
    L = np.mean(en + w_phi * rp * rp + w_trust * bce)
    dO = np.zeros_like(o)
    dO[:, :3] = 2 * r / B
    dO[:, 3] = 2 * w_phi * rp / B
    dO[:, 4] = w_trust * (1 / (1 + np.exp(-z)) - y) / B
    grads = {}
    dZ = dO
    for l in (4, 3, 2, 1):
        hprev = acts[l - 1]
        grads[f"W{l}"] = dZ.T @ hprev
        grads[f"b{l}"] = dZ.sum(axis=0)
        if l > 1:
            dH = dZ @ w[f"W{l}"]
            dZ = dH * (acts[l - 1] > 0)
    g = np.concatenate([grads[name].ravel() for name, _ in SHAPES])
    return L, g


def quat_rot(q):
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    s, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - s * z)
    R[..., 0, 2] = 2 * (x * z + s * y)
    R[..., 1, 0] = 2 * (x * y + s * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - s * x)
    R[..., 2, 0] = 2 * (x * z - s * y)
    R[..., 2, 1] = 2 * (y * z + s * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def features(pairs, x, q, axes, box, snsd_out=None):
    """Features (P, 16) and, with the SNSD outputs, targets (P, 4)."""
    i, j = pairs[:, 0], pairs[:, 1]
    d = x[j] - x[i]
    for k in range(3):
        if box[k] > 0:
            d[:, k] -= box[k] * np.rint(d[:, k] / box[k])
    qa = q[i] / np.linalg.norm(q[i], axis=1, keepdims=True)
    qb = q[j] / np.linalg.norm(q[j], axis=1, keepdims=True)
    R = quat_rot(qa)
    s = axes[i].max(axis=1) + axes[j].max(axis=1)
    f = np.zeros((pairs.shape[0], 16))
    f[:, 0:3] = np.einsum("pki,pk->pi", R, d) / s[:, None]
    conj = qa * np.array([1.0, -1.0, -1.0, -1.0])
    s1, v1 = conj[:, :1], conj[:, 1:]
    s2, v2 = qb[:, :1], qb[:, 1:]
    qr = np.concatenate([s1 * s2 - np.sum(v1 * v2, axis=1, keepdims=True), s1 * v2 + s2 * v1 + np.cross(v1, v2)],
                        axis=1)
    qr *= np.where(qr[:, :1] < 0, -1.0, 1.0)
    f[:, 3:7] = qr
    f[:, 7:10] = axes[i]
    f[:, 10:13] = axes[j]
    # analytic seed (P_a + P_b)^-1 d, normalised, in a's frame
    Rb = quat_rot(qb)
    Pa = np.einsum("pij,pj,pkj->pik", R, axes[i] ** 2, R)
    Pb = np.einsum("pij,pj,pkj->pik", Rb, axes[j] ** 2, Rb)
    w = np.linalg.solve(Pa + Pb, d[:, :, None])[:, :, 0]
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    seed = np.einsum("pki,pk->pi", R, w)
    f[:, 13:16] = seed
    t = None
    if snsd_out is not None:
        n = snsd_out[:, 1:4]
        t = np.zeros((pairs.shape[0], 4))
        t[:, :3] = CORR_SCALE * (np.einsum("pki,pk->pi", R, n) - seed)
        t[:, 3] = snsd_out[:, 0] / s
    return f, t
