"""Training loop of the learned SNSD guess: orchestration only.

harvest() collects (features, target) pairs that the method itself produces:
candidate pairs of simulation states, their FP64 SNSD solutions (shared normal
in body a's frame and Phi) and the network features -- every number comes from
the library's kernels (relcp_broadphase, relcp_snsd_eval, relcp_mlp_features).
train() runs Adam with the library's tensor-core forward/backward kernels
(relcp_mlp_train_step); PyTorch only holds the device buffers and shuffles
batch indices.
"""
from __future__ import annotations

import math

import numpy as np

from . import relcp as R
from . import scenes


def init_params(seed: int = 0):
    """He-initialised FP32 parameter vector (padded entries zero), on the GPU."""
    import torch

    rng = np.random.default_rng(seed)
    p = np.zeros(R.MLP_NPARAMS, dtype=np.float32)
    o = 0
    for rows, cols, is_w in ((128, 16, 1), (128, 1, 0), (128, 128, 1), (128, 1, 0), (128, 128, 1), (128, 1, 0),
                             (8, 128, 1), (8, 1, 0)):
        k = rows * cols
        if is_w:
            w = rng.normal(0.0, math.sqrt(2.0 / cols), size=(rows, cols)).astype(np.float32)
            if rows == 8:
                w[5:, :] = 0
            p[o:o + k] = w.ravel()
        o += k
    return torch.tensor(p, device="cuda")


def harvest_state(x, q, axes, box, skin):
    """Features and targets of every candidate pair of one state (device)."""
    import torch

    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    xd, qd, ad = dev(x), dev(q), dev(axes)
    rb = dev(np.asarray(axes).max(axis=1))
    pairs = R.relcp_broadphase(xd, rb, box, skin)
    if pairs.shape[0] == 0:
        return None, None
    out, _ = R.relcp_snsd_eval(pairs, xd, qd, ad, box, R.RELCP_FP64)
    return R.relcp_mlp_features(pairs, xd, qd, ad, box, out)


def harvest_compaction(n=4096, seed=11, steps=400, every=20, precision=R.RELCP_MIXED):
    """States along a compaction run of n ellipsoids (volume fraction 0.1 ->
    0.55 over `steps` steps), harvested every `every` steps."""
    import torch

    sc = scenes.suspension_scene(seed=seed, n=n, phi=0.1, phi_final=0.55, steps=steps, dt=5e-3)
    amin = float(sc.axes.min())
    cfg = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=precision, dt=sc.dt, eps_ncp=1e-3 * amin,
                        box=tuple(sc.box), skin=0.1 * amin, strain_rate=sc.meta["strain_rate"], length_scale=amin)
    sim = R.Simulation(cfg)
    sim.set_bodies(sc.x, sc.q, sc.axes)
    feats, targs = [], []
    for k in range(steps):
        if k % every == every - 1:
            x, q, _ = sim.bodies()
            f, t = harvest_state(x, q, sc.axes, R.relcp_get_box(sim.ctx), 0.1 * amin)
            if f is not None:
                feats.append(f)
                targs.append(t)
        sim.step(1, allow=(R.RELCP_ERR_NOT_CONVERGED,))
    sim.close()
    return torch.cat(feats), torch.cat(targs)


def train(feat, targets, epochs=30, batch=4096, lr=2e-3, seed=0, w_phi=0.1, w_trust=0.02, trust_tol=0.25,
          params=None, log=None):
    """Adam on the library's kernels; returns (params, list of epoch losses)."""
    import torch

    if params is None:
        params = init_params(seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    cfg = R.relcp_mlp_train_config()
    cfg.lr, cfg.beta1, cfg.beta2, cfg.eps = lr, 0.9, 0.999, 1e-8
    cfg.w_phi, cfg.w_trust, cfg.trust_tol = w_phi, w_trust, trust_tol
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    N = int(feat.shape[0])
    losses = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(N, device="cuda", generator=gen)
        tot, cnt = 0.0, 0
        for s0 in range(0, N - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            step += 1
            cfg.step = step
            tot += R.relcp_mlp_train_step(params, m, v, feat[idx].contiguous(), targets[idx].contiguous(), cfg)
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(ep, losses[-1])
    return params, losses
