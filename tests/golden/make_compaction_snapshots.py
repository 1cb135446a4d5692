"""Writes compaction1024_snapshots.npz: states of the FP64 oracle's own
trajectory through the 1,024-body version of the compacting-suspension
schedule (seed 1, semi-axes U[0.4, 1.0], volume fraction 0.1 -> 0.55 by affine
compaction over 2,000 overdamped steps of dt = 5e-3, eps_NCP = 1e-3 a_min,
skin = 0.1 a_min; the paper's Sec. 5.3 suspension restated as an affine box).

The stored arrays are inputs of the parity tests and of the benchmark's
subset check: C^k (positions, quaternions) and the box side before the listed
steps, plus the semi-axes.  Only the seeded scene generator and oracle/ are
used, so no stored state comes from the CUDA path.  The run takes a few hours
on one core (Lemke's method is cubic in the number of rows, ~3 per body at the
dense end):

    python tests/golden/make_compaction_snapshots.py [--checkpoint FILE]

--checkpoint saves the running state every 25 steps and resumes from it.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N_BODIES = 1024
SEED = 1
TOTAL_STEPS = 2000
SNAPSHOT_STEPS = (500, 1000, 1500, 1750, 1900, 1990)
OUT = os.path.join(HERE, "compaction1024_snapshots.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import relcp_oracle as O
    from paper_2506_14097_gb300 import scenes

    sc = scenes.suspension_scene(seed=SEED, n=N_BODIES, phi=0.1, phi_final=0.55, steps=TOTAL_STEPS, dt=5e-3)
    amin = float(sc.axes.min())
    rate = sc.meta["strain_rate"]
    x, q, box, k0 = sc.x, sc.q, np.asarray(sc.box), 0
    snaps = {}
    if args.checkpoint and os.path.exists(args.checkpoint):
        ck = np.load(args.checkpoint)
        x, q, box, k0 = ck["x"], ck["q"], ck["box"], int(ck["k"])
        for s in SNAPSHOT_STEPS:
            if f"x_{s}" in ck:
                snaps[s] = (ck[f"x_{s}"], ck[f"q_{s}"], ck[f"box_{s}"])
    last = max(SNAPSHOT_STEPS)
    t0 = time.time()
    for k in range(k0, last + 1):
        if k in SNAPSHOT_STEPS:
            snaps[k] = (x.copy(), q.copy(), box.copy())
        if k == last:
            break
        cfg = O.Config(dynamics=O.OVERDAMPED, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(box), skin=0.1 * amin,
                       strain_rate=rate)
        r = O.step(cfg, x, q, sc.axes)
        if r.status != 0:
            raise RuntimeError(f"oracle step {k} returned status {r.status}")
        x, q, box = r.x, r.q, np.asarray(r.box)
        if args.checkpoint and (k + 1) % 25 == 0:
            extra = {}
            for s, (xs, qs, bs) in snaps.items():
                extra.update({f"x_{s}": xs, f"q_{s}": qs, f"box_{s}": bs})
            np.savez(args.checkpoint, x=x, q=q, box=box, k=k + 1, **extra)
            print(f"step {k + 1}: phi {sc.meta['volume'] / np.prod(box):.4f}, rows {r.rows_ia.size}, "
                  f"depth {r.depth}, {time.time() - t0:.0f} s", flush=True)
    steps = np.array(sorted(snaps), dtype=np.int64)
    np.savez(args.out, steps=steps, axes=sc.axes, strain_rate=rate, dt=sc.dt, seed=SEED,
             x=np.stack([snaps[s][0] for s in steps]), q=np.stack([snaps[s][1] for s in steps]),
             box=np.stack([snaps[s][2] for s in steps]), volume=sc.meta["volume"])
    print("wrote", args.out)


if __name__ == "__main__":
    main()
