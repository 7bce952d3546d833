"""Train the learned Voigt surrogate on the GPU and store its parameters.

    python -m paper_2411_03418_gb300.train_surrogate --samples S.npz --out W.npy

S.npz holds float32 arrays x, y, t (t = ln(K / K0) of the surrogate's contract, from an
FP64 Faddeeva evaluation). Training runs in libmarfa's own forward/backward and Adam
kernels (marfa_mlp_train), with the forward pass rounding to BF16 where inference
does; the result is a float32 vector of MARFA_MLP_PARAMS parameters (.npy). The script
then loads the parameters, builds the guard against the plain FP32 Voigt, and reports
how many guard cells it switched on.

surrogate_weights.npy beside this file came from this script with its defaults, on
samples written by ``python -m oracle.mlp_oracle --n 10000000 --out S.npz`` (the FP64
Faddeeva oracle, seed 7).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import marfa as M

H = 64


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (+-sqrt(6 / fan_in)), zero biases, in the packed order
    W1[64][2], b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for shape, fan_in in [((H, 2), 2), ((H,), 0), ((H, H), H), ((H,), 0), ((H, H), H), ((H,), 0),
                          ((H,), H), ((1,), 0)]:
        if fan_in:
            lim = math.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == M.MLP_PARAMS
    return p


def train(x, y, t, steps: int, batch: int, lr0: float, lr1: float, seed: int, init=None, qat: bool = True,
          chunk: int = 5000):
    """Train in chunks of `chunk` steps (one marfa_mlp_train call each, the cosine
    schedule split across them) and return (params, per-step loss curve)."""
    p = init_params(seed) if init is None else np.asarray(init, dtype=np.float32)
    curves = []
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        # the learning rate of a chunk follows the global cosine at its own start and end
        a = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * done / steps))
        b = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * (done + k) / steps))
        # each chunk restarts Adam's moments; rotate the data so chunks see new batches
        off = (done * batch) % len(x)
        xr, yr, tr = (np.roll(v, -off) for v in (x, y, t))
        p, c = M.marfa_mlp_train(p, xr, yr, tr, k, batch, a, b, qat)
        curves.append(c)
        done += k
    return p, np.concatenate(curves)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--samples", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=300000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr0", type=float, default=3e-3)
    ap.add_argument("--lr1", type=float, default=1e-6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--budget", type=float, default=6e-4)
    ap.add_argument("--lattice", type=int, default=32)
    ap.add_argument("--chunk", type=int, default=300000)
    a = ap.parse_args(argv)
    from . import build

    build.build()
    d = np.load(a.samples)
    x, y, t = d["x"], d["y"], d["t"]
    t0 = time.time()
    p, curve = train(x, y, t, a.steps, a.batch, a.lr0, a.lr1, a.seed, chunk=a.chunk)
    dt = time.time() - t0
    np.save(a.out, p)
    on, err = M.marfa_surrogate_load(p, a.budget, a.lattice)
    elig = err >= 0
    tail = curve[-max(1, len(curve) // 50):]
    print(json.dumps({"samples": int(len(x)), "steps": a.steps, "batch": a.batch, "train_s": round(dt, 2),
                      "loss_first": float(curve[0]), "loss_last": float(np.mean(tail)),
                      "rms_t_last": float(math.sqrt(np.mean(tail))), "guard_budget": a.budget, "guard_lattice": a.lattice,
                      "cells_eligible": int(elig.sum()), "cells_on": int(on),
                      "cell_err_median": float(np.median(err[elig])) if elig.any() else None}))


if __name__ == "__main__":
    main()
