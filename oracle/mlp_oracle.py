"""FP64 reference of the learned Voigt surrogate (the 2-64-64-64-1 SiLU network).

TEST INFRASTRUCTURE, like ``marfa_oracle``: only tests/, ``__graft_entry__.smoke()``
and bench.py may import it; the CUDA path has its own implementation of the same
contract and shares no code with this module.

The surrogate is not part of the paper. Its contract, which the CUDA path implements
independently:

* features  u1 = ln y,  u2 = ln(1 + |x| / (1 + y));
* baseline  K0(x, y) = exp(-x^2) / (1 + 2y/sqrt(pi)) + y / (sqrt(pi) (x^2 + y^2 + 1)),
  a Gauss core plus Lorentz wing with the right limits at x = 0, in the far wing and for
  large y, so that ln(K / K0) stays within [-0.9, 0.5] over the training domain;
* the network predicts t = ln(K(x, y) / K0(x, y)), so K = K0 exp(t);
* layers: z1 = W1 u + b1, a1 = silu(z1); z2 = W2 a1 + b2, a2 = silu(z2);
  z3 = W3 a2 + b3, a3 = silu(z3); t = W4 a3 + b4, with silu(z) = z / (1 + e^-z);
* parameters are packed in this order: W1 [64][2], b1 [64], W2 [64][64], b2 [64],
  W3 [64][64], b3 [64], W4 [64], b4 [1] (8,577 floats, W row-major [out][in]);
* loss = mean over the batch of (t_pred - t)^2;
* inference precision: W2, W3 and the activations a1, a2 are rounded to BF16 (round to
  nearest even), everything else stays FP32 or wider; ``forward(..., bf16=True)`` applies
  exactly these roundings to the FP64 evaluation.

The samples the network is trained on come from ``marfa_oracle.voigt_K`` (the FP64
Faddeeva function): y log-uniform in [1e-4, 10], |x| half uniform in [0, 12] and half
log-uniform in [1e-2, 1e3].
"""
from __future__ import annotations

import math

import numpy as np

from . import marfa_oracle as O

H = 64
SIZES = [("W1", (H, 2)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("W4", (H,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)
assert N_PARAMS == 8577


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(x, y):
    x = np.abs(np.asarray(x, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    return np.stack([np.log(y), np.log1p(x / (1.0 + y))], axis=-1)


def baseline(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sp = math.sqrt(math.pi)
    return np.exp(-x * x) / (1.0 + 2.0 * y / sp) + y / (sp * (x * x + y * y + 1.0))


def target(x, y):
    return np.log(O.voigt_K(x, y) / baseline(x, y))


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64: BF16 keeps the
    top 16 bits of the IEEE float32 pattern."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, u, bf16_inference: bool = False):
    P = unpack(params)
    q = bf16 if bf16_inference else (lambda a: a)
    z1 = u @ P["W1"].T + P["b1"]
    a1 = q(silu(z1))
    z2 = a1 @ q(P["W2"]).T + P["b2"]
    a2 = q(silu(z2))
    z3 = a2 @ q(P["W3"]).T + P["b3"]
    a3 = silu(z3)
    t = a3 @ P["W4"] + P["b4"][0]
    return t, (u, z1, a1, z2, a2, z3, a3)


def loss_and_grad(params, u, t_true, bf16_inference: bool = False):
    """Mean squared error and its gradient with respect to the packed parameters. With
    bf16_inference the forward pass rounds as inference does and the backward pass takes
    each rounding as the identity (straight-through), using the rounded W2, W3."""
    P = unpack(params)
    t, (u, z1, a1, z2, a2, z3, a3) = forward(params, u, bf16_inference)
    if bf16_inference:
        P = dict(P, W2=bf16(P["W2"]), W3=bf16(P["W3"]))
    n = len(t)
    r = t - t_true
    loss = float(np.mean(r * r))
    d4 = 2.0 * r / n                         # dL/dt
    g = {"W4": a3.T @ d4, "b4": np.array([d4.sum()])}
    d3 = np.outer(d4, P["W4"]) * dsilu(z3)   # dL/dz3
    g["W3"] = d3.T @ a2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ P["W3"]) * dsilu(z2)
    g["W2"] = d2.T @ a1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * dsilu(z1)
    g["W1"] = d1.T @ u
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights (uniform +-sqrt(6 / fan_in)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            lim = math.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)


def samples(n: int, seed: int = 7):
    """Training samples (x, y, t) drawn from the surrogate's domain, t from the FP64
    Faddeeva function."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = np.exp(rng.uniform(math.log(1e-4), math.log(10.0), n))
    half = n // 2
    x = np.concatenate([rng.uniform(0.0, 12.0, half),
                        np.exp(rng.uniform(math.log(1e-2), math.log(1e3), n - half))])
    perm = rng.permutation(n)
    x = x[perm]
    return x, y, target(x, y)


def surrogate_K(params, x, y, bf16_inference: bool = False):
    """K predicted by the network (FP64 evaluation of given parameters)."""
    t, _ = forward(params, features(x, y), bf16_inference)
    return baseline(x, y) * np.exp(t)


def write_samples(path: str, n: int, seed: int = 7) -> None:
    """Store n training samples (x, y, t as float32 arrays) in an .npz file."""
    x, y, t = samples(n, seed)
    np.savez(path, x=x.astype(np.float32), y=y.astype(np.float32), t=t.astype(np.float32))


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description="write surrogate training samples from the FP64 Faddeeva")
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    write_samples(a.out, a.n, a.seed)
