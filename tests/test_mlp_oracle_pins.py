"""CPU pins of the surrogate's FP64 reference (oracle/mlp_oracle.py): backpropagation
against central finite differences, hand-built networks with closed-form outputs, the
baseline's limits, BF16 rounding against its bit-level definition, and the sample
generator's domain."""
import math

import numpy as np
import pytest

from oracle import marfa_oracle as O
from oracle import mlp_oracle as MO


def _rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = MO.init_params(seed)
    # non-zero biases so that their gradients are exercised too
    d = MO.unpack(p.copy())
    for b in ("b1", "b2", "b3", "b4"):
        d[b] = rng.uniform(-0.5, 0.5, d[b].shape)
    return MO.pack(d) * scale


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_matches_finite_differences(bf16):
    x, y, t = MO.samples(24, seed=3)
    u = MO.features(x, y)
    p = _rand_params(1)
    loss, g = MO.loss_and_grad(p, u, t)
    assert loss > 0 and g.shape == (MO.N_PARAMS,)
    rng = np.random.default_rng(0)
    # every block of the packing, plus random entries
    idx = [0, 1, 127, 128, 191, 192, 4287, 4288, 4351, 4352, 8447, 8448, 8511, 8512, 8575, 8576]
    idx += list(rng.integers(0, MO.N_PARAMS, 40))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = MO.loss_and_grad(p + e, u, t)
        lm, _ = MO.loss_and_grad(p - e, u, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])
    if bf16:
        # straight-through gradient: the exact gradient of the network whose W2, W3 are the
        # rounded ones, evaluated with the rounded activations held fixed, so at the points
        # where no activation sits on a rounding boundary it equals the FP64 gradient of the
        # same network with activations rounded; compare its W4 block, whose chain has no
        # rounding, with finite differences of the bf16 loss
        lq, gq = MO.loss_and_grad(p, u, t, bf16_inference=True)
        for i in range(8512, 8577):
            e = np.zeros_like(p)
            e[i] = h
            lp, _ = MO.loss_and_grad(p + e, u, t, bf16_inference=True)
            lm, _ = MO.loss_and_grad(p - e, u, t, bf16_inference=True)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gq[i]) <= 1e-6 * (1 + abs(gq[i])), (i, fd, gq[i])


def test_hand_built_network_closed_form():
    d = {name: np.zeros(shape) for name, shape in MO.SIZES}
    d["b4"][0] = 0.3
    p = MO.pack(d)
    x = np.array([0.0, 0.7, 5.0, 300.0])
    y = np.array([1e-3, 0.2, 2.0, 9.0])
    np.testing.assert_allclose(MO.surrogate_K(p, x, y), MO.baseline(x, y) * math.exp(0.3), rtol=1e-15)
    # a chain u2 -> unit 1 of layer 1 -> unit 0 of layer 2 (W2[0][1]) -> unit 0 of layer 3
    # -> output: t = silu(silu(silu(u2))) + W1 and W2 transposition shows up as t = 0
    d = {name: np.zeros(shape) for name, shape in MO.SIZES}
    d["W1"][1, 1] = 1.0
    d["W2"][0, 1] = 1.0
    d["W3"][0, 0] = 1.0
    d["W4"][0] = 1.0
    p = MO.pack(d)
    u = MO.features(x, y)
    t, _ = MO.forward(p, u)
    s = lambda z: z / (1 + np.exp(-z))
    np.testing.assert_allclose(t, s(s(s(np.log1p(np.abs(x) / (1 + y))))), rtol=1e-14)
    assert np.all(t[1:] > 0)


def test_features_and_baseline_limits():
    u = MO.features(np.array([0.0, -3.0]), np.array([0.5, 2.0]))
    np.testing.assert_allclose(u[:, 0], np.log([0.5, 2.0]), rtol=1e-15)
    np.testing.assert_allclose(u[:, 1], [0.0, math.log(2.0)], rtol=1e-15)
    # K0(0, 0) = K(0, 0) = 1; far wing K0 -> y / (sqrt(pi) x^2), the Lorentz limit of K
    assert MO.baseline(0.0, 0.0) == 1.0
    x, y = 1e3, 1.0
    assert abs(MO.baseline(x, y) / (y / (math.sqrt(math.pi) * x * x)) - 1) < 3e-6
    assert abs(MO.target(np.array([x]), np.array([y]))[0]) < 1e-5
    # target = ln(K / K0) with K the FP64 Faddeeva (pinned in test_oracle_pins)
    xs, ys = np.array([0.3, 4.0]), np.array([0.01, 3.0])
    np.testing.assert_allclose(np.exp(MO.target(xs, ys)) * MO.baseline(xs, ys), O.voigt_K(xs, ys), rtol=1e-14)


def test_bf16_rounding_bit_definition():
    one = 1.0
    cases = [
        (one, one),
        (one + 2.0 ** -8, one),                       # tie, 1.0 is even
        (one + 3 * 2.0 ** -8, one + 2.0 ** -6),        # tie, rounds up to the even mantissa
        (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7),
        (-(one + 2.0 ** -7), -(one + 2.0 ** -7)),      # representable
    ]
    for v, want in cases:
        assert MO.bf16(np.array([v]))[0] == want, (v, MO.bf16(np.array([v]))[0], want)
    # the result always has its low 16 float32 bits clear and is within half a BF16 ulp
    r = np.random.default_rng(1).standard_normal(10000) * 100
    q = MO.bf16(r)
    assert np.all(q.astype(np.float32).view(np.uint32) & 0xFFFF == 0)
    ulp = 2.0 ** (np.floor(np.log2(np.abs(r.astype(np.float32)))) - 7)
    assert np.all(np.abs(q - r.astype(np.float32)) <= ulp / 2 + 1e-30)


def test_samples_domain_and_target_range():
    x, y, t = MO.samples(20000, seed=7)
    assert np.all((y >= 1e-4) & (y <= 10)) and np.all((x >= 0) & (x <= 1e3))
    assert np.mean(x <= 12) > 0.5
    assert t.min() > -0.95 and t.max() < 0.55
    x2, y2, t2 = MO.samples(20000, seed=7)
    assert np.array_equal(x, x2) and np.array_equal(t, t2)


def test_pack_roundtrip():
    p = np.arange(MO.N_PARAMS, dtype=np.float64)
    d = MO.unpack(p)
    assert d["W2"][1, 0] == 192 + 64 and d["b4"][0] == 8576
    assert np.array_equal(MO.pack(d), p)
