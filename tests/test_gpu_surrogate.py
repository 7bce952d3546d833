"""The learned Voigt surrogate on the GPU: training kernels against the FP64 reference
(oracle/mlp_oracle.py), BF16 tensor-core inference against the FP64 forward of the same
parameters, the guard (judged by the plain FP32 Voigt), and the absorption path with the
surrogate against the FP64 eleven-grid oracle at 1e-3 relative."""
import math
import os
import time

import numpy as np
import pytest

from oracle import marfa_oracle as O
from oracle import mlp_oracle as MO
from workloads import tiny_workload

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2411_03418_gb300", "surrogate_weights.npy")
BUDGET = 6e-4       # guard budget against the plain FP32 Voigt
LATTICE = 32        # guard lattice points per cell side
SURR_RTOL = 1e-3    # k(nu) with the surrogate against the FP64 oracle
FLOOR = 1e-8


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_03418_gb300 import build, marfa
    build.build()
    marfa.load()
    return marfa


@pytest.fixture(scope="module")
def weights():
    if not os.path.exists(WEIGHTS):
        pytest.skip("trained surrogate parameters not present")
    return np.load(WEIGHTS).astype(np.float32)


@pytest.fixture
def loaded(M, weights):
    on, err = M.marfa_surrogate_load(weights, BUDGET, LATTICE)
    yield on, err
    M.marfa_surrogate_unload()


def guard_cell(x, y):
    """Guard cell index of (x, y) (float32 inputs), -1 outside: |x| by 1/8 below 12; y by
    binary exponent e in [-14, 3] and its two leading mantissa bits."""
    x = np.abs(np.asarray(x, np.float32))
    y = np.asarray(y, np.float32)
    bits = y.view(np.uint32).astype(np.int64)
    e = (bits >> 23) - 127
    iy = (e + 14) * 4 + ((bits >> 21) & 3)
    ix = (x * np.float32(8)).astype(np.int64)
    ok = (x < 12) & (y >= np.float32(2.0 ** -14)) & (y < 16)
    return np.where(ok, iy * 96 + ix, -1)


def rand_params(seed):
    rng = np.random.default_rng(seed)
    d = MO.unpack(MO.init_params(seed))
    for b in ("b1", "b2", "b3", "b4"):
        d[b] = rng.uniform(-0.5, 0.5, d[b].shape)
    return MO.pack(d).astype(np.float32)


# ------------------------------------------------------------ training kernels
@pytest.mark.parametrize("qat", [False, True])
def test_loss_and_gradient_match_oracle(M, qat):
    p = rand_params(5)
    x, y, t = MO.samples(777, seed=11)  # 48 full tiles of 16 and a ragged one
    x, y, t = (v.astype(np.float32) for v in (x, y, t))
    loss, g = M.marfa_mlp_loss_grad(p, x, y, t, qat=qat)
    u = MO.features(x.astype(np.float64), y.astype(np.float64))
    lref, gref = MO.loss_and_grad(p.astype(np.float64), u, t.astype(np.float64), bf16_inference=qat)
    assert abs(loss / lref - 1) < (2e-3 if qat else 2e-5), (loss, lref)
    err = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    # FP32 sums of 777 products (qat: an FP32 activation can round to the other BF16
    # neighbour than the FP64 one; each such flip moves one activation by 2^-8)
    assert err < (2e-2 if qat else 1e-4), err
    if not qat:
        assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()


def test_training_reduces_loss(M):
    x, y, t = MO.samples(65536, seed=21)
    x, y, t = (v.astype(np.float32) for v in (x, y, t))
    p0 = rand_params(2)
    p, curve = M.marfa_mlp_train(p0, x, y, t, steps=400, batch=4096, lr0=3e-3, lr1=3e-4, qat=True)
    assert np.all(np.isfinite(curve)) and np.all(np.isfinite(p))
    assert curve[-20:].mean() < 0.2 * curve[:5].mean(), (curve[:5], curve[-20:])
    # the trained parameters' loss, by the FP64 reference, agrees with the GPU's
    loss, _ = M.marfa_mlp_loss_grad(p, x[:4096], y[:4096], t[:4096], qat=False)
    lref, _ = MO.loss_and_grad(p.astype(np.float64), MO.features(x[:4096], y[:4096]), t[:4096].astype(np.float64))
    assert abs(loss / lref - 1) < 1e-4
    # deterministic: the same call gives the same parameters bit for bit
    p2, _ = M.marfa_mlp_train(p0, x, y, t, steps=400, batch=4096, lr0=3e-3, lr1=3e-4, qat=True)
    assert np.array_equal(p, p2)


def test_training_rejects_bad_input(M):
    p = rand_params(1)
    x = np.ones(8, np.float32)
    with pytest.raises(M.MarfaError):
        M.marfa_mlp_train(p, x, -x, x, steps=1, batch=8, lr0=1e-3, lr1=1e-3)
    with pytest.raises(M.MarfaError):
        M.marfa_mlp_train(p, x, x, x, steps=1, batch=M.MLP_MAX_BATCH + 1, lr0=1e-3, lr1=1e-3)
    with pytest.raises(M.MarfaError):
        M.marfa_mlp_loss_grad(p, np.ones(M.MLP_MAX_BATCH + 1, np.float32), np.ones(M.MLP_MAX_BATCH + 1, np.float32),
                              np.ones(M.MLP_MAX_BATCH + 1, np.float32))


# ------------------------------------------------------------ inference
def test_inference_matches_fp64_forward(M, weights, loaded):
    rng = np.random.default_rng(3)
    n = 20000
    y = np.exp(rng.uniform(math.log(1e-4), math.log(10), n)).astype(np.float32)
    x = np.concatenate([rng.uniform(-12, 12, n // 2), np.exp(rng.uniform(math.log(1e-2), math.log(1e3), n - n // 2))])
    x = x.astype(np.float32)
    got = M.marfa_surrogate_eval(x, y, guarded=False).astype(np.float64)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    ref = MO.surrogate_K(weights.astype(np.float64), xd, yd, bf16_inference=True)
    dt = np.abs(np.log(got / ref))
    # tanh.approx in the BF16 layers moves an activation to the neighbouring BF16 value
    # now and then (2^-8 relative each); FP32 accumulation order differs
    assert dt.max() < 1.5e-2, dt.max()
    assert dt.mean() < 1.5e-3, dt.mean()


def test_guard_cells_and_guarded_evaluation(M, weights, loaded):
    on, err = loaded
    assert on > 0
    elig = err >= 0
    assert on == int(((err >= 0) & (err <= BUDGET)).sum())
    rng = np.random.default_rng(4)
    n = 200000
    y = np.exp(rng.uniform(math.log(5e-5), math.log(12), n)).astype(np.float32)
    x = rng.uniform(-13, 13, n).astype(np.float32)
    got = M.marfa_surrogate_eval(x, y, guarded=True).astype(np.float64)
    plain = M.marfa_diag_voigt(x, y).astype(np.float64)
    ref = O.voigt_K(x.astype(np.float64), y.astype(np.float64))
    cell = guard_cell(x, y)
    onmask = np.zeros(n, bool)
    ok = cell >= 0
    onmask[ok] = (err.ravel()[cell[ok]] >= 0) & (err.ravel()[cell[ok]] <= BUDGET)
    assert onmask.sum() > 1000
    # where the guard is off the plain FP32 Voigt is used unchanged
    np.testing.assert_array_equal(got[~onmask], plain[~onmask])
    # where it is on the surrogate holds the budget (plus the plain FP32 error) off the lattice too
    rel = np.abs(got[onmask] / ref[onmask] - 1)
    assert rel.max() < SURR_RTOL, rel.max()
    # no cell outside the eligible domain is on
    assert np.all(~onmask[(y < 1e-4) | (y > 10) | (np.abs(x) >= 12)])


# ------------------------------------------------------------ absorption with the surrogate
def _run(M, wl, counted=False):
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    rq = M.request_of(wl)
    if counted:
        return M.marfa_diag_absorption_counted_surrogate(lines, M.levels_of(wl), wl.vmr, rq)
    n = M.marfa_num_points(wl.nu_lo, wl.nu_hi)
    out = np.empty((wl.n_levels, n), dtype=np.float32)
    M.marfa_absorption(lines, M.levels_of(wl), wl.vmr, rq, out, None)
    return out


def _assert_close(got, ref, rtol, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    mx = np.abs(ref).max()
    big = np.abs(ref) > FLOOR * mx
    rel = np.abs(got[big] / ref[big] - 1)
    assert rel.max() < rtol, f"{what}: max rel err {rel.max():.3e}"
    if (~big).any():
        assert np.abs(got[~big] - ref[~big]).max() <= rtol * FLOOR * mx


SURR_CASES = [
    # Venus-like levels with narrow (low p) and broad (high p) lines, chi-factor on
    tiny_workload(31, 400, 2400.0, 2402.5, 25.0, T=(735.0, 400.0, 230.0, 170.0), p=(92.0, 1.0, 1e-2, 1e-5),
                  chi="tonkov", chi_species=1),
    tiny_workload(32, 200, 3000.0, 3001.0, 10.0, T=(296.0, 250.0), p=(0.1, 1e-3), spread=2.0),
]


@pytest.mark.parametrize("case", range(len(SURR_CASES)))
def test_surrogate_absorption_vs_oracle(M, loaded, case):
    wl = SURR_CASES[case].with_(surrogate=1)
    k, counts, sc = _run(M, wl, counted=True)
    assert sc.sum() > 0, "the guard let no evaluation through"
    assert np.all(sc <= counts)
    plain = _run(M, SURR_CASES[case])
    for lev in range(wl.n_levels):
        ref = O.eleven_grid(wl, lev)
        _assert_close(k[lev], ref, SURR_RTOL, f"surrogate level {lev}")
        _assert_close(k[lev], plain[lev], SURR_RTOL, f"surrogate vs plain level {lev}")


def test_surrogate_batch_matches_single(M, loaded):
    """A batch holding a surrogate request runs every request through the
    surrogate-capable kernels: the surrogate request's result is the same bit for bit as
    alone; the plain request takes, alone, the plain kernels, whose sums run in another
    order (within FP32 rounding of the batch result)."""
    a = SURR_CASES[0].with_(surrogate=1)
    b = SURR_CASES[1]
    ka, kb = _run(M, a), _run(M, b)
    la = M.marfa_prepare_lines(a.lines, a.species)
    lb = M.marfa_prepare_lines(b.lines, b.species)
    oa = np.empty_like(ka)
    ob = np.empty_like(kb)
    M.marfa_absorption_batch([la, lb], [M.levels_of(a), M.levels_of(b)], [a.vmr, b.vmr],
                             [M.request_of(a), M.request_of(b)], [oa, ob])
    assert np.array_equal(oa, ka)
    for lev in range(b.n_levels):
        _assert_close(ob[lev], kb[lev], 1e-5, f"plain request in a surrogate batch, level {lev}")


def test_surrogate_plan_matches_call(M, loaded):
    """A captured plan of a surrogate request (grids whose guard never fires for the batch
    switched to the plain kernels) against the direct call and the oracle."""
    import torch
    wl = SURR_CASES[0].with_(surrogate=1)
    direct = _run(M, wl)
    lines = M.marfa_prepare_lines(wl.lines, wl.species)
    out = torch.empty(direct.shape, dtype=torch.float32, device="cuda")
    plan = M.marfa_plan_create([lines], [M.levels_of(wl)], [wl.vmr], [M.request_of(wl)], [out])
    out.fill_(float("nan"))
    M.marfa_plan_execute(plan)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for lev in range(wl.n_levels):
        _assert_close(got[lev], direct[lev], 1e-5, f"plan vs call level {lev}")
        _assert_close(got[lev], O.eleven_grid(wl, lev), SURR_RTOL, f"plan vs oracle level {lev}")
    M.marfa_plan_destroy(plan)


def test_surrogate_request_validation(M, weights):
    wl = SURR_CASES[1].with_(surrogate=1)
    M.marfa_surrogate_unload()
    with pytest.raises(M.MarfaError, match="none is loaded"):
        _run(M, wl)
    M.marfa_surrogate_load(weights, BUDGET, LATTICE)
    try:
        with pytest.raises(M.MarfaError, match="Voigt"):
            _run(M, wl.with_(shape="lorentz"))
        bad = wl.with_(surrogate=2)
        with pytest.raises(M.MarfaError):
            _run(M, bad)
    finally:
        M.marfa_surrogate_unload()


def test_surrogate_gain_report(M, loaded):
    """What the surrogate buys on a narrow-line window: the same request timed with the
    plain FP32 Voigt and with the surrogate (both within their tolerances of the oracle
    in the tests above). The gain is reported, not asserted: the surrogate's cost per
    evaluation (two 64x64 BF16 layers) exceeds the plain evaluation's."""
    import torch
    wl = tiny_workload(33, 3000, 2500.0, 2510.0, 25.0, T=tuple(np.linspace(300, 170, 12)),
                       p=tuple(np.geomspace(1e-1, 1e-5, 12)), chi="tonkov", chi_species=1)
    res = {}
    for s in (0, 1):
        w = wl.with_(surrogate=s)
        lines = M.marfa_prepare_lines(w.lines, w.species)
        rq = M.request_of(w)
        n = M.marfa_num_points(w.nu_lo, w.nu_hi)
        out = torch.empty((w.n_levels, n), dtype=torch.float32, device="cuda")
        for _ in range(2):
            M.marfa_absorption(lines, M.levels_of(w), w.vmr, rq, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            M.marfa_absorption(lines, M.levels_of(w), w.vmr, rq, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        res[s] = (time.perf_counter() - t0) / 5
    _, counts, sc = _run(M, wl.with_(surrogate=1), counted=True)
    print(f"\nsurrogate gain: plain {res[0] * 1e3:.2f} ms, surrogate {res[1] * 1e3:.2f} ms, "
          f"speed-up {res[0] / res[1]:.3f}x, surrogate share of evaluations {sc.sum() / counts.sum():.3f}")
    assert res[0] > 0 and res[1] > 0
