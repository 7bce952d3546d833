"""ctypes binding of libmarfa (include/marfa.h): argument marshalling only.

Every function here has the name of the C entry point it calls and converts numpy
arrays, torch tensors and CUDA streams into plain pointers and sizes. All the
computation happens in the library's CUDA kernels; there is no fallback, and a
missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LINE_DTYPE = np.dtype([("nu0", "<f8"), ("S296", "<f4"), ("gamma_air", "<f4"), ("gamma_self", "<f4"),
                       ("E_lower", "<f4"), ("n_air", "<f4"), ("mol_iso", "<i4"), ("delta_air", "<f4")])
SPECIES_DTYPE = np.dtype([("mol_iso", "<i4"), ("chi_enabled", "<i4"), ("mass_amu", "<f8"), ("q_exp", "<f8")])
LEVEL_DTYPE = np.dtype([("T_K", "<f8"), ("p_atm", "<f8")])

SHAPES = {"lorentz": 0, "voigt": 1, "doppler": 2, "voigt_paper": 3, "user": 4, "const": 100, "quad": 101,
          "quart": 102}
CHI = {"none": 0, "tonkov": 1}
UNITS = {"sigma": 0, "k_cm1": 1, "k_km1": 2}
ERRORS = {-1: "MARFA_E_INVAL", -2: "MARFA_E_NOMEM", -3: "MARFA_E_CUDA", -4: "MARFA_E_IO",
          -5: "MARFA_E_INTERNAL"}


class MarfaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class marfa_request_t(C.Structure):
    _fields_ = [("nu_lo", C.c_double), ("nu_hi", C.c_double), ("cutoff", C.c_double),
                ("shape", C.c_int32), ("chi", C.c_int32), ("units", C.c_int32),
                ("surrogate", C.c_int32), ("R_w", C.c_int32), ("R_c", C.c_int32),
                ("stencil", C.c_int32)]


_LIB = None
EXPORTS = ["marfa_prepare_lines", "marfa_free_lines", "marfa_num_points", "marfa_absorption",
           "marfa_absorption_batch", "marfa_write_pt_table", "marfa_last_error", "marfa_diag_voigt",
           "marfa_diag_level_lines", "marfa_diag_owned", "marfa_diag_absorption_counted",
           "marfa_diag_kernel_timing", "marfa_absorption_noalloc", "marfa_mlp_loss_grad",
           "marfa_mlp_train", "marfa_surrogate_load", "marfa_surrogate_unload", "marfa_surrogate_eval",
           "marfa_diag_absorption_counted_surrogate", "marfa_plan_create", "marfa_plan_execute",
           "marfa_plan_info", "marfa_plan_destroy", "marfa_diag_absorption_counts", "marfa_read_par",
           "marfa_diag_pipe_rate", "marfa_diag_line_order", "marfa_diag_shape", "marfa_diag_variants",
           "marfa_diag_fail_alloc", "marfa_diag_device_memory", "marfa_diag_check",
           "marfa_plan_classes", "marfa_shape_user_set", "marfa_prepare_lines_batch"]

MLP_PARAMS = 8577
MLP_MAX_BATCH = 65536
GUARD_NX, GUARD_NY = 96, 72


class marfa_mlp_train_t(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("qat", C.c_int32), ("reserved", C.c_int32),
                ("lr0", C.c_float), ("lr1", C.c_float)]


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmarfa (built in-tree by paper_2411_03418_gb300.build). Raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libmarfa is not built ({p} missing): call paper_2411_03418_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "marfa_prepare_lines": (C.c_int, [vp, i64, vp, i32, C.POINTER(vp)]),
        "marfa_prepare_lines_batch": (C.c_int, [i32, vp, vp, vp, vp, vp]),
        "marfa_free_lines": (None, [vp]),
        "marfa_num_points": (i64, [dbl, dbl]),
        "marfa_absorption": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
        "marfa_absorption_batch": (C.c_int, [i32, vp, vp, vp, vp, vp, vp, vp]),
        "marfa_write_pt_table": (C.c_int, [C.c_char_p, i32, dbl, dbl, vp, i64]),
        "marfa_read_par": (C.c_int, [C.c_char_p, i64, vp, i64, C.POINTER(C.c_int64)]),
        "marfa_last_error": (C.c_char_p, []),
        "marfa_diag_voigt": (C.c_int, [vp, vp, vp, i64]),
        "marfa_diag_level_lines": (C.c_int, [vp, vp, vp, i32, vp, vp, vp, vp]),
        "marfa_diag_owned": (C.c_int, [vp, vp, vp, i32, vp, i32, i32, i64, i32, vp]),
        "marfa_diag_absorption_counted": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
        "marfa_diag_kernel_timing": (C.c_int, [i32, vp, vp]),
        "marfa_diag_pipe_rate": (C.c_int, [i32, vp]),
        "marfa_diag_line_order": (C.c_int, [vp, i64, vp]),
        "marfa_diag_shape": (C.c_int, [i32, vp, vp, vp, i64]),
        "marfa_absorption_noalloc": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
        "marfa_mlp_loss_grad": (C.c_int, [vp, vp, vp, vp, i64, i32, vp, vp]),
        "marfa_mlp_train": (C.c_int, [vp, vp, vp, vp, i64, vp, vp]),
        "marfa_surrogate_load": (C.c_int, [vp, C.c_float, i32, vp, vp]),
        "marfa_surrogate_unload": (C.c_int, []),
        "marfa_surrogate_eval": (C.c_int, [vp, vp, vp, i64, i32]),
        "marfa_diag_absorption_counted_surrogate": (C.c_int, [vp, vp, vp, i32, vp, vp, vp, vp]),
        "marfa_plan_create": (C.c_int, [i32, vp, vp, vp, vp, vp, vp, i32, vp, C.POINTER(vp)]),
        "marfa_plan_execute": (C.c_int, [vp, vp]),
        "marfa_plan_info": (C.c_int, [vp, vp, vp, vp]),
        "marfa_diag_variants": (C.c_int, [vp, vp]),
        "marfa_plan_classes": (C.c_int, [vp, vp, vp, vp]),
        "marfa_shape_user_set": (C.c_int, [vp, C.c_int32, C.c_double]),
        "marfa_diag_fail_alloc": (C.c_int, [C.c_int64, vp]),
        "marfa_diag_device_memory": (C.c_int, [vp, vp]),
        "marfa_diag_check": (C.c_int, [C.c_int32, vp]),
        "marfa_plan_destroy": (None, [vp]),
        "marfa_diag_absorption_counts": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(rc):
    if rc != 0:
        raise MarfaError(rc, load().marfa_last_error().decode())


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return C.c_void_p(s.cuda_stream)
    return C.c_void_p(int(s))


class Lines:
    """A prepared line list (owns the library handle)."""

    def __init__(self, handle, n, n_species):
        self.handle = handle
        self.n = n
        self.n_species = n_species

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.marfa_free_lines(self.handle)
            self.handle = None


def marfa_prepare_lines(lines: np.ndarray, species: np.ndarray) -> Lines:
    lines = np.ascontiguousarray(lines, dtype=LINE_DTYPE)
    species = np.ascontiguousarray(species, dtype=SPECIES_DTYPE)
    h = C.c_void_p()
    _check(load().marfa_prepare_lines(_ptr(lines), len(lines), _ptr(species), len(species), C.byref(h)))
    return Lines(h, len(lines), len(species))


def marfa_prepare_lines_batch(line_lists, species_lists) -> list:
    """Several line lists at once (marfa_prepare_lines_batch): one Lines per request."""
    ls = [np.ascontiguousarray(x, dtype=LINE_DTYPE) for x in line_lists]
    ss = [np.ascontiguousarray(x, dtype=SPECIES_DTYPE) for x in species_lists]
    q = len(ls)
    assert q == len(ss) and q >= 1
    lp = (C.c_void_p * q)(*[x.ctypes.data for x in ls])
    sp = (C.c_void_p * q)(*[x.ctypes.data for x in ss])
    n = np.array([len(x) for x in ls], dtype=np.int64)
    ns = np.array([len(x) for x in ss], dtype=np.int32)
    out = (C.c_void_p * q)()
    _check(load().marfa_prepare_lines_batch(q, lp, _ptr(n), sp, _ptr(ns), out))
    return [Lines(C.c_void_p(out[i]), len(ls[i]), len(ss[i])) for i in range(q)]


def marfa_free_lines(lines: Lines) -> None:
    if lines.handle:
        load().marfa_free_lines(lines.handle)
        lines.handle = None


def marfa_num_points(nu_lo: float, nu_hi: float) -> int:
    return int(load().marfa_num_points(float(nu_lo), float(nu_hi)))


def make_request(nu_lo, nu_hi, cutoff, shape="voigt", chi="none", units="k_cm1", surrogate=0,
                 R_w=8, R_c=8, stencil=3) -> marfa_request_t:
    return marfa_request_t(float(nu_lo), float(nu_hi), float(cutoff), SHAPES[shape], CHI[chi],
                           UNITS[units], int(surrogate), int(R_w), int(R_c), int(stencil))


def make_levels(T, p) -> np.ndarray:
    lv = np.zeros(len(T), dtype=LEVEL_DTYPE)
    lv["T_K"] = T
    lv["p_atm"] = p
    return lv


def marfa_absorption(lines: Lines, levels: np.ndarray, vmr: np.ndarray, rq: marfa_request_t,
                     k_out, stream=None) -> None:
    """k_out: float32 [n_levels, npts], a numpy array (host) or a CUDA torch tensor."""
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    _check(load().marfa_absorption(lines.handle, _ptr(levels), _ptr(vmr), len(levels), C.byref(rq),
                                   _ptr(k_out), _stream(stream)))


def marfa_absorption_noalloc(lines: Lines, levels: np.ndarray, vmr: np.ndarray, rq: marfa_request_t,
                             k_out, stream=None) -> None:
    """marfa_absorption without device allocation (scratch in the library's own
    32 MiB device array); k_out must be a CUDA tensor [n_levels, npts] float32."""
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    _check(load().marfa_absorption_noalloc(lines.handle, _ptr(levels), _ptr(vmr), len(levels), C.byref(rq),
                                           _ptr(k_out), _stream(stream)))


def marfa_absorption_batch(lines, levels, vmrs, rqs, k_outs, stream=None) -> None:
    n = len(lines)
    levels = [np.ascontiguousarray(x, dtype=LEVEL_DTYPE) for x in levels]
    vmrs = [np.ascontiguousarray(v, dtype=np.float64) for v in vmrs]
    VP = C.c_void_p * n
    lh = VP(*[l.handle.value for l in lines])
    lp = VP(*[x.ctypes.data for x in levels])
    vp = VP(*[v.ctypes.data for v in vmrs])
    nl = (C.c_int32 * n)(*[len(x) for x in levels])
    rq = (marfa_request_t * n)(*rqs)
    outs = VP(*[_ptr(o).value for o in k_outs])
    _check(load().marfa_absorption_batch(n, lh, lp, vp, nl, rq, outs, _stream(stream)))


class Plan:
    """A captured batch (marfa_plan_create); keeps its line lists and outputs alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.marfa_plan_destroy(self.handle)
            self.handle = None


PLAN_AUTOTUNE, PLAN_SERIAL = 1, 2


def marfa_plan_create(lines, levels, vmrs, rqs, k_outs, autotune: bool = False, serial: bool = False,
                      stream=None) -> Plan:
    """k_outs: CUDA tensors [n_levels, npts] float32, rewritten by every execution."""
    n = len(lines)
    levels = [np.ascontiguousarray(x, dtype=LEVEL_DTYPE) for x in levels]
    vmrs = [np.ascontiguousarray(v, dtype=np.float64) for v in vmrs]
    VP = C.c_void_p * n
    lh = VP(*[l.handle.value for l in lines])
    lp = VP(*[x.ctypes.data for x in levels])
    vp = VP(*[v.ctypes.data for v in vmrs])
    nl = (C.c_int32 * n)(*[len(x) for x in levels])
    rq = (marfa_request_t * n)(*rqs)
    outs = VP(*[_ptr(o).value for o in k_outs])
    h = C.c_void_p()
    flags = (PLAN_AUTOTUNE if autotune else 0) | (PLAN_SERIAL if serial else 0)
    _check(load().marfa_plan_create(n, lh, lp, vp, nl, rq, outs, flags, _stream(stream), C.byref(h)))
    return Plan(h, (list(lines), list(k_outs)))


def marfa_plan_execute(plan: Plan, stream=None) -> None:
    _check(load().marfa_plan_execute(plan.handle, _stream(stream)))


PLAN_KINDS, PLAN_VARIANTS = 11, 6


def marfa_plan_info(plan: Plan, kernel_ms: bool = False):
    """(variant[11] for grids 1..10 and the finest grid, tune_ms[11, 6], kernel_ms[12] or None)."""
    v = np.empty(PLAN_KINDS, dtype=np.int32)
    t = np.empty((PLAN_KINDS, PLAN_VARIANTS), dtype=np.float32)
    k = np.empty(12, dtype=np.float64) if kernel_ms else None
    _check(load().marfa_plan_info(plan.handle, _ptr(v), _ptr(t), _ptr(k)))
    return v, t, k


def marfa_shape_user_set(g, x_max: float) -> None:
    """The user-defined line shape of the current device: g(x) sampled at
    x = k x_max / (n - 1) (linear between samples, g(x_max) (x_max/x)^2 beyond), on the
    Lorentz scaling x = (nu - nu~0) / gamma_L, f = S / (pi gamma_L) g(x)."""
    g = np.ascontiguousarray(g, dtype=np.float32)
    _check(load().marfa_shape_user_set(_ptr(g), len(g), float(x_max)))


PLAN_CLASSES = 2


def marfa_plan_classes(plan: Plan, n_req: int):
    """(req_class[n_req], choice[2, 11] (column 0: the grid-1 split), tune_ms[2, 11, 6])."""
    rc = np.empty(n_req, dtype=np.int32)
    ch = np.empty((PLAN_CLASSES, PLAN_KINDS), dtype=np.int32)
    t = np.empty((PLAN_CLASSES, PLAN_KINDS, PLAN_VARIANTS), dtype=np.float32)
    _check(load().marfa_plan_classes(plan.handle, _ptr(rc), _ptr(ch), _ptr(t)))
    return rc, ch, t


def marfa_diag_fail_alloc(nth: int) -> int:
    """Make the nth allocation from now on fail (0 disarms); returns what the previous
    arming still had to let through plus one (0: it was not armed)."""
    left = C.c_int64(0)
    _check(load().marfa_diag_fail_alloc(int(nth), C.byref(left)))
    return left.value


def marfa_diag_check(index: int) -> bool:
    """Run the device-check probe at index; returns whether the library is a MARFA_DEBUG
    build (raises MarfaError MARFA_E_INTERNAL when the probe's check fails there)."""
    dbg = C.c_int32(0)
    _check(load().marfa_diag_check(int(index), C.byref(dbg)))
    return bool(dbg.value)


def marfa_diag_device_memory():
    """(bytes in use from the device's default memory pool, free device memory)."""
    used, free = C.c_int64(0), C.c_int64(0)
    _check(load().marfa_diag_device_memory(C.byref(used), C.byref(free)))
    return used.value, free.value


def marfa_diag_variants(variants=None) -> np.ndarray:
    """Set (when given, 11 entries: grids 1..10 and the finest grid; entry 0 ignored) and
    return the kernel variants of calls without autotuning."""
    get = np.empty(PLAN_KINDS, dtype=np.int32)
    if variants is None:
        _check(load().marfa_diag_variants(None, _ptr(get)))
    else:
        sv = np.ascontiguousarray(variants, dtype=np.int32)
        assert sv.shape == (PLAN_KINDS,)
        _check(load().marfa_diag_variants(_ptr(sv), _ptr(get)))
    return get


def marfa_plan_destroy(plan: Plan) -> None:
    if plan.handle:
        load().marfa_plan_destroy(plan.handle)
        plan.handle = None


def marfa_read_par(text: bytes) -> np.ndarray:
    """Appendix B records (LINE_DTYPE) from the text of a HITRAN .par file."""
    lib = load()
    n = C.c_int64(0)
    _check(lib.marfa_read_par(text, len(text), None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=LINE_DTYPE)
    if n.value:
        _check(lib.marfa_read_par(text, len(text), _ptr(out), n.value, C.byref(n)))
    return out


def marfa_write_pt_table(directory: str, level_number: int, nu_lo: float, nu_hi: float, k: np.ndarray) -> None:
    k = np.ascontiguousarray(k, dtype=np.float32)
    _check(load().marfa_write_pt_table(directory.encode(), int(level_number), float(nu_lo), float(nu_hi),
                                       _ptr(k), len(k)))


def marfa_last_error() -> str:
    return load().marfa_last_error().decode()


def marfa_diag_voigt(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    out = np.empty_like(x)
    _check(load().marfa_diag_voigt(_ptr(x), _ptr(y), _ptr(out), len(x)))
    return out


def marfa_diag_level_lines(lines: Lines, levels, vmr, rq):
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    nl = len(levels)
    c = np.empty((nl, lines.n), dtype=np.int64)
    g = np.empty((nl, lines.n), dtype=np.int8)
    perm = np.empty(lines.n, dtype=np.int64)
    _check(load().marfa_diag_level_lines(lines.handle, _ptr(levels), _ptr(vmr), nl, C.byref(rq),
                                         _ptr(c), _ptr(g), _ptr(perm)))
    return c, g, perm


def marfa_diag_owned(lines: Lines, levels, vmr, rq, level: int, grid: int, first: int, count: int):
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    out = np.empty((lines.n, count), dtype=np.uint8)
    _check(load().marfa_diag_owned(lines.handle, _ptr(levels), _ptr(vmr), len(levels), C.byref(rq),
                                   int(level), int(grid), int(first), int(count), _ptr(out)))
    return out


def marfa_diag_absorption_counted(lines: Lines, levels, vmr, rq):
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    n = marfa_num_points(rq.nu_lo, rq.nu_hi)
    k = np.empty((len(levels), n), dtype=np.float32)
    counts = np.empty((len(levels), 11), dtype=np.int64)
    _check(load().marfa_diag_absorption_counted(lines.handle, _ptr(levels), _ptr(vmr), len(levels),
                                                C.byref(rq), _ptr(k), _ptr(counts)))
    return k, counts


def marfa_diag_absorption_counts(lines: Lines, levels, vmr, rq):
    """(k, counts[n_levels, 11, 5]): all, surrogate, 9x9 polynomial-cell, asymptotic and
    small-y-cell evaluations per level and grid."""
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    n = marfa_num_points(rq.nu_lo, rq.nu_hi)
    k = np.empty((len(levels), n), dtype=np.float32)
    counts = np.empty((len(levels), 11, 5), dtype=np.int64)
    _check(load().marfa_diag_absorption_counts(lines.handle, _ptr(levels), _ptr(vmr), len(levels),
                                               C.byref(rq), _ptr(k), _ptr(counts)))
    return k, counts


def marfa_diag_absorption_counted_surrogate(lines: Lines, levels, vmr, rq):
    """(k, counts, surrogate_counts), counts [n_levels, 11] per grid."""
    levels = np.ascontiguousarray(levels, dtype=LEVEL_DTYPE)
    vmr = np.ascontiguousarray(vmr, dtype=np.float64)
    n = marfa_num_points(rq.nu_lo, rq.nu_hi)
    k = np.empty((len(levels), n), dtype=np.float32)
    counts = np.empty((len(levels), 11), dtype=np.int64)
    sc = np.empty((len(levels), 11), dtype=np.int64)
    _check(load().marfa_diag_absorption_counted_surrogate(lines.handle, _ptr(levels), _ptr(vmr), len(levels),
                                                          C.byref(rq), _ptr(k), _ptr(counts), _ptr(sc)))
    return k, counts, sc


# ------------------------------------------------------------------ learned Voigt surrogate
def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def marfa_mlp_loss_grad(params, x, y, t, qat: bool = False):
    """(loss, grad[MLP_PARAMS]) of the mean squared error of t over the samples."""
    params, x, y, t = _f32(params), _f32(x), _f32(y), _f32(t)
    assert params.shape == (MLP_PARAMS,)
    grad = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = C.c_double()
    _check(load().marfa_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(y), _ptr(t), len(x), int(qat),
                                      C.byref(loss), _ptr(grad)))
    return loss.value, grad


def marfa_mlp_train(params, x, y, t, steps: int, batch: int, lr0: float, lr1: float, qat: bool = True):
    """Train a copy of params; returns (params, loss_curve[steps])."""
    p = _f32(params).copy()
    assert p.shape == (MLP_PARAMS,)
    x, y, t = _f32(x), _f32(y), _f32(t)
    cfg = marfa_mlp_train_t(int(steps), int(batch), int(qat), 0, float(lr0), float(lr1))
    curve = np.empty(int(steps), dtype=np.float32)
    _check(load().marfa_mlp_train(_ptr(p), _ptr(x), _ptr(y), _ptr(t), len(x), C.byref(cfg), _ptr(curve)))
    return p, curve


def marfa_surrogate_load(params, budget: float = 8e-4, samples: int = 16):
    """Load params as the surrogate of the current device; returns (cells_on,
    cell_err[GUARD_NY, GUARD_NX])."""
    params = _f32(params)
    assert params.shape == (MLP_PARAMS,)
    on = C.c_int32()
    err = np.empty((GUARD_NY, GUARD_NX), dtype=np.float32)
    _check(load().marfa_surrogate_load(_ptr(params), float(budget), int(samples), C.byref(on), _ptr(err)))
    return on.value, err


def marfa_surrogate_unload() -> None:
    _check(load().marfa_surrogate_unload())


def marfa_surrogate_eval(x, y, guarded: bool = False) -> np.ndarray:
    x, y = _f32(x), _f32(y)
    out = np.empty_like(x)
    _check(load().marfa_surrogate_eval(_ptr(x), _ptr(y), _ptr(out), len(x), int(guarded)))
    return out


def marfa_diag_kernel_timing(enable: bool):
    """Start (True) or stop (False) per-kernel event timing; stopping returns
    (ms[12], launches[12]): level preparation, grids 1..10, finest grid."""
    ms = np.zeros(12, dtype=np.float64)
    n = np.zeros(12, dtype=np.int64)
    _check(load().marfa_diag_kernel_timing(1 if enable else 0, _ptr(ms), _ptr(n)))
    return ms, n


PIPES = {"fma": 0, "ex2": 1, "rcp": 2, "cos": 3}


def marfa_diag_shape(shape: str, x, y) -> np.ndarray:
    """The kernels' line shape (K(x, y) for the Voigt shapes) at float32 points x, y."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    out = np.empty_like(x)
    _check(load().marfa_diag_shape(SHAPES[shape], _ptr(x), _ptr(y), _ptr(out), len(x)))
    return out


def marfa_diag_line_order(lines: np.ndarray) -> np.ndarray:
    """The prepared order of a line list (input index of each sorted line), host only."""
    lines = np.ascontiguousarray(lines, dtype=LINE_DTYPE)
    order = np.empty(len(lines), dtype=np.int64)
    _check(load().marfa_diag_line_order(_ptr(lines), len(lines), _ptr(order)))
    return order


def marfa_diag_pipe_rate(pipe: str) -> float:
    """Measured issue rate (instructions/s) of FP32 FMA or a MUFU kind on this device."""
    r = C.c_double(0.0)
    _check(load().marfa_diag_pipe_rate(PIPES[pipe], C.byref(r)))
    return r.value


# ------------------------------------------------------------------ workload marshalling
def request_of(wl) -> marfa_request_t:
    return make_request(wl.nu_lo, wl.nu_hi, wl.cutoff, wl.shape, wl.chi, wl.units, wl.surrogate,
                        wl.R_w, wl.R_c, getattr(wl, "stencil", 3))


def levels_of(wl) -> np.ndarray:
    return make_levels(wl.T, wl.p)
