"""Thin ctypes binding of libchamfer (include/chamfer.h).

Argument marshalling only: each function takes torch tensors (device memory and
streams come from PyTorch), numpy arrays (host memory) or plain numbers, passes
raw pointers to the C entry point of the same name, and raises ChamferError on
a non-zero status.  There is no CPU fallback: without the compiled library
every call fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchamfer.so")

CH_OK, CH_EINVAL, CH_ENOMEM, CH_ECUDA, CH_ENOTSUP, CH_ETIMEOUT, CH_EBUSY, CH_EAGAIN = range(8)
CH_SAMPLING_IMPORTANCE, CH_SAMPLING_UNIFORM = 0, 1
CH_FAMILY_GRID, CH_FAMILY_SIMHASH = 0, 1
CH_L1, CH_L2 = 1, 2
CH_F32, CH_BF16, CH_FP8E4M3 = 0, 1, 2
CH_SCREEN_AUTO, CH_SCREEN_EXACT, CH_SCREEN_TF32, CH_SCREEN_BF16, CH_SCREEN_FP8 = range(5)
CH_GROUP_HASH, CH_GROUP_SORT = 0, 1
CH_TOP_EXP_AUTO = -(2**31)
STATUS_NAMES = ["CH_OK", "CH_EINVAL", "CH_ENOMEM", "CH_ECUDA", "CH_ENOTSUP", "CH_ETIMEOUT", "CH_EBUSY",
                "CH_EAGAIN"]


class ChamferError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}" + (f" ({message})" if message else ""))


class ch_hash_params(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int32), ("levels", ctypes.c_uint32), ("proj_dim", ctypes.c_uint32),
                ("top_exp", ctypes.c_int32), ("hash_seed", ctypes.c_uint64), ("group", ctypes.c_int32),
                ("window", ctypes.c_uint32), ("repeats", ctypes.c_uint32), ("family", ctypes.c_int32)]


class ch_est_params(ctypes.Structure):
    _fields_ = [("hash", ch_hash_params), ("eps", ctypes.c_double), ("T", ctypes.c_int64),
                ("sample_seed", ctypes.c_uint64), ("screen", ctypes.c_int32), ("rerank_k", ctypes.c_uint32),
                ("sampling", ctypes.c_int32)]


class ch_est_report(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("D_total", ctypes.c_double), ("W", ctypes.c_uint64),
                ("T", ctypes.c_int64), ("top_exp", ctypes.c_int32), ("shift_S", ctypes.c_int32),
                ("t_crude_ms", ctypes.c_float), ("t_sample_ms", ctypes.c_float), ("t_scan_ms", ctypes.c_float),
                ("t_total_ms", ctypes.c_float), ("t_kernel_ms", ctypes.c_float), ("screen", ctypes.c_int32)]


class ch_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("max_queue", ctypes.c_int32)]


class ch_serve_stats(ctypes.Structure):
    _fields_ = [("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("throughput_rps", ctypes.c_double), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("pending", ctypes.c_int64), ("peak_bytes", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_P = ctypes.POINTER

# every symbol include/chamfer.h declares, with its ctypes signature
SIGNATURES = {
    "ch_default_params": (None, [_P(ch_est_params)]),
    "ch_ctx_create": (_i32, [ctypes.c_int, _vp, _P(_vp)]),
    "ch_ctx_destroy": (None, [_vp]),
    "ch_last_error": (ctypes.c_char_p, [_vp]),
    "ch_ctx_sync": (_i32, [_vp]),
    "ch_ctx_workspace_bytes": (_i64, [_vp]),
    "ch_ctx_set_wait_cycles": (_i32, [_vp, _i64]),
    "ch_kernel_launches": (_i64, []),
    "ch_set_create": (_i32, [_vp, _vp, ctypes.c_int, _i64, _i32, _i32, _vp, _P(_vp)]),
    "ch_set_destroy": (None, [_vp]),
    "ch_set_prepare": (_i32, [_vp, _vp]),
    "ch_set_size": (_i64, [_vp]),
    "ch_set_dim": (_i32, [_vp]),
    "ch_top_exp": (_i32, [_vp, _vp, _vp, _P(ch_hash_params), _P(_i32)]),
    "ch_hash_keys": (_i32, [_vp, _vp, _P(ch_hash_params), _i32, _vp]),
    "ch_crude_nn": (_i32, [_vp, _vp, _vp, _P(ch_hash_params), _vp, _vp, _vp]),
    "ch_sample": (_i32, [_vp, _vp, _i64, _i64, _u64, _vp, _vp, _P(_u64)]),
    "ch_sample_static": (_i32, [_vp, _i64, _i64, _u64, _vp, _vp, _vp, _vp]),
    "ch_sampled_nn": (_i32, [_vp, _vp, _vp, _i64, _vp, _i32, _i32, _u32, _vp, _vp]),
    "ch_estimate": (_i32, [_vp, _vp, _vp, _P(ch_est_params), _P(ctypes.c_double), _P(ch_est_report)]),
    "ch_estimate_batch": (_i32, [_vp, _i64, _P(_vp), _P(_vp), _P(ch_est_params), _P(ctypes.c_double), _P(_i32)]),
    "ch_estimate_sym": (_i32, [_vp, _vp, _vp, _P(ch_est_params), _P(ctypes.c_double), _P(ctypes.c_double),
                               _P(ctypes.c_double)]),
    "ch_exact": (_i32, [_vp, _vp, _vp, _i32, _i32, _P(ctypes.c_double), _vp]),
    "ch_serve_create": (_i32, [_vp, _P(ch_serve_config), _P(_vp)]),
    "ch_serve_index": (_i32, [_vp, _P(ch_hash_params)]),
    "ch_set_embed": (_i32, [_vp, _vp, _P(ch_hash_params)]),
    "ch_serve_register": (_i32, [_vp, _vp, ctypes.c_int, _i64, _i32, _i32, _vp, _P(_u64)]),
    "ch_serve_submit": (_i32, [_vp, _u64, _u64, _P(ch_est_params), _P(_u64)]),
    "ch_serve_poll": (_i32, [_vp, _u64, _P(ctypes.c_double), _P(_i32)]),
    "ch_serve_wait": (_i32, [_vp, _u64, _u32, _P(ctypes.c_double), _P(_i32)]),
    "ch_serve_stats_get": (_i32, [_vp, _P(ch_serve_stats)]),
    "ch_serve_stats_reset": (_i32, [_vp]),
    "ch_serve_destroy": (None, [_vp]),
}

_lib = None


def lib():
    """Load libchamfer.so (build it first with paper_2307_03043_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ChamferError(CH_ENOTSUP, "load", f"{LIB_PATH} is not built; run the package build first")
        so = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(so, name)
            fn.restype = res
            fn.argtypes = args
        _lib = so
    return _lib


def _ptr(x):
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(st, where, ctx=None):
    if st != CH_OK:
        msg = ""
        if ctx is not None:
            m = lib().ch_last_error(ctx)
            msg = m.decode() if m else ""
        raise ChamferError(st, where, msg)


def hash_params(metric=CH_L1, levels=10, proj_dim=16, top_exp=None, hash_seed=0, group=CH_GROUP_HASH, window=1,
                repeats=1, family=0):
    return ch_hash_params(metric, levels, proj_dim, CH_TOP_EXP_AUTO if top_exp is None else top_exp,
                          hash_seed, group, window, repeats, family)


def est_params(metric=CH_L1, levels=10, proj_dim=16, top_exp=None, hash_seed=0, group=CH_GROUP_HASH,
               eps=0.1, T=0, sample_seed=0, screen=CH_SCREEN_AUTO, rerank_k=8, sampling=None, window=1, repeats=1,
               family=0):
    p = ch_est_params()
    lib().ch_default_params(ctypes.byref(p))
    p.hash = hash_params(metric, levels, proj_dim, top_exp, hash_seed, group, window, repeats, family)
    p.eps, p.T, p.sample_seed, p.screen, p.rerank_k = eps, T, sample_seed, screen, rerank_k
    p.sampling = CH_SAMPLING_IMPORTANCE if sampling is None else sampling
    return p


# ----------------------------------------------------------------- context
def ch_ctx_create(device: int = 0, stream=None):
    """stream: a torch.cuda.Stream, an int cudaStream_t, or None (own stream).
    torch's default stream (handle 0) is passed as cudaStreamLegacy (0x1), so
    the library's work stays ordered with torch's."""
    h = _vp()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    if stream is not None and s == 0:
        s = 1  # cudaStreamLegacy
    _check(lib().ch_ctx_create(device, s, ctypes.byref(h)), "ch_ctx_create")
    return h


def ch_ctx_destroy(ctx):
    lib().ch_ctx_destroy(ctx)


def ch_last_error(ctx) -> str:
    m = lib().ch_last_error(ctx)
    return m.decode() if m else ""


def ch_ctx_sync(ctx):
    _check(lib().ch_ctx_sync(ctx), "ch_ctx_sync", ctx)


def ch_ctx_workspace_bytes(ctx) -> int:
    return int(lib().ch_ctx_workspace_bytes(ctx))


def ch_ctx_set_wait_cycles(ctx, cycles: int):
    _check(lib().ch_ctx_set_wait_cycles(ctx, cycles), "ch_ctx_set_wait_cycles", ctx)


def ch_kernel_launches() -> int:
    return int(lib().ch_kernel_launches())


# ----------------------------------------------------------------- sets
def ch_set_create(ctx, data, mode: int, n: int, d: int, dtype: int = CH_F32, row_scales=None):
    """mode 0: host data copied; 1: device data copied; 2: device data adopted."""
    h = _vp()
    _check(lib().ch_set_create(ctx, _ptr(data), mode, n, d, dtype, _ptr(row_scales), ctypes.byref(h)),
           "ch_set_create", ctx)
    return h


def ch_set_destroy(s):
    lib().ch_set_destroy(s)


def ch_set_prepare(ctx, s):
    _check(lib().ch_set_prepare(ctx, s), "ch_set_prepare", ctx)


def ch_set_size(s) -> int:
    return int(lib().ch_set_size(s))


def ch_set_dim(s) -> int:
    return int(lib().ch_set_dim(s))


# ----------------------------------------------------------------- method
def ch_top_exp(ctx, A, B, hp: ch_hash_params) -> int:
    e = _i32()
    _check(lib().ch_top_exp(ctx, A, B, ctypes.byref(hp), ctypes.byref(e)), "ch_top_exp", ctx)
    return int(e.value)


def ch_hash_keys(ctx, X, hp: ch_hash_params, e_lo: int, keys):
    _check(lib().ch_hash_keys(ctx, X, ctypes.byref(hp), e_lo, _ptr(keys)), "ch_hash_keys", ctx)


def ch_crude_nn(ctx, A, B, hp: ch_hash_params, b_idx, D, level=None):
    _check(lib().ch_crude_nn(ctx, A, B, ctypes.byref(hp), _ptr(b_idx), _ptr(D), _ptr(level)), "ch_crude_nn", ctx)


def ch_sample(ctx, D, nA: int, T: int, seed: int, idx, w=None, want_total: bool = False):
    W = _u64()
    _check(lib().ch_sample(ctx, _ptr(D), nA, T, seed, _ptr(idx), _ptr(w), ctypes.byref(W) if want_total else None),
           "ch_sample", ctx)
    return int(W.value) if want_total else None


def ch_sample_static(D, nA: int, T: int, seed: int, idx, w, W_total=None, stream=None):
    """ch_sample for callers that cannot allocate device memory (no context;
    fixed library-held scratch, nA <= 1,048,576).  W_total: device uint64 or None.
    stream: torch.cuda.Stream / int handle / None (legacy default stream)."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(lib().ch_sample_static(_ptr(D), nA, T, seed, _ptr(idx), _ptr(w), _ptr(W_total), s),
           "ch_sample_static")


def ch_sampled_nn(ctx, A, idx, T: int, B, metric: int, screen: int, rerank_k: int, min_d, argmin=None):
    _check(lib().ch_sampled_nn(ctx, A, _ptr(idx), T, B, metric, screen, rerank_k, _ptr(min_d), _ptr(argmin)),
           "ch_sampled_nn", ctx)


def ch_estimate(ctx, A, B, p: ch_est_params, report: bool = False):
    eta = ctypes.c_double()
    rep = ch_est_report()
    _check(lib().ch_estimate(ctx, A, B, ctypes.byref(p), ctypes.byref(eta), ctypes.byref(rep) if report else None),
           "ch_estimate", ctx)
    return (eta.value, rep) if report else eta.value


def ch_estimate_batch(ctx, A_sets, B_sets, params):
    """Estimates of the pairs (A_sets[i], B_sets[i]) under params[i] in one call.
    Returns (etas, statuses) as lists; never raises for a failing pair."""
    n = len(A_sets)
    assert len(B_sets) == n and len(params) == n
    a = (_vp * n)(*A_sets)
    b = (_vp * n)(*B_sets)
    p = (ch_est_params * n)(*params)
    eta = (ctypes.c_double * n)()
    st = (_i32 * n)()
    rc = lib().ch_estimate_batch(ctx, n, a, b, p, eta, st)
    if rc not in (CH_OK,) and all(x == CH_OK for x in st):
        _check(rc, "ch_estimate_batch", ctx)
    return list(eta), list(st)


def ch_estimate_sym(ctx, A, B, p: ch_est_params):
    """CH(A, B) + CH(B, A); returns (sum, eta_AB, eta_BA)."""
    e, ab, ba = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().ch_estimate_sym(ctx, A, B, ctypes.byref(p), ctypes.byref(e), ctypes.byref(ab), ctypes.byref(ba)),
           "ch_estimate_sym", ctx)
    return e.value, ab.value, ba.value


def ch_exact(ctx, A, B, metric: int, mode: int = 0, per_a_min=None) -> float:
    v = ctypes.c_double()
    _check(lib().ch_exact(ctx, A, B, metric, mode, ctypes.byref(v), _ptr(per_a_min)), "ch_exact", ctx)
    return v.value


# ----------------------------------------------------------------- serving
def ch_serve_create(ctx, hbm_budget_bytes: int, max_slots: int = 8, max_queue: int = 1024):
    h = _vp()
    cfg = ch_serve_config(hbm_budget_bytes, max_slots, max_queue)
    _check(lib().ch_serve_create(ctx, ctypes.byref(cfg), ctypes.byref(h)), "ch_serve_create", ctx)
    return h


def ch_serve_index(srv, hp: ch_hash_params):
    _check(lib().ch_serve_index(srv, ctypes.byref(hp)), "ch_serve_index")


def ch_set_embed(ctx, s, hp: ch_hash_params):
    _check(lib().ch_set_embed(ctx, s, ctypes.byref(hp)), "ch_set_embed", ctx)


def ch_serve_register(srv, data, mode: int, n: int, d: int, dtype: int = CH_F32, row_scales=None) -> int:
    sid = _u64()
    _check(lib().ch_serve_register(srv, _ptr(data), mode, n, d, dtype, _ptr(row_scales), ctypes.byref(sid)),
           "ch_serve_register")
    return int(sid.value)


def ch_serve_submit(srv, set_a: int, set_b: int, p: ch_est_params):
    """Returns (status, ticket); CH_EAGAIN / CH_EBUSY are returned, not raised."""
    t = _u64()
    st = lib().ch_serve_submit(srv, set_a, set_b, ctypes.byref(p), ctypes.byref(t))
    if st not in (CH_OK, CH_EAGAIN, CH_EBUSY):
        _check(st, "ch_serve_submit")
    return st, int(t.value)


def ch_serve_poll(srv, ticket: int):
    """Returns (status, eta, request_status)."""
    eta = ctypes.c_double()
    rs = _i32()
    st = lib().ch_serve_poll(srv, ticket, ctypes.byref(eta), ctypes.byref(rs))
    if st not in (CH_OK, CH_EAGAIN):
        _check(st, "ch_serve_poll")
    return st, eta.value, int(rs.value)


def ch_serve_wait(srv, ticket: int, timeout_ms: int = 60000):
    eta = ctypes.c_double()
    rs = _i32()
    st = lib().ch_serve_wait(srv, ticket, timeout_ms, ctypes.byref(eta), ctypes.byref(rs))
    if st not in (CH_OK, CH_ETIMEOUT):
        _check(st, "ch_serve_wait")
    return st, eta.value, int(rs.value)


def ch_serve_stats_reset(srv):
    _check(lib().ch_serve_stats_reset(srv), "ch_serve_stats_reset")


def ch_serve_stats_get(srv) -> ch_serve_stats:
    s = ch_serve_stats()
    _check(lib().ch_serve_stats_get(srv, ctypes.byref(s)), "ch_serve_stats_get")
    return s


def ch_serve_destroy(srv):
    lib().ch_serve_destroy(srv)
