"""CPU oracle for Chamfer-Estimate -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the paper's method (Fig. 1 Chamfer-Estimate,
Fig. 2 CrudeNN, the hash families of Appendix A.2) in C (``oracle.c``), plus the
plain definition CH(A, B) = sum_a min_b d(a, b) in binary64 (Section 1).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never calls it.

Parity status of each function (what pins it; see ``tests/test_oracle.py``):
  philox            Random123 known-answer vectors (tests/golden/philox_kat.txt)
  mix64             published splitmix64 sequence (tests/golden/splitmix64.txt)
  dist              binary64 brute force within the rounding bound; hand cases
  dist_fp64         hand cases; closed forms
  shift/cell/key    hand-worked grid cells; collision rate vs the closed form
                    prod_k max(0, 1-|x_k-y_k|/r) (Lemma on l1 hashing, App. A.2)
  proj_matrix       moments of the Irwin-Hall normal; E|<g,x>| = beta ||x||_2
  crude_nn          bit-exact vs the O(|A||B|L) brute-force restatement;
                    D_a >= min_b d(a, b) (Lemma 2); |B| = 1 special case
  weights/draws     exact integer checks; chi-square vs w_a / W; special cases
  scan/combine      |B| = 1 gives eta = CH exactly; unbiasedness and the
                    variance bound of Lemma 1 over many seeds; hand examples
  exact_fp64        hand-worked examples (Section 1 definition)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

L1 = 1
L2 = 2
INT32_MIN = -(2**31)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


class Report(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("D_total", ctypes.c_double),
                ("W", ctypes.c_uint64), ("T", ctypes.c_int64),
                ("top_exp", ctypes.c_int32), ("shift_S", ctypes.c_int32)]


_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int


def _bind(so):
    sig = {
        "or_philox4x32_10": (None, [_p, _p, _p]),
        "or_mix64": (_u64, [_u64]),
        "or_dist": (ctypes.c_float, [_p, _p, _i32, _i32]),
        "or_dist_fp64": (ctypes.c_double, [_p, _p, _i32, _i32]),
        "or_proj_matrix": (None, [_u64, _i32, _i32, _p]),
        "or_project": (None, [_p, _i64, _i32, _p, _i32, _p]),
        "or_shift": (ctypes.c_float, [_u64, _i32, _i32]),
        "or_coord_mult": (_u64, [_u64, _i32]),
        "or_cell": (ctypes.c_float, [ctypes.c_float, ctypes.c_float, _i32]),
        "or_key": (_u64, [_p, _i32, _i32, _u64]),
        "or_keys": (None, [_p, _i64, _i32, _i32, _i32, _u64, _p]),
        "or_top_exp": (_i32, [_p, _i64, _p, _i64, _i32]),
        "or_crude_nn": (_i32, [_p, _i64, _p, _i64, _i32, _i32, _u64, _i32, _i32, _i32, _i32,
                               _p, _p, _p, _p, _p]),
        "or_weights": (_i32, [_p, _i64, _p, _p, _p]),
        "or_draws": (None, [_p, _i64, _u64, _i64, _u64, _p]),
        "or_scan": (None, [_p, _p, _i64, _p, _i64, _i32, _i32, _p, _p]),
        "or_combine": (ctypes.c_double, [_p, _p, _p, _u64, _i64]),
        "or_default_T": (_i64, [_i64, _i64, ctypes.c_double]),
        "or_estimate": (ctypes.c_double, [_p, _i64, _p, _i64, _i32, _i32, _u64, _i32, _i32, _i32,
                                          _i64, _u64, _p, _p, _p, _p, _p, _p]),
        "or_draws_uniform": (None, [_i64, _i64, _u64, _p]),
        "or_keys_simhash": (None, [_p, _i64, _i32, _i32, _u64, _p]),
        "or_crude_nn_simhash": (None, [_p, _i64, _p, _i64, _i32, _i32, _u64, _i32, _i32, _p, _p, _p]),
        "or_crude_nn_kw": (None, [_p, _i64, _p, _i64, _i32, _i32, _u64, _i32, _i32, _i32, _i32, _i32, _p, _p, _p]),
        "or_estimate_uniform": (ctypes.c_double, [_p, _i64, _p, _i64, _i32, _i32, _i64, _u64, _p, _p]),
        "or_exact_fp64": (ctypes.c_double, [_p, _i64, _p, _i64, _i32, _i32, _p]),
        "or_exact_canonical": (ctypes.c_double, [_p, _i64, _p, _i64, _i32, _i32, _p]),
        "or_num_threads": (_i32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


def _f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x.reshape(-1, 1) if x.size else x.reshape(0, 1)
    return x


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def mix64(x: int) -> int:
    return int(lib().or_mix64(x & (2**64 - 1)))


def dist(a, b, metric: int) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    return float(lib().or_dist(_ptr(a), _ptr(b), a.size, metric))


def dist_fp64(a, b, metric: int) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    return float(lib().or_dist_fp64(_ptr(a), _ptr(b), a.size, metric))


def proj_matrix(seed: int, k: int, d: int) -> np.ndarray:
    G = np.zeros((k, d), dtype=np.float32)
    lib().or_proj_matrix(seed, k, d, _ptr(G))
    return G


def project(X, G) -> np.ndarray:
    X = _f32(X)
    G = np.ascontiguousarray(G, dtype=np.float32)
    Y = np.zeros((X.shape[0], G.shape[0]), dtype=np.float32)
    lib().or_project(_ptr(X), X.shape[0], X.shape[1], _ptr(G), G.shape[0], _ptr(Y))
    return Y


def shift(seed: int, e: int, j: int) -> float:
    return float(lib().or_shift(seed, e, j))


def coord_mult(seed: int, j: int) -> int:
    return int(lib().or_coord_mult(seed, j))


def cell(y: float, z: float, e: int) -> float:
    return float(lib().or_cell(y, z, e))


def key(y, e: int, seed: int) -> int:
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    return int(lib().or_key(_ptr(y), y.size, e, seed))


def keys(Y, e_lo: int, L: int, seed: int) -> np.ndarray:
    Y = _f32(Y)
    out = np.zeros((L, Y.shape[0]), dtype=np.uint64)
    lib().or_keys(_ptr(Y), Y.shape[0], Y.shape[1], e_lo, L, seed, _ptr(out))
    return out


def top_exp(YA, YB) -> int:
    YA, YB = _f32(YA), _f32(YB)
    return int(lib().or_top_exp(_ptr(YA), YA.shape[0], _ptr(YB), YB.shape[0], YA.shape[1]))


def hashed(X, metric: int, seed: int, proj_dim: int = 16) -> np.ndarray:
    """y-space of a set: x for l1, the Gaussian projection T(x) for l2."""
    X = _f32(X)
    if metric == L1:
        return X.copy()
    return project(X, proj_matrix(seed, proj_dim, X.shape[1]))


# ---------------------------------------------------------------- the method
def crude_nn(A, B, metric: int, hash_seed: int, L: int = 10, proj_dim: int = 16,
             top_exp: int | None = None, brute: bool = False, want_keys: bool = False):
    """CrudeNN (Fig. 2).  Returns dict(bidx, D, level, top_exp[, keysA, keysB])."""
    A, B = _f32(A), _f32(B)
    nA, d = A.shape
    nB = B.shape[0]
    bidx = np.zeros(nA, dtype=np.int64)
    D = np.zeros(nA, dtype=np.float32)
    level = np.zeros(nA, dtype=np.uint8)
    kA = np.zeros((L, nA), dtype=np.uint64) if want_keys else None
    kB = np.zeros((L, nB), dtype=np.uint64) if want_keys else None
    e = lib().or_crude_nn(_ptr(A), nA, _ptr(B), nB, d, metric, hash_seed, L, proj_dim,
                          INT32_MIN if top_exp is None else int(top_exp), int(brute),
                          _ptr(bidx), _ptr(D), _ptr(level), _ptr(kA), _ptr(kB))
    out = dict(bidx=bidx, D=D, level=level, top_exp=int(e))
    if want_keys:
        out.update(keysA=kA, keysB=kB)
    return out


def weights(D):
    D = np.ascontiguousarray(D, dtype=np.float32)
    n = D.size
    w = np.zeros(n, dtype=np.uint64)
    prefix = np.zeros(n, dtype=np.uint64)
    W = np.zeros(1, dtype=np.uint64)
    S = lib().or_weights(_ptr(D), n, _ptr(w), _ptr(prefix), _ptr(W))
    return w, prefix, int(W[0]), int(S)


def draws(prefix, W: int, T: int, seed: int) -> np.ndarray:
    prefix = np.ascontiguousarray(prefix, dtype=np.uint64)
    idx = np.zeros(max(T, 0), dtype=np.int64)
    lib().or_draws(_ptr(prefix), prefix.size, W, T, seed, _ptr(idx))
    return idx


def scan(A, idx, B, metric: int):
    A, B = _f32(A), _f32(B)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    T = idx.size
    m = np.zeros(T, dtype=np.float32)
    am = np.zeros(T, dtype=np.int64)
    lib().or_scan(_ptr(A), _ptr(idx), T, _ptr(B), B.shape[0], A.shape[1], metric, _ptr(m), _ptr(am))
    return m, am


def combine(m, idx, w, W: int) -> float:
    m = np.ascontiguousarray(m, dtype=np.float32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.uint64)
    return float(lib().or_combine(_ptr(m), _ptr(idx), _ptr(w), W, m.size))


def default_T(nA: int, nB: int, eps: float) -> int:
    return int(lib().or_default_T(nA, nB, eps))


def estimate(A, B, metric: int, hash_seed: int, sample_seed: int, T: int, L: int = 10,
             proj_dim: int = 16, top_exp: int | None = None, details: bool = False):
    """Chamfer-Estimate(A, B, T) (Fig. 1).  Returns eta, or (eta, dict) with details."""
    A, B = _f32(A), _f32(B)
    nA, d = A.shape
    rep = Report()
    bidx = np.zeros(nA, dtype=np.int64)
    D = np.zeros(nA, dtype=np.float32)
    level = np.zeros(nA, dtype=np.uint8)
    idx = np.zeros(max(T, 1), dtype=np.int64)
    m = np.zeros(max(T, 1), dtype=np.float32)
    eta = lib().or_estimate(_ptr(A), nA, _ptr(B), B.shape[0], d, metric, hash_seed, L, proj_dim,
                            INT32_MIN if top_exp is None else int(top_exp), T, sample_seed,
                            _ptr(bidx), _ptr(D), _ptr(level), _ptr(idx), _ptr(m),
                            ctypes.byref(rep))
    if not details:
        return float(eta)
    return float(eta), dict(bidx=bidx, D=D, level=level, idx=idx[:T], m=m[:T], W=int(rep.W),
                            D_total=rep.D_total, top_exp=rep.top_exp, S=rep.shift_S)


def crude_nn_kw(A, B, metric: int, hash_seed: int = 0, L: int = 10, proj_dim: int = 16,
                top_exp: int | None = None, k: int = 1, W: int = 1) -> dict:
    """k x W CrudeNN (Section 3): k structures, the first W distinct points of B
    from a's buckets in increasing scale order, D_a the closest of them."""
    A, B = _f32(A), _f32(B)
    nA = A.shape[0]
    bidx = np.zeros(nA, dtype=np.int64)
    D = np.zeros(nA, dtype=np.float32)
    level = np.zeros(nA, dtype=np.uint8)
    lib().or_crude_nn_kw(_ptr(A), nA, _ptr(B), B.shape[0], A.shape[1], metric, hash_seed, L, proj_dim,
                         INT32_MIN if top_exp is None else int(top_exp), k, W, _ptr(bidx), _ptr(D), _ptr(level))
    return {"bidx": bidx, "D": D, "level": level}


def keys_simhash(Y, L: int, seed: int) -> np.ndarray:
    """SimHash keys [L][n] of embedded points Y [n][K] (first K >> l sign bits at level l)."""
    Y = _f32(Y)
    out = np.zeros((L, Y.shape[0]), dtype=np.uint64)
    lib().or_keys_simhash(_ptr(Y), Y.shape[0], Y.shape[1], L, seed, _ptr(out))
    return out


def crude_nn_simhash(A, B, metric: int, hash_seed: int = 0, L: int = 10, K: int = 16) -> dict:
    """CrudeNN (Fig. 2) with SimHash buckets on the K-wide Gaussian embedding."""
    A, B = _f32(A), _f32(B)
    nA = A.shape[0]
    bidx = np.zeros(nA, dtype=np.int64)
    D = np.zeros(nA, dtype=np.float32)
    level = np.zeros(nA, dtype=np.uint8)
    lib().or_crude_nn_simhash(_ptr(A), nA, _ptr(B), B.shape[0], A.shape[1], metric, hash_seed, L, K,
                              _ptr(bidx), _ptr(D), _ptr(level))
    return {"bidx": bidx, "D": D, "level": level}


def draws_uniform(nA: int, T: int, seed: int) -> np.ndarray:
    """Uniform draws over A from the Philox counters of the importance draws."""
    idx = np.zeros(max(T, 0), dtype=np.int64)
    lib().or_draws_uniform(nA, T, seed, _ptr(idx))
    return idx


def estimate_uniform(A, B, metric: int, sample_seed: int, T: int, details: bool = False):
    """The uniform-sampling baseline: (nA / T) sum_l min_b d(x_l, b), x_l uniform over A."""
    A, B = _f32(A), _f32(B)
    idx = np.zeros(max(T, 1), dtype=np.int64)
    m = np.zeros(max(T, 1), dtype=np.float32)
    eta = float(lib().or_estimate_uniform(_ptr(A), A.shape[0], _ptr(B), B.shape[0], A.shape[1], metric, T,
                                          sample_seed, _ptr(idx), _ptr(m)))
    return (eta, dict(idx=idx[:T], m=m[:T])) if details else eta


# sample seed of the (B, A) direction of a symmetric estimate
SYM_SEED_XOR = 0x9E3779B97F4A7C15


def estimate_sym(A, B, metric: int, hash_seed: int, sample_seed: int, T: int, L: int = 10, proj_dim: int = 16,
                 top_exp: int | None = None, uniform: bool = False):
    """CH(A, B) + CH(B, A) estimated as two one-sided estimates (Section 1's symmetric
    form): the same hash seed, the (B, A) draws keyed by sample_seed ^ SYM_SEED_XOR.
    Returns (eta_AB + eta_BA, eta_AB, eta_BA)."""
    s2 = sample_seed ^ SYM_SEED_XOR
    if uniform:
        ab = estimate_uniform(A, B, metric, sample_seed, T)
        ba = estimate_uniform(B, A, metric, s2, T)
    else:
        ab = estimate(A, B, metric, hash_seed, sample_seed, T, L, proj_dim, top_exp)
        ba = estimate(B, A, metric, hash_seed, s2, T, L, proj_dim, top_exp)
    return ab + ba, ab, ba


def exact_fp64(A, B, metric: int, per_a: bool = False):
    """CH(A, B) in binary64 (Section 1)."""
    A, B = _f32(A), _f32(B)
    pa = np.zeros(A.shape[0], dtype=np.float64) if per_a else None
    v = float(lib().or_exact_fp64(_ptr(A), A.shape[0], _ptr(B), B.shape[0], A.shape[1], metric, _ptr(pa)))
    return (v, pa) if per_a else v


def exact_canonical(A, B, metric: int):
    """sum_a min_b of the canonical binary32 distance, summed in binary64."""
    A, B = _f32(A), _f32(B)
    pa = np.zeros(A.shape[0], dtype=np.float32)
    v = float(lib().or_exact_canonical(_ptr(A), A.shape[0], _ptr(B), B.shape[0], A.shape[1], metric,
                                       _ptr(pa)))
    return v, pa


def num_threads() -> int:
    return int(lib().or_num_threads())
