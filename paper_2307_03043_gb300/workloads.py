"""Seeded synthetic point sets shaped like the paper's workloads.

This module only draws random inputs (numpy, fixed seeds); it contains none of
the method's arithmetic, so both the CUDA library's tests and the CPU oracle can
take their inputs from it.  The paper's own datasets (ShapeNet, the Federalist
word2vec clouds, DEEP1B, MS-Turing; Table 1) are not available here; each
generator below is a stand-in with the shapes and value structure of one of them.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n_a: int, n_b: int, d: int, seed: int):
    """Coordinates i.i.d. uniform[0, 1): the small plain-method case."""
    g = _rng(seed)
    A = g.random((n_a, d), dtype=np.float32)
    B = g.random((n_b, d), dtype=np.float32)
    return A, B


def gaussian_mixture(n_a: int, n_b: int, d: int, seed: int, clusters: int = 100,
                     centre_box: float = 10.0, point_std: float = 1.0,
                     centre_jitter: float = 0.5):
    """Mixture of isotropic Gaussians (the high-dimensional plain-method case).

    Centres uniform in [-centre_box, centre_box]^d, cluster labels uniform,
    points = centre + N(0, point_std^2 I).  B uses the same centres moved by
    N(0, centre_jitter^2 I) (the jitter read as a standard deviation).
    """
    g = _rng(seed)
    C = g.uniform(-centre_box, centre_box, size=(clusters, d))
    la = g.integers(0, clusters, size=n_a)
    A = (C[la] + point_std * g.standard_normal((n_a, d))).astype(np.float32)
    CB = C + centre_jitter * g.standard_normal((clusters, d))
    lb = g.integers(0, clusters, size=n_b)
    B = (CB[lb] + point_std * g.standard_normal((n_b, d))).astype(np.float32)
    return A, B


def _pool_map(fn, items):
    """Runs fn over items on a thread pool (numpy's random fills and ufuncs
    release the GIL); results in item order."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    items = list(items)
    if len(items) <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=min(len(items), os.cpu_count() or 1)) as ex:
        return list(ex.map(fn, items))


def unit_mixture(n_a: int, n_b: int, d: int, seed: int, clusters: int = 1000,
                 sigma: float = 0.3, chunk: int = 1 << 16):
    """Unit-norm mixture vectors (stand-in for DEEP1B / MS-Turing embeddings).

    1000 unit centres (normalised N(0, I)); point = normalise(centre +
    N(0, sigma^2 I / d)); A and B are independent draws of the same mixture.
    Rows are drawn in chunks of `chunk`, each from its own PCG64 stream spawned
    from `seed`, in binary32 and on all host threads, so a 1M x 384 set takes
    seconds; the values depend only on (seed, sizes, chunk), never on the thread
    count.
    """
    g = _rng(seed)
    C = g.standard_normal((clusters, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    C32 = C.astype(np.float32)
    s = np.float32(sigma / math.sqrt(d))
    streams = np.random.SeedSequence([seed, 0x756E6974]).spawn(2)

    def draw(n, ss):
        out = np.empty((n, d), dtype=np.float32)
        spans = [(lo, min(n, lo + chunk)) for lo in range(0, n, chunk)]
        kids = ss.spawn(len(spans))

        def fill(k):
            lo, hi = spans[k]
            gk = np.random.Generator(np.random.PCG64(kids[k]))
            lab = gk.integers(0, clusters, size=hi - lo)
            x = out[lo:hi]
            gk.standard_normal(size=(hi - lo, d), dtype=np.float32, out=x)
            x *= s
            x += C32[lab]
            x /= np.sqrt(np.einsum("ij,ij->i", x, x))[:, None]

        _pool_map(fill, range(len(spans)))
        return out

    return draw(n_a, streams[0]), draw(n_b, streams[1])


def shape_surface(n_a: int, n_b: int, seed: int, noise: float = 0.01):
    """d = 3 surface samples of a random ellipsoid or box (ShapeNet stand-in).

    A random-axis shape is sampled n_a times for A; B is an independent
    resample of the same surface; both get Gaussian noise of `noise` times the
    shape's extent.
    """
    g = _rng(seed)
    axes = g.uniform(0.2, 1.0, size=3)
    Q, _ = np.linalg.qr(g.standard_normal((3, 3)))
    box = bool(g.integers(0, 2))

    def draw(n):
        if box:
            face = g.integers(0, 6, size=n)
            u = g.uniform(-1.0, 1.0, size=(n, 3))
            ax = face // 2
            u[np.arange(n), ax] = np.where(face % 2 == 0, -1.0, 1.0)
            p = u * axes
        else:
            v = g.standard_normal((n, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            p = v * axes
        p = p @ Q.T
        p += noise * axes.max() * g.standard_normal((n, 3))
        return p.astype(np.float32)

    return draw(n_a), draw(n_b)


def outlier_gaussian(n: int, d: int, seed: int):
    """Two standard Gaussian clouds in R^d plus one outlier 0.5 n * (1,...,1) in A
    (the robustness experiment of Section 3)."""
    g = _rng(seed)
    A = g.standard_normal((n, d)).astype(np.float32)
    B = g.standard_normal((n, d)).astype(np.float32)
    A = np.vstack([A, np.full((1, d), 0.5 * n, dtype=np.float32)])
    return A, B


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Set sizes drawn log-uniformly from [lo, hi]."""
    g = _rng(seed)
    return np.exp(g.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)


def to_bf16_bits(X: np.ndarray, chunk: int = 1 << 22) -> np.ndarray:
    """Round binary32 to bfloat16 (nearest even); returns the uint16 bit patterns.

    Works on 32-bit words in chunks on all host threads; patterns whose rounding
    increment would carry out of 32 bits (negative NaNs near 0xFFFFFFFF) wrap to
    0, as a 64-bit sum truncated to 16 bits would.
    """
    u = np.ascontiguousarray(X, dtype=np.float32).reshape(-1).view(np.uint32)
    out = np.empty(u.shape, dtype=np.uint16)

    def conv(lo):
        v = u[lo:lo + chunk]
        r = ((v >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
        out[lo:lo + chunk] = ((v + r) >> np.uint32(16)).astype(np.uint16)

    with np.errstate(over="ignore"):
        _pool_map(conv, range(0, u.size, chunk))
    return out.reshape(np.shape(X))


def bf16_bits_to_f32(H: np.ndarray) -> np.ndarray:
    H = np.asarray(H, dtype=np.uint16)
    out = np.empty(H.shape, dtype=np.uint32)
    flat_in, flat_out = H.reshape(-1), out.reshape(-1)
    step = 1 << 22

    def conv(lo):
        flat_out[lo:lo + step] = flat_in[lo:lo + step].astype(np.uint32) << np.uint32(16)

    _pool_map(conv, range(0, flat_in.size, step))
    return out.view(np.float32)


# E4M3 (OCP FP8, 'fn' variant: no infinities, max 448) value table
def _e4m3_table() -> np.ndarray:
    vals = np.zeros(256, dtype=np.float64)
    for b in range(256):
        s = -1.0 if b & 0x80 else 1.0
        e = (b >> 3) & 0xF
        m = b & 7
        if e == 0xF and m == 7:
            vals[b] = np.nan
        elif e == 0:
            vals[b] = s * m * 2.0 ** -9
        else:
            vals[b] = s * (1 + m / 8.0) * 2.0 ** (e - 7)
    return vals


E4M3_VALUES = _e4m3_table()


def _fp8_rows(X: np.ndarray):
    amax = np.abs(X).max(axis=1)
    scale = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    Y = (X / scale[:, None]).astype(np.float64)
    pos = E4M3_VALUES[:127]              # codes 0..126: non-negative finite, increasing
    mag = np.abs(Y)
    i = np.clip(np.searchsorted(pos, mag), 1, 126)
    lo, hi = pos[i - 1], pos[i]
    pick_hi = (hi - mag < mag - lo) | ((hi - mag == mag - lo) & (i % 2 == 0))
    code = np.where(pick_hi, i, i - 1).astype(np.uint8)
    code = np.where(mag >= pos[126], 126, code).astype(np.uint8)
    code = np.where(Y < 0, code | 0x80, code).astype(np.uint8)
    code = np.where(mag == 0, 0, code).astype(np.uint8)
    return code, scale


def to_fp8_e4m3(X: np.ndarray, chunk: int = 1 << 14):
    """Per-row scale = max|x| / 448, codes = nearest E4M3 of x / scale.

    Returns (codes uint8 [n, d], scales float32 [n]).  Ties go to the even code.
    Rows are converted in chunks on all host threads (each row on its own).
    """
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    code = np.empty(X.shape, dtype=np.uint8)
    scale = np.empty(n, dtype=np.float32)

    def conv(lo):
        code[lo:lo + chunk], scale[lo:lo + chunk] = _fp8_rows(X[lo:lo + chunk])

    _pool_map(conv, range(0, n, chunk))
    return code, scale


def fp8_dequant(codes: np.ndarray, scales: np.ndarray, chunk: int = 1 << 14) -> np.ndarray:
    """float32(E4M3 value) * row scale, one binary32 rounding."""
    codes = np.asarray(codes, dtype=np.uint8)
    scales = np.asarray(scales, dtype=np.float32)
    table = E4M3_VALUES.astype(np.float32)
    out = np.empty(codes.shape, dtype=np.float32)

    def conv(lo):
        out[lo:lo + chunk] = table[codes[lo:lo + chunk]] * scales[lo:lo + chunk, None]

    _pool_map(conv, range(0, codes.shape[0], chunk))
    return out
