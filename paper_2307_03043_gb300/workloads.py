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


def unit_mixture(n_a: int, n_b: int, d: int, seed: int, clusters: int = 1000,
                 sigma: float = 0.3, chunk: int = 1 << 18):
    """Unit-norm mixture vectors (stand-in for DEEP1B / MS-Turing embeddings).

    1000 unit centres (normalised N(0, I)); point = normalise(centre +
    N(0, sigma^2 I / d)); A and B are independent draws of the same mixture.
    """
    g = _rng(seed)
    C = g.standard_normal((clusters, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    s = sigma / math.sqrt(d)

    def draw(n):
        out = np.empty((n, d), dtype=np.float32)
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            lab = g.integers(0, clusters, size=hi - lo)
            x = C[lab] + s * g.standard_normal((hi - lo, d))
            x /= np.linalg.norm(x, axis=1, keepdims=True)
            out[lo:hi] = x
        return out

    return draw(n_a), draw(n_b)


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


def to_bf16_bits(X: np.ndarray) -> np.ndarray:
    """Round binary32 to bfloat16 (nearest even); returns the uint16 bit patterns."""
    u = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def bf16_bits_to_f32(H: np.ndarray) -> np.ndarray:
    return (np.asarray(H, dtype=np.uint32) << 16).view(np.float32)


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


def to_fp8_e4m3(X: np.ndarray):
    """Per-row scale = max|x| / 448, codes = nearest E4M3 of x / scale.

    Returns (codes uint8 [n, d], scales float32 [n]).  Ties go to the even code.
    """
    X = np.asarray(X, dtype=np.float32)
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


def fp8_dequant(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """float32(E4M3 value) * row scale, one binary32 rounding."""
    v = E4M3_VALUES[np.asarray(codes, dtype=np.uint8)].astype(np.float32)
    return (v * np.asarray(scales, dtype=np.float32)[:, None]).astype(np.float32)
