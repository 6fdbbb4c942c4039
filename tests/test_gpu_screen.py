"""Tensor-core screen (tcgen05 TF32 / BF16 / FP8) + canonical rerank of the
sampled l2 scan, against the oracle's exact scan.

The screen keeps each sample's R best candidates by |b|^2 - 2 q.b computed on
the tensor cores; the rerank evaluates the canonical binary32 distance on them.
So every reported minimum is a real canonical distance (>= the exact minimum,
with its argmin attaining it) and equals the exact minimum whenever the nearest
point survives the screen.  BF16 / FP8 sets are compared with the oracle run on
their dequantised binary32 values.
"""
import numpy as np
import pytest

import oracle
from paper_2307_03043_gb300 import binding as ch
from paper_2307_03043_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L2 = ch.CH_L2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03043_gb300 import build
    build.build()
    c = ch.ch_ctx_create(0, torch.cuda.current_stream())
    yield c
    ch.ch_ctx_destroy(c)


def _set(ctx, host, dtype, scales=None):
    t = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    sc = torch.from_numpy(scales).cuda() if scales is not None else None
    s = ch.ch_set_create(ctx, t, 2 if scales is None else 1, host.shape[0], host.shape[1], dtype, sc)
    return s, t, sc


def _run(ctx, sA, sB, idx, screen, R=8):
    T = idx.size
    m = torch.zeros(T, dtype=torch.float32, device="cuda")
    am = torch.zeros(T, dtype=torch.int64, device="cuda")
    ch.ch_sampled_nn(ctx, sA, torch.from_numpy(idx).cuda(), T, sB, L2, screen, R, m, am)
    return m.cpu().numpy(), am.cpu().numpy()


def _check(A32, B32, idx, m, am, max_miss):
    ok = idx >= 0
    mo, _ = oracle.scan(A32, idx[ok], B32, L2)
    mg, ag = m[ok], am[ok]
    assert np.all(mg >= mo)
    for l in np.flatnonzero(ok)[:: max(1, ok.sum() // 200)]:
        assert oracle.dist(A32[idx[l]], B32[am[l]], L2) == m[l]
    miss = float(np.mean(mg != mo))
    assert miss <= max_miss, miss
    assert np.all(m[~ok] == 0) and np.all(am[~ok] == -1)
    return miss


@pytest.mark.parametrize("nA,nB,d,T", [(300, 1000, 32, 130), (700, 3000, 128, 515), (256, 255, 64, 129),
                                       (1000, 4099, 16, 1), (900, 5000, 96, 2000)])
def test_tf32_screen(ctx, nA, nB, d, T):
    A, B = workloads.gaussian_mixture(nA, nB, d, d + T, clusters=13)
    sA, tA, _ = _set(ctx, A, ch.CH_F32)
    sB, tB, _ = _set(ctx, B, ch.CH_F32)
    idx = np.random.default_rng(T).integers(0, nA, T).astype(np.int64)
    idx[1::29] = -1
    m, am = _run(ctx, sA, sB, idx, ch.CH_SCREEN_TF32)
    _check(A, B, idx, m, am, 0.01)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_bf16_screen(ctx):
    A, B = workloads.unit_mixture(2000, 6000, 384, 1, clusters=50)
    Ah, Bh = workloads.to_bf16_bits(A), workloads.to_bf16_bits(B)
    A32, B32 = workloads.bf16_bits_to_f32(Ah), workloads.bf16_bits_to_f32(Bh)
    sA, tA, _ = _set(ctx, Ah, ch.CH_BF16)
    sB, tB, _ = _set(ctx, Bh, ch.CH_BF16)
    idx = np.random.default_rng(2).integers(0, 2000, 777).astype(np.int64)
    m, am = _run(ctx, sA, sB, idx, ch.CH_SCREEN_BF16)
    _check(A32, B32, idx, m, am, 0.005)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_fp8_screen(ctx):
    A, B = workloads.unit_mixture(1500, 5000, 256, 3, clusters=40)
    ca, sa = workloads.to_fp8_e4m3(A)
    cb, sb = workloads.to_fp8_e4m3(B)
    A32, B32 = workloads.fp8_dequant(ca, sa), workloads.fp8_dequant(cb, sb)
    sA, tA, _ = _set(ctx, ca, ch.CH_FP8E4M3, sa)
    sB, tB, _ = _set(ctx, cb, ch.CH_FP8E4M3, sb)
    idx = np.random.default_rng(4).integers(0, 1500, 600).astype(np.int64)
    m, am = _run(ctx, sA, sB, idx, ch.CH_SCREEN_FP8)
    _check(A32, B32, idx, m, am, 0.01)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_rerank_width(ctx):
    A, B = workloads.gaussian_mixture(500, 2000, 64, 9, clusters=5)
    sA, tA, _ = _set(ctx, A, ch.CH_F32)
    sB, tB, _ = _set(ctx, B, ch.CH_F32)
    idx = np.arange(500, dtype=np.int64)
    misses = []
    for R in (1, 8, 16, 32):
        m, am = _run(ctx, sA, sB, idx, ch.CH_SCREEN_TF32, R)
        misses.append(_check(A, B, idx, m, am, 0.05 if R == 1 else 0.01))
    assert misses[-1] <= misses[0]
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_estimate_with_tf32_screen_matches_oracle(ctx):
    A, B = workloads.gaussian_mixture(20000, 20000, 128, 5)
    sA, tA, _ = _set(ctx, A, ch.CH_F32)
    sB, tB, _ = _set(ctx, B, ch.CH_F32)
    p = ch.est_params(L2, 10, 16, None, 3, eps=0.1, sample_seed=4, screen=ch.CH_SCREEN_AUTO)
    eta, rep = ch.ch_estimate(ctx, sA, sB, p, report=True)
    eta_o = oracle.estimate(A, B, L2, 3, 4, T=rep.T)
    assert abs(eta / eta_o - 1) < 1e-5
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_exact_tc_mode_matches_direct(ctx):
    A, B = workloads.gaussian_mixture(3000, 2500, 64, 6, clusters=20)
    sA, tA, _ = _set(ctx, A, ch.CH_F32)
    sB, tB, _ = _set(ctx, B, ch.CH_F32)
    m0 = torch.zeros(3000, device="cuda")
    m1 = torch.zeros(3000, device="cuda")
    v0 = ch.ch_exact(ctx, sA, sB, L2, 0, m0)
    v1 = ch.ch_exact(ctx, sA, sB, L2, 1, m1)
    m0, m1 = m0.cpu().numpy(), m1.cpu().numpy()
    assert np.all(m1 >= m0) and np.mean(m1 != m0) < 0.01
    assert abs(v1 / v0 - 1) < 1e-4
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


@pytest.mark.parametrize("dtype,d", [(ch.CH_F32, 768), (ch.CH_F32, 1000), (ch.CH_BF16, 768), (ch.CH_BF16, 1536),
                                     (ch.CH_FP8E4M3, 1024)])
def test_wide_rows_stream_the_sample_tile(ctx, dtype, d):
    """Rows of 768 bytes or more: the sample tile's K blocks stream through the
    stages with B's instead of staying resident (the serving mix has d = 768)."""
    A, B = workloads.unit_mixture(900, 2600, d, 7 + d, clusters=30)
    if dtype == ch.CH_F32:
        A32, B32, sa, sb = A, B, None, None
        sA, tA, _ = _set(ctx, A, dtype)
        sB, tB, _ = _set(ctx, B, dtype)
        screen = ch.CH_SCREEN_TF32
    elif dtype == ch.CH_BF16:
        Ah, Bh = workloads.to_bf16_bits(A), workloads.to_bf16_bits(B)
        A32, B32 = workloads.bf16_bits_to_f32(Ah), workloads.bf16_bits_to_f32(Bh)
        sA, tA, _ = _set(ctx, Ah, dtype)
        sB, tB, _ = _set(ctx, Bh, dtype)
        screen = ch.CH_SCREEN_BF16
    else:
        ca, sa = workloads.to_fp8_e4m3(A)
        cb, sb = workloads.to_fp8_e4m3(B)
        A32, B32 = workloads.fp8_dequant(ca, sa), workloads.fp8_dequant(cb, sb)
        sA, tA, _ = _set(ctx, ca, dtype, sa)
        sB, tB, _ = _set(ctx, cb, dtype, sb)
        screen = ch.CH_SCREEN_FP8
    idx = np.random.default_rng(d).integers(0, 900, 333).astype(np.int64)
    idx[::41] = -1
    m, am = _run(ctx, sA, sB, idx, screen)
    _check(A32, B32, idx, m, am, 0.01)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)
