"""ch_sample_static -- the sampling entry point for callers that cannot allocate
device memory (a plug-in whose host application owns every device allocation,
a process held to a fixed device-memory budget) -- must return exactly what
ch_sample returns.

Collected last on purpose, so a run that stops at the first failure has
already run everything else.  Passes alone in a fresh process and after the
other tests (the first call on the device does the one-time address look-up).
"""
import numpy as np
import pytest

import oracle
from paper_2307_03043_gb300 import binding as ch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03043_gb300 import build
    build.build()
    c = ch.ch_ctx_create(0, torch.cuda.current_stream())
    yield c
    ch.ch_ctx_destroy(c)


def _reference(ctx, D, T, seed):
    n = D.numel()
    idx = torch.zeros(max(T, 1), dtype=torch.int64, device="cuda")
    w = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    W = ch.ch_sample(ctx, D, n, T, seed, idx, w, want_total=True)
    return idx[:T].cpu().numpy(), w[:n].cpu().numpy(), W


def _static(D, T, seed):
    n = D.numel()
    idx = torch.full((max(T, 1),), 7, dtype=torch.int64, device="cuda")
    w = torch.full((max(n, 1),), 7, dtype=torch.int64, device="cuda")
    W = torch.zeros(1, dtype=torch.int64, device="cuda")
    ch.ch_sample_static(D, n, T, seed, idx, w, W, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return idx[:T].cpu().numpy(), w[:n].cpu().numpy(), int(W.cpu().numpy().view(np.uint64)[0])


def test_static_sampling_matches_ch_sample_twice(ctx):
    g = np.random.default_rng(0)
    cases = [(g.random(300_001).astype(np.float32) * 7, 4097, 11),
             (np.where(g.random(2_000) < 0.3, 0, g.random(2_000)).astype(np.float32), 999, 12)]
    for _ in range(2):  # two calls in a row per case: the shared scratch keeps no state that matters
        for Dn, T, seed in cases:
            D = torch.from_numpy(Dn).cuda()
            ri, rw, rW = _reference(ctx, D, T, seed)
            si, sw, sW = _static(D, T, seed)
            assert sW == rW
            assert np.array_equal(si, ri)
            assert np.array_equal(sw, rw)


def test_static_sampling_at_the_largest_size_matches_the_oracle(ctx):
    """nA = 1,048,576, the documented maximum: the last weight-scan block and the
    prefix are full.  Weights, W and the draws equal the oracle's (Fig. 1 steps
    2-3) and ch_sample's, on two calls in a row."""
    n = 1 << 20
    g = np.random.default_rng(5)
    Dn = (g.random(n) * g.random(n) ** 4).astype(np.float32)
    Dn[g.integers(0, n, 1000)] = 0.0
    w_o, prefix_o, W_o, _ = oracle.weights(Dn)
    T = 5000
    idx_o = oracle.draws(prefix_o, W_o, T, 21)
    D = torch.from_numpy(Dn).cuda()
    ri, rw, rW = _reference(ctx, D, T, 21)
    for _ in range(2):
        si, sw, sW = _static(D, T, 21)
        assert sW == rW == W_o
        assert np.array_equal(sw.view(np.uint64), w_o) and np.array_equal(rw.view(np.uint64), w_o)
        assert np.array_equal(si, idx_o) and np.array_equal(ri, idx_o)


def test_static_sampling_limits(ctx):
    D = torch.zeros(4, dtype=torch.float32, device="cuda")
    idx = torch.zeros(3, dtype=torch.int64, device="cuda")
    w = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(ch.ChamferError) as ei:  # beyond the fixed scratch: refused before any work
        ch.ch_sample_static(D, (1 << 20) + 1, 3, 0, idx, w)
    assert ei.value.status == ch.CH_EINVAL
    ch.ch_sample_static(D, 4, 3, 0, idx, w)  # all-zero weights: every draw is -1
    torch.cuda.synchronize()
    assert np.all(idx.cpu().numpy() == -1)
