"""A tensor-core screen whose pipeline waits run out (the bounded waits every
mbarrier wait of the kernel has): with a budget of a few SM cycles the screen's
first wait for a copy expires, the kernel stops issuing work, drains the copies
and MMAs it has issued, frees its tensor memory and the call reports
CH_ETIMEOUT.  The same context then runs normally and matches the oracle (Fig. 1,
step 3), so the expiry left it usable.  No GPU fault is involved: the wait gives
up on a barrier that has simply not completed yet."""
import numpy as np
import pytest

import oracle
from paper_2307_03043_gb300 import binding as ch
from paper_2307_03043_gb300 import workloads

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


@pytest.mark.parametrize("d,screen", [(64, ch.CH_SCREEN_TF32), (384, ch.CH_SCREEN_TF32)])
def test_screen_wait_expiry_reports_timeout_and_leaves_the_context_usable(ctx, d, screen):
    A, B = workloads.gaussian_mixture(3000, 20_000, d, 91, clusters=12)
    sA = ch.ch_set_create(ctx, A, 0, A.shape[0], d)
    sB = ch.ch_set_create(ctx, B, 0, B.shape[0], d)
    try:
        g = np.random.default_rng(d)
        idx_h = g.integers(0, A.shape[0], 700).astype(np.int64)
        idx = torch.from_numpy(idx_h).cuda()
        m = torch.zeros(700, dtype=torch.float32, device="cuda")
        am = torch.zeros(700, dtype=torch.int64, device="cuda")
        ch.ch_ctx_set_wait_cycles(ctx, 8)
        # the synchronising calls report the expiry: an estimate and the screened exact scan
        with pytest.raises(ch.ChamferError) as ei:
            ch.ch_estimate(ctx, sA, sB, ch.est_params(ch.CH_L2, T=700, sample_seed=3, screen=screen))
        assert ei.value.status == ch.CH_ETIMEOUT
        with pytest.raises(ch.ChamferError) as ei:
            ch.ch_exact(ctx, sA, sB, ch.CH_L2, 1)
        assert ei.value.status == ch.CH_ETIMEOUT
        ch.ch_ctx_set_wait_cycles(ctx, 0)
        # the context runs normally afterwards
        ch.ch_sampled_nn(ctx, sA, idx, 700, sB, ch.CH_L2, screen, 8, m, am)
        mo, amo = oracle.scan(A, idx_h, B, oracle.L2)
        m_h, am_h = m.cpu().numpy(), am.cpu().numpy()
        hit = am_h == amo
        assert np.mean(hit) >= 0.99
        assert np.array_equal(m_h[hit].view(np.uint32), mo[hit].view(np.uint32))
        eta = ch.ch_estimate(ctx, sA, sB, ch.est_params(ch.CH_L2, T=700, sample_seed=3, hash_seed=2, screen=screen))
        eta_o = oracle.estimate(A, B, oracle.L2, 2, 3, T=700)
        assert abs(eta / eta_o - 1) < 1e-5
    finally:
        ch.ch_ctx_set_wait_cycles(ctx, 0)
        ch.ch_set_destroy(sA)
        ch.ch_set_destroy(sB)


def test_wait_budget_argument_checks(ctx):
    with pytest.raises(ch.ChamferError) as ei:
        ch.ch_ctx_set_wait_cycles(ctx, -1)
    assert ei.value.status == ch.CH_EINVAL
    ch.ch_ctx_set_wait_cycles(ctx, 0)
