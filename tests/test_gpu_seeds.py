"""Theorem 1 and Lemma 1 on the GPU: over 256 independent seeds of the full
estimator (CrudeNN + importance sampling + screened scans) at eps = 0.1 on a
50k x 50k, d = 128 Gaussian mixture, at least 99 % of the estimates lie within
(1 +- 0.1) of the exact Chamfer distance (GPU brute force, canonical binary32
distances summed in binary64), and their mean lies within 4 standard errors of
it (the estimator is unbiased)."""
import numpy as np
import pytest

from paper_2307_03043_gb300 import binding as ch
from paper_2307_03043_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = 256
BATCH = 32


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03043_gb300 import build
    build.build()
    c = ch.ch_ctx_create(0, torch.cuda.current_stream())
    yield c
    ch.ch_ctx_destroy(c)


@pytest.mark.parametrize("metric", [ch.CH_L2, ch.CH_L1])
def test_estimates_over_seeds(ctx, metric):
    A, B = workloads.gaussian_mixture(50_000, 50_000, 128, 77)
    sA = ch.ch_set_create(ctx, A, 0, A.shape[0], 128)
    sB = ch.ch_set_create(ctx, B, 0, B.shape[0], 128)
    try:
        exact = ch.ch_exact(ctx, sA, sB, metric, 0)
        etas = []
        for b0 in range(0, SEEDS, BATCH):
            prm = [ch.est_params(metric, 10, 16, None, 1000 + s, eps=0.1, sample_seed=5000 + s)
                   for s in range(b0, b0 + BATCH)]
            e, st = ch.ch_estimate_batch(ctx, [sA] * BATCH, [sB] * BATCH, prm)
            assert all(x == ch.CH_OK for x in st)
            etas += e
        etas = np.asarray(etas)
        rel = etas / exact - 1.0
        assert np.mean(np.abs(rel) <= 0.1) >= 0.99, np.sort(np.abs(rel))[-5:]
        se = etas.std(ddof=1) / np.sqrt(SEEDS)
        assert abs(etas.mean() - exact) <= 4 * se, (etas.mean(), exact, se)
    finally:
        ch.ch_set_destroy(sA)
        ch.ch_set_destroy(sB)
