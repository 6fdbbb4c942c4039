"""Serving loop (ch_serve_*): continuous admission over resident sets, results
identical alone and in the mix, footprint admission, bounded waits, and
host-side fault injection (no device fault is ever provoked)."""
import os

import numpy as np
import pytest

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
    c = ch.ch_ctx_create(0, None)
    yield c
    ch.ch_ctx_destroy(c)


def _server(ctx, budget=8 << 30, slots=4, queue=1024, fault=None):
    old = os.environ.pop("CH_SERVE_FAULT", None)
    if fault:
        os.environ["CH_SERVE_FAULT"] = fault
    try:
        return ch.ch_serve_create(ctx, budget, slots, queue)
    finally:
        os.environ.pop("CH_SERVE_FAULT", None)
        if old is not None:
            os.environ["CH_SERVE_FAULT"] = old


def _sets(n_sets=6, seed=0):
    sizes = workloads.log_uniform_sizes(n_sets, 500, 20000, seed)
    out = []
    for i, n in enumerate(sizes):
        A, _ = workloads.gaussian_mixture(int(n), 1, 64, seed * 100 + i, clusters=10)
        out.append(A)
    return out


def test_results_identical_alone_and_mixed(ctx):
    data = _sets()
    srv = _server(ctx)
    ids = [ch.ch_serve_register(srv, X, 0, X.shape[0], 64) for X in data]
    rng = np.random.default_rng(1)
    jobs = []
    for k in range(24):
        a, b = rng.integers(0, len(ids), 2)
        metric = ch.CH_L2 if k % 3 else ch.CH_L1
        p = ch.est_params(metric, 10, 16, None, k, eps=0.2, sample_seed=100 + k)
        st, t = ch.ch_serve_submit(srv, ids[a], ids[b], p)
        assert st == ch.CH_OK
        jobs.append((t, a, b, p))
    got = {}
    for t, a, b, p in jobs:
        st, eta, rs = ch.ch_serve_wait(srv, t, 60000)
        assert st == ch.CH_OK and rs == ch.CH_OK
        got[t] = eta
    stats = ch.ch_serve_stats_get(srv)
    assert stats.completed == 24 and stats.failed == 0
    assert stats.p50_us > 0 and stats.p99_us >= stats.p50_us
    ch.ch_serve_stats_reset(srv)  # a new measurement window
    stats = ch.ch_serve_stats_get(srv)
    assert stats.completed == 0 and stats.p50_us == 0 and stats.peak_bytes > 0
    st, t = ch.ch_serve_submit(srv, ids[0], ids[1], jobs[0][3])
    ch.ch_serve_wait(srv, t, 60000)
    assert ch.ch_serve_stats_get(srv).completed == 1
    ch.ch_serve_destroy(srv)
    # each request alone, on a fresh context and fresh sets
    c2 = ch.ch_ctx_create(0, None)
    sets = [ch.ch_set_create(c2, X, 0, X.shape[0], 64) for X in data]
    for t, a, b, p in jobs:
        assert ch.ch_estimate(c2, sets[a], sets[b], p) == got[t]
    for s in sets:
        ch.ch_set_destroy(s)
    ch.ch_ctx_destroy(c2)


def test_admission_by_footprint(ctx):
    A, B = workloads.gaussian_mixture(20000, 20000, 128, 3)
    srv = _server(ctx, budget=1 << 20)  # 1 MiB: nothing of this size fits
    ia = ch.ch_serve_register(srv, A, 0, 20000, 128)
    ib = ch.ch_serve_register(srv, B, 0, 20000, 128)
    st, _ = ch.ch_serve_submit(srv, ia, ib, ch.est_params(ch.CH_L2, eps=0.1))
    assert st == ch.CH_EBUSY
    assert ch.ch_serve_stats_get(srv).rejected == 1
    ch.ch_serve_destroy(srv)
    # a budget that admits one request at a time still completes them all
    srv = _server(ctx, budget=200 << 20, slots=4)
    ia = ch.ch_serve_register(srv, A, 0, 20000, 128)
    ib = ch.ch_serve_register(srv, B, 0, 20000, 128)
    ts = [ch.ch_serve_submit(srv, ia, ib, ch.est_params(ch.CH_L2, eps=0.1, hash_seed=k, sample_seed=k))[1]
          for k in range(6)]
    for t in ts:
        st, eta, rs = ch.ch_serve_wait(srv, t, 60000)
        assert st == ch.CH_OK and rs == ch.CH_OK and eta > 0
    assert ch.ch_serve_stats_get(srv).peak_bytes <= 200 << 20
    ch.ch_serve_destroy(srv)


def test_queue_full_and_wait_timeout(ctx):
    A, B = workloads.uniform(3000, 3000, 32, 4)
    srv = _server(ctx, slots=1, queue=1, fault="slow")  # each request sleeps 50 ms on the host
    ia = ch.ch_serve_register(srv, A, 0, 3000, 32)
    ib = ch.ch_serve_register(srv, B, 0, 3000, 32)
    p = ch.est_params(ch.CH_L1, T=200)
    st1, t1 = ch.ch_serve_submit(srv, ia, ib, p)
    assert st1 == ch.CH_OK
    statuses = [ch.ch_serve_submit(srv, ia, ib, p)[0] for _ in range(5)]
    assert ch.CH_EAGAIN in statuses
    st, _, _ = ch.ch_serve_wait(srv, t1, 1)
    assert st in (ch.CH_ETIMEOUT, ch.CH_OK)
    st, eta, rs = ch.ch_serve_wait(srv, t1, 60000) if st == ch.CH_ETIMEOUT else (st, 1.0, ch.CH_OK)
    assert st == ch.CH_OK and rs == ch.CH_OK
    ch.ch_serve_destroy(srv)


def test_injected_launch_failure_is_reported_and_server_survives(ctx):
    A, B = workloads.uniform(1000, 1200, 16, 5)
    srv = _server(ctx, fault="launch")
    ia = ch.ch_serve_register(srv, A, 0, 1000, 16)
    ib = ch.ch_serve_register(srv, B, 0, 1200, 16)
    t = ch.ch_serve_submit(srv, ia, ib, ch.est_params(T=100))[1]
    st, _, rs = ch.ch_serve_wait(srv, t, 60000)
    assert st == ch.CH_OK and rs == ch.CH_ECUDA
    assert ch.ch_serve_stats_get(srv).failed == 1
    ch.ch_serve_destroy(srv)
    # an injected admission refusal, then a healthy server on the same context
    srv = _server(ctx, fault="admit")
    ia = ch.ch_serve_register(srv, A, 0, 1000, 16)
    ib = ch.ch_serve_register(srv, B, 0, 1200, 16)
    assert ch.ch_serve_submit(srv, ia, ib, ch.est_params(T=100))[0] == ch.CH_EBUSY
    ch.ch_serve_destroy(srv)
    srv = _server(ctx)
    ia = ch.ch_serve_register(srv, A, 0, 1000, 16)
    ib = ch.ch_serve_register(srv, B, 0, 1200, 16)
    t = ch.ch_serve_submit(srv, ia, ib, ch.est_params(T=100))[1]
    st, eta, rs = ch.ch_serve_wait(srv, t, 60000)
    assert st == ch.CH_OK and rs == ch.CH_OK and eta > 0
    ch.ch_serve_destroy(srv)


def test_register_rejects_non_finite(ctx):
    A = np.ones((10, 8), np.float32)
    A[3, 3] = np.inf
    srv = _server(ctx)
    with pytest.raises(ch.ChamferError) as ei:
        ch.ch_serve_register(srv, A, 0, 10, 8)
    assert ei.value.status == ch.CH_EINVAL
    ch.ch_serve_destroy(srv)


def test_indexed_server_same_bits_as_plain_estimates(ctx):
    """A server made an index (ch_serve_index): every registered set keeps its
    l2 embedding under the index's hash seed resident; requests with that seed
    skip both projections, others project as before.  Every result, alone or
    mixed, is the plain ch_estimate's bit for bit; registering before indexing is
    refused with CH_EBUSY."""
    data = _sets(5, seed=3)
    srv = _server(ctx)
    hp = ch.hash_params(ch.CH_L2, 10, 16, None, 77)
    ch.ch_serve_index(srv, hp)
    ids = [ch.ch_serve_register(srv, X, 0, X.shape[0], 64) for X in data]
    with pytest.raises(ch.ChamferError) as ei:
        ch.ch_serve_index(srv, hp)
    assert ei.value.status == ch.CH_EBUSY
    rng = np.random.default_rng(5)
    jobs = []
    for k in range(20):
        a, b = rng.integers(0, len(ids), 2)
        seed = 77 if k % 4 else 1000 + k  # most on the index's seed, some off it
        p = ch.est_params(ch.CH_L2, 10, 16, None, seed, eps=0.2, sample_seed=300 + k)
        st, t = ch.ch_serve_submit(srv, ids[a], ids[b], p)
        assert st == ch.CH_OK
        jobs.append((t, a, b, p))
    got = {}
    for t, a, b, p in jobs:
        st, eta, rs = ch.ch_serve_wait(srv, t, 60000)
        assert st == ch.CH_OK and rs == ch.CH_OK
        got[t] = eta
    ch.ch_serve_destroy(srv)
    c2 = ch.ch_ctx_create(0, None)
    sets = [ch.ch_set_create(c2, X, 0, X.shape[0], 64) for X in data]
    for t, a, b, p in jobs:
        assert ch.ch_estimate(c2, sets[a], sets[b], p) == got[t]
    for x in sets:
        ch.ch_set_destroy(x)
    ch.ch_ctx_destroy(c2)
