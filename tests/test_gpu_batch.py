"""ch_estimate_batch: many pairs in one call, each equal bit for bit to its own
ch_estimate; failing pairs report their status without stopping the others."""
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
    c = ch.ch_ctx_create(0, torch.cuda.current_stream())
    yield c
    ch.ch_ctx_destroy(c)


def _pairs(ctx, n_pairs, d, seed):
    sizes = workloads.log_uniform_sizes(2 * n_pairs, 100, 20_000, seed)
    sets = []
    for i in range(2 * n_pairs):
        if d == 3:
            X, _ = workloads.shape_surface(int(sizes[i]), 1, seed * 100 + i)
        else:
            X, _ = workloads.gaussian_mixture(int(sizes[i]), 1, d, seed * 100 + i, clusters=10)
        sets.append(ch.ch_set_create(ctx, X, 0, X.shape[0], d))
    return sets


@pytest.mark.parametrize("d", [3, 64])
def test_batch_equals_single(ctx, d):
    sets = _pairs(ctx, 12, d, d)
    A, B, P = [], [], []
    for i in range(12):
        for metric in (ch.CH_L1, ch.CH_L2):
            A.append(sets[2 * i])
            B.append(sets[2 * i + 1])
            P.append(ch.est_params(metric, 10, 16, None, 3 * i + metric, eps=0.1, sample_seed=7 * i + metric))
    # one set in several pairs, on different lanes
    A.append(sets[0]); B.append(sets[3]); P.append(ch.est_params(ch.CH_L2, hash_seed=1, sample_seed=2))
    A.append(sets[3]); B.append(sets[0]); P.append(ch.est_params(ch.CH_L2, hash_seed=1, sample_seed=2))
    eta, st = ch.ch_estimate_batch(ctx, A, B, P)
    assert all(s == ch.CH_OK for s in st)
    for i in range(len(A)):
        assert eta[i] == ch.ch_estimate(ctx, A[i], B[i], P[i]), i
        assert eta[i] > 0
    for s in sets:
        ch.ch_set_destroy(s)


def test_batch_failures_and_empty(ctx):
    X, Y = workloads.uniform(500, 700, 8, 4)
    sX = ch.ch_set_create(ctx, X, 0, 500, 8)
    sY = ch.ch_set_create(ctx, Y, 0, 700, 8)
    sE = ch.ch_set_create(ctx, np.zeros((0, 8), np.float32), 0, 0, 8)
    bad = X.copy()
    bad[7, 3] = np.inf
    sBad = ch.ch_set_create(ctx, bad, 0, 500, 8)
    A = [sX, sE, sX, sBad, sY]
    B = [sY, sY, sE, sY, sX]
    P = [ch.est_params(ch.CH_L2, T=300, hash_seed=k, sample_seed=k) for k in range(5)]
    P[4] = ch.est_params(ch.CH_L1, T=0, eps=1.5)  # eps outside (0, 1)
    eta, st = ch.ch_estimate_batch(ctx, A, B, P)
    assert st == [ch.CH_OK, ch.CH_OK, ch.CH_EINVAL, ch.CH_EINVAL, ch.CH_EINVAL]
    assert eta[0] == ch.ch_estimate(ctx, sX, sY, P[0])
    assert eta[1] == 0.0 and eta[2] == 0.0 and eta[3] == 0.0 and eta[4] == 0.0
    assert ch.ch_estimate_batch(ctx, [], [], []) == ([], [])
    for s in (sX, sY, sE, sBad):
        ch.ch_set_destroy(s)


@pytest.mark.parametrize("d", [1, 2, 4])
def test_batch_small_d_all_storage_types(ctx, d):
    """Pairs of d <= 4 go through one batched exact scan per (storage type,
    metric, d); the first call tunes its chunk length, the second reuses it, and
    both equal the single-pair estimates bit for bit."""
    sizes = workloads.log_uniform_sizes(12, 50, 30_000, 40 + d)
    made, A, B, P = [], [], [], []
    for i in range(6):
        X, _ = workloads.gaussian_mixture(int(sizes[2 * i]), 1, d, 500 + i, clusters=5)
        Y, _ = workloads.gaussian_mixture(int(sizes[2 * i + 1]), 1, d, 600 + i, clusters=5)
        for kind in ("f32", "bf16", "fp8"):
            if kind == "f32":
                sX = ch.ch_set_create(ctx, X, 0, X.shape[0], d)
                sY = ch.ch_set_create(ctx, Y, 0, Y.shape[0], d)
            elif kind == "bf16":
                sX = ch.ch_set_create(ctx, torch.from_numpy(workloads.to_bf16_bits(X)).cuda(), 1, X.shape[0], d,
                                      ch.CH_BF16)
                sY = ch.ch_set_create(ctx, torch.from_numpy(workloads.to_bf16_bits(Y)).cuda(), 1, Y.shape[0], d,
                                      ch.CH_BF16)
            else:
                cx, sx = workloads.to_fp8_e4m3(X)
                cy, sy = workloads.to_fp8_e4m3(Y)
                sX = ch.ch_set_create(ctx, torch.from_numpy(cx).cuda(), 1, X.shape[0], d, ch.CH_FP8E4M3,
                                      torch.from_numpy(sx).cuda())
                sY = ch.ch_set_create(ctx, torch.from_numpy(cy).cuda(), 1, Y.shape[0], d, ch.CH_FP8E4M3,
                                      torch.from_numpy(sy).cuda())
            made += [sX, sY]
            for metric in (ch.CH_L1, ch.CH_L2):
                A.append(sX)
                B.append(sY)
                P.append(ch.est_params(metric, hash_seed=i, sample_seed=10 * i + metric, eps=0.2))
    single = [ch.ch_estimate(ctx, A[i], B[i], P[i]) for i in range(len(A))]
    for _ in range(2):
        eta, st = ch.ch_estimate_batch(ctx, A, B, P)
        assert all(s == ch.CH_OK for s in st)
        assert eta == single
    torch.cuda.synchronize()
    for s in made:
        ch.ch_set_destroy(s)


def test_batch_mixes_batched_and_lane_crude_nn(ctx):
    """One call holding pairs whose CrudeNN runs in the batched launches (one
    table group, grid family, hash tables) beside pairs that take the per-pair
    path (sort grouping, SimHash, k x W, uniform sampling, a pair with several
    table groups): every estimate equals its lone one."""
    sets = _pairs(ctx, 6, 8, 21)
    Xb, Yb = workloads.gaussian_mixture(400_000, 600_000, 8, 5, clusters=50)  # 600k points: several table groups
    sBig = ch.ch_set_create(ctx, Xb, 0, Xb.shape[0], 8)
    sBig2 = ch.ch_set_create(ctx, Yb, 0, Yb.shape[0], 8)
    A, B, P = [], [], []
    variants = [dict(), dict(group=ch.CH_GROUP_SORT), dict(family=ch.CH_FAMILY_SIMHASH), dict(window=4, repeats=2),
                dict(sampling=ch.CH_SAMPLING_UNIFORM), dict()]
    for i, kw in enumerate(variants):
        for metric in (ch.CH_L1, ch.CH_L2):
            if kw.get("family") == ch.CH_FAMILY_SIMHASH and metric == ch.CH_L1:
                continue
            A.append(sets[2 * i])
            B.append(sets[2 * i + 1])
            P.append(ch.est_params(metric, hash_seed=5 * i + metric, sample_seed=3 * i + metric, eps=0.2, **kw))
    A.append(sBig); B.append(sBig2); P.append(ch.est_params(ch.CH_L2, hash_seed=9, sample_seed=9, eps=0.2))
    A.append(sBig); B.append(sBig2); P.append(ch.est_params(ch.CH_L1, hash_seed=9, sample_seed=9, eps=0.2))
    eta, st = ch.ch_estimate_batch(ctx, A, B, P)
    assert all(s == ch.CH_OK for s in st), st
    for i in range(len(A)):
        assert eta[i] == ch.ch_estimate(ctx, A[i], B[i], P[i]), i
    torch.cuda.synchronize()
    for s in sets + [sBig, sBig2]:
        ch.ch_set_destroy(s)
