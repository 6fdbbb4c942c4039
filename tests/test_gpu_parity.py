"""GPU (libchamfer through its C ABI) versus the CPU oracle, element by element.

Bit-exact: bucket keys, scale exponents, b(a), level, D_a, weights w_a, W and
the sample indices, the exact-scan minima and argmins.  Estimates: within
1e-5 relative (the binary64 sums differ only in order).
"""
import numpy as np
import pytest

import oracle
from paper_2307_03043_gb300 import binding as ch
from paper_2307_03043_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L1, L2 = ch.CH_L1, ch.CH_L2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03043_gb300 import build
    build.build()
    c = ch.ch_ctx_create(0, torch.cuda.current_stream())
    yield c
    ch.ch_ctx_destroy(c)


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


class Pair:
    """Device copies of A and B registered as libchamfer sets (adopted)."""

    def __init__(self, ctx, A, B):
        self.ctx = ctx
        self.A_np, self.B_np = A, B
        self.A, self.B = dev(A), dev(B)
        self.sA = ch.ch_set_create(ctx, self.A, 2, A.shape[0], A.shape[1])
        self.sB = ch.ch_set_create(ctx, self.B, 2, B.shape[0], B.shape[1])

    def close(self):
        ch.ch_set_destroy(self.sA)
        ch.ch_set_destroy(self.sB)
        torch.cuda.synchronize()


@pytest.fixture
def pair_factory(ctx):
    made = []

    def make(A, B):
        p = Pair(ctx, A, B)
        made.append(p)
        return p

    yield make
    for p in made:
        p.close()


def gpu_crude(ctx, p, metric, seed, L=10, k=16, top_exp=None, group=ch.CH_GROUP_HASH):
    nA = p.A_np.shape[0]
    bidx = torch.full((nA,), -5, dtype=torch.int64, device="cuda")
    D = torch.full((nA,), -1.0, dtype=torch.float32, device="cuda")
    lv = torch.full((nA,), 255, dtype=torch.uint8, device="cuda")
    ch.ch_crude_nn(ctx, p.sA, p.sB, ch.hash_params(metric, L, k, top_exp, seed, group), bidx, D, lv)
    return bidx.cpu().numpy(), D.cpu().numpy(), lv.cpu().numpy()


# ------------------------------------------------------------------ hashing
@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("n,d", [(1037, 16), (517, 3), (300, 33), (260, 128)])
def test_keys_bit_exact(ctx, pair_factory, metric, n, d):
    A, B = workloads.gaussian_mixture(n, 50, d, n + d, clusters=7)
    p = pair_factory(A, B)
    for L, e_lo in ((10, -6), (3, 2), (17, -12)):
        hp = ch.hash_params(metric, L, 16, None, 1234 + L)
        keys = torch.zeros((L, n), dtype=torch.int64, device="cuda")
        ch.ch_hash_keys(ctx, p.sA, hp, e_lo, keys)
        got = keys.cpu().numpy().view(np.uint64)
        Y = oracle.hashed(A, metric, 1234 + L, 16)
        want = oracle.keys(Y, e_lo, L, 1234 + L)
        assert np.array_equal(got, want)


def _typed_set(ctx, X32, dtype, keep):
    """A set of X32 stored as dtype; returns (set, dequantised binary32 values)."""
    if dtype == ch.CH_F32:
        t = dev(X32)
        keep.append(t)
        return ch.ch_set_create(ctx, t, 2, X32.shape[0], X32.shape[1]), X32
    if dtype == ch.CH_BF16:
        h = workloads.to_bf16_bits(X32)
        t = dev(h)
        keep.append(t)
        return ch.ch_set_create(ctx, t, 2, X32.shape[0], X32.shape[1], dtype), workloads.bf16_bits_to_f32(h)
    c, sc = workloads.to_fp8_e4m3(X32)
    t, tsc = dev(c), dev(sc)
    keep += [t, tsc]
    return ch.ch_set_create(ctx, t, 1, X32.shape[0], X32.shape[1], dtype, tsc), workloads.fp8_dequant(c, sc)


@pytest.mark.parametrize("dtype", [ch.CH_F32, ch.CH_BF16, ch.CH_FP8E4M3], ids=["f32", "bf16", "fp8"])
@pytest.mark.parametrize("n,d", [(1000, 16), (4097, 128), (333, 384), (70, 40), (129, 24), (2500, 200)])
def test_projection_keys_all_types(ctx, dtype, n, d):
    """l2 keys (projection, |x|^2 pass, scales, fingerprints) for every storage
    type against the oracle on the dequantised values: row lengths that are and
    are not multiples of 16 bytes and of one 128-byte slice, ragged tiles."""
    keep = []
    A32, B32 = workloads.gaussian_mixture(n, 300, d, n + d, clusters=5)
    sA, Ad = _typed_set(ctx, A32, dtype, keep)
    sB, Bd = _typed_set(ctx, B32, dtype, keep)
    for L, k, seed in ((10, 16, 3), (6, 8, 4), (4, 12, 5)):
        hp = ch.hash_params(L2, L, k, None, seed)
        Y = oracle.hashed(Ad, L2, seed, k)
        YB = oracle.hashed(Bd, L2, seed, k)
        assert ch.ch_top_exp(ctx, sA, sB, hp) == oracle.top_exp(Y, YB)
        keys = torch.zeros((L, n), dtype=torch.int64, device="cuda")
        ch.ch_hash_keys(ctx, sA, hp, -3, keys)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), oracle.keys(Y, -3, L, seed))
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


def test_projection_many_tiles(ctx, pair_factory):
    """More 32-row tiles than resident warps (each warp streams several tiles)."""
    A, B = workloads.gaussian_mixture(131_101, 20_000, 64, 9, clusters=40)
    p = pair_factory(A, B)
    bidx, D, lv = gpu_crude(ctx, p, L2, 6)
    r = oracle.crude_nn(A, B, L2, hash_seed=6)
    assert np.array_equal(bidx, r["bidx"]) and np.array_equal(lv, r["level"])
    assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))


@pytest.mark.parametrize("metric", [L1, L2])
def test_top_exp_matches(ctx, pair_factory, metric):
    for seed, scale in ((1, 1.0), (2, 1e-3), (3, 300.0)):
        A, B = workloads.uniform(333, 211, 7, seed)
        p = pair_factory(A * scale, B * scale + 0.5)
        hp = ch.hash_params(metric, 10, 16, None, seed)
        YA = oracle.hashed(A * scale, metric, seed, 16)
        YB = oracle.hashed(B * scale + 0.5, metric, seed, 16)
        assert ch.ch_top_exp(ctx, p.sA, p.sB, hp) == oracle.top_exp(YA, YB)


# ------------------------------------------------------------------ CrudeNN
GROUPS = [ch.CH_GROUP_HASH, ch.CH_GROUP_SORT]


@pytest.mark.parametrize("group", GROUPS, ids=["hash", "sort"])
@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("shape", ["tiny", "ragged", "dup", "one_b", "d3"])
def test_crude_nn_bit_exact(ctx, pair_factory, metric, shape, group):
    if shape == "tiny":
        A, B = workloads.uniform(2000, 2000, 16, 0)
    elif shape == "ragged":
        A, B = workloads.gaussian_mixture(1531, 977, 37, 1, clusters=11)
    elif shape == "dup":
        A, B = workloads.uniform(700, 900, 8, 2)
        B[100:800] = A
    elif shape == "one_b":
        A, B = workloads.uniform(513, 1, 5, 3)
    else:
        A, B = workloads.shape_surface(3001, 2999, 4)
    p = pair_factory(A, B)
    for seed in (0, 7):
        bidx, D, lv = gpu_crude(ctx, p, metric, seed, group=group)
        r = oracle.crude_nn(A, B, metric, hash_seed=seed)
        assert np.array_equal(bidx, r["bidx"])
        assert np.array_equal(lv, r["level"])
        assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))


@pytest.mark.parametrize("metric", [L1, L2])
def test_crude_nn_bit_exact_two_table_groups(ctx, pair_factory, metric):
    """|B| = 300k: a scale's bucket table takes 2^20 slots (16 MB), so the ten
    scales run as two groups of five under the table budget; the second group
    only probes the points the first left unresolved.  Also the size where the
    two l2 projections run side by side."""
    A, B = workloads.gaussian_mixture(40_000, 300_000, 16, 21, clusters=60)
    A[:2000] += np.float32(25.0)  # far from every cluster: resolved only at the coarse scales
    p = pair_factory(A, B)
    bidx, D, lv = gpu_crude(ctx, p, metric, 5)
    r = oracle.crude_nn(A, B, metric, hash_seed=5)
    assert np.array_equal(bidx, r["bidx"])
    assert np.array_equal(lv, r["level"])
    assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))
    assert lv.max() >= 5  # some points resolve in the second group


@pytest.mark.parametrize("top_exp,expect", [(4, "forward"), (6, "reverse")])
def test_crude_nn_later_group_forward_and_reverse(ctx, pair_factory, top_exp, expect):
    """|A| = 100k, |B| = 300k: two groups of five scales.  The first group
    resolves a number of points set by the top scale: with top_exp = 4 one point,
    leaving more than 65536 for the second group (B into its tables, as the
    first); with top_exp = 6 about 69k, leaving about 31k, so the second group
    runs in reverse (the unresolved a's buckets into small tables, B streamed past
    them).  Either way b(a), the scale and D_a equal the oracle's bit for bit."""
    A, B = workloads.uniform(100_000, 300_000, 16, 5)
    p = pair_factory(A, B)
    bidx, D, lv = gpu_crude(ctx, p, L2, 3, top_exp=top_exp)
    r = oracle.crude_nn(A, B, L2, hash_seed=3, top_exp=top_exp)
    assert np.array_equal(bidx, r["bidx"])
    assert np.array_equal(lv, r["level"])
    assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))
    left = int(np.sum(r["level"] >= 5))
    assert (left > 65536) == (expect == "forward") and left > 0


def test_crude_nn_five_groups_l1_surface(ctx, pair_factory):
    """d = 3 surfaces, l1, |B| = 600k: 32 MB tables, five groups of two scales;
    the first resolves all but a few points, the second resolves them in reverse,
    the other three return at once."""
    A, B = workloads.shape_surface(60_000, 600_000, 9)
    p = pair_factory(A, B)
    bidx, D, lv = gpu_crude(ctx, p, L1, 3)
    r = oracle.crude_nn(A, B, L1, hash_seed=3)
    assert np.array_equal(bidx, r["bidx"])
    assert np.array_equal(lv, r["level"])
    assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))
    assert 0 < int(np.sum(r["level"] >= 2)) < 100


@pytest.mark.parametrize("group", GROUPS, ids=["hash", "sort"])
def test_crude_nn_few_levels_and_fallback(ctx, pair_factory, group):
    A, B = workloads.uniform(400, 600, 6, 5)
    p = pair_factory(A, B)
    for L, top in ((1, None), (2, -8), (32, None), (5, 40)):
        bidx, D, lv = gpu_crude(ctx, p, L1, 3, L=L, top_exp=top, group=group)
        r = oracle.crude_nn(A, B, L1, hash_seed=3, L=L, top_exp=top)
        assert np.array_equal(bidx, r["bidx"]) and np.array_equal(lv, r["level"])
        assert np.array_equal(D, r["D"])


@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("k,W", [(1, 4), (3, 1), (2, 8), (4, 16), (1, 64)])
def test_kw_crude_nn_bit_exact(ctx, pair_factory, metric, k, W):
    """k x W CrudeNN (Section 3): b(a), level and D_a bit-exact against the oracle."""
    A, B = workloads.gaussian_mixture(2100, 2600, 12, 5 + k + W, clusters=8)
    B[2000:2300] = B[10:310]  # duplicates: ties by index
    p = pair_factory(A, B)
    nA = A.shape[0]
    bidx = torch.full((nA,), -5, dtype=torch.int64, device="cuda")
    D = torch.full((nA,), -1.0, dtype=torch.float32, device="cuda")
    lv = torch.full((nA,), 255, dtype=torch.uint8, device="cuda")
    hp = ch.hash_params(metric, 10, 16, None, 7, ch.CH_GROUP_HASH, W, k)
    ch.ch_crude_nn(ctx, p.sA, p.sB, hp, bidx, D, lv)
    r = oracle.crude_nn_kw(A, B, metric, hash_seed=7, k=k, W=W)
    assert np.array_equal(bidx.cpu().numpy(), r["bidx"])
    assert np.array_equal(lv.cpu().numpy(), r["level"])
    assert np.array_equal(D.cpu().numpy().view(np.uint32), r["D"].view(np.uint32))


@pytest.mark.parametrize("metric", [L1, L2])
def test_kw_estimate_matches_oracle(ctx, pair_factory, metric):
    A, B = workloads.gaussian_mixture(3000, 2000, 16, 77, clusters=5)
    p = pair_factory(A, B)
    T = 1500
    prm = ch.est_params(metric, 10, 16, None, 3, T=T, sample_seed=9, screen=ch.CH_SCREEN_EXACT, window=8, repeats=2)
    eta, rep = ch.ch_estimate(ctx, p.sA, p.sB, prm, report=True)
    r = oracle.crude_nn_kw(A, B, metric, hash_seed=3, k=2, W=8)
    w, prefix, W, _ = oracle.weights(r["D"])
    idx = oracle.draws(prefix, W, T, 9)
    m, _ = oracle.scan(A, idx, B, metric)
    eta_o = oracle.combine(m, idx, w, W)
    assert rep.W == W and abs(eta / eta_o - 1) < 1e-5
    # a wider window never raises D, so D_total does not grow
    _, rep1 = ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(metric, 10, 16, None, 3, T=T, sample_seed=9,
                                                            screen=ch.CH_SCREEN_EXACT), report=True)
    assert rep.D_total <= rep1.D_total


@pytest.mark.parametrize("K", [16, 33, 64])
def test_simhash_keys_and_crude_nn(ctx, pair_factory, K):
    """SimHash family (Section 3): keys and CrudeNN bit-exact against the oracle, on
    unit-norm data; with k x W the window rule runs on SimHash buckets."""
    A, B = workloads.unit_mixture(2500, 3000, 48, 6, clusters=40)
    p = pair_factory(A, B)
    L = 7
    hp = ch.hash_params(L2, L, K, None, 12, family=ch.CH_FAMILY_SIMHASH)
    keys = torch.zeros((L, 2500), dtype=torch.int64, device="cuda")
    ch.ch_hash_keys(ctx, p.sA, hp, 0, keys)
    want = oracle.keys_simhash(oracle.hashed(A, L2, 12, K), L, 12)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), want)
    bidx = torch.full((2500,), -5, dtype=torch.int64, device="cuda")
    D = torch.full((2500,), -1.0, dtype=torch.float32, device="cuda")
    lv = torch.full((2500,), 255, dtype=torch.uint8, device="cuda")
    ch.ch_crude_nn(ctx, p.sA, p.sB, hp, bidx, D, lv)
    r = oracle.crude_nn_simhash(A, B, L2, hash_seed=12, L=L, K=K)
    assert np.array_equal(bidx.cpu().numpy(), r["bidx"]) and np.array_equal(lv.cpu().numpy(), r["level"])
    assert np.array_equal(D.cpu().numpy().view(np.uint32), r["D"].view(np.uint32))
    eta = ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(L2, L, K, None, 12, T=2000, sample_seed=3,
                                                        screen=ch.CH_SCREEN_EXACT, family=ch.CH_FAMILY_SIMHASH))
    w, prefix, W, _ = oracle.weights(r["D"])
    idx = oracle.draws(prefix, W, 2000, 3)
    m, _ = oracle.scan(A, idx, B, L2)
    assert abs(eta / oracle.combine(m, idx, w, W) - 1) < 1e-5
    with pytest.raises(ch.ChamferError):
        ch.ch_crude_nn(ctx, p.sA, p.sB, ch.hash_params(L1, L, K, None, 12, family=ch.CH_FAMILY_SIMHASH), bidx, D, lv)


def test_sort_grouping_long_runs(ctx, pair_factory):
    """Radix-sort grouping over many tiles: runs of equal keys that cross sort
    tiles and head-scan blocks (B holds few distinct points, A many copies)."""
    rng = np.random.default_rng(11)
    base = rng.standard_normal((37, 8)).astype(np.float32)
    B = base[rng.integers(0, 37, 60_000)]
    A = np.vstack([base[rng.integers(0, 37, 30_000)], rng.standard_normal((20_000, 8)).astype(np.float32)])
    p = pair_factory(A, B)
    for metric in (L1, L2):
        bh, Dh, lh = gpu_crude(ctx, p, metric, 2)
        bs, Ds, ls = gpu_crude(ctx, p, metric, 2, group=ch.CH_GROUP_SORT)
        assert np.array_equal(bh, bs) and np.array_equal(lh, ls)
        assert np.array_equal(Dh.view(np.uint32), Ds.view(np.uint32))
        r = oracle.crude_nn(A, B, metric, hash_seed=2)
        assert np.array_equal(bs, r["bidx"]) and np.array_equal(ls, r["level"])


def test_estimate_sort_equals_hash(ctx, pair_factory):
    A, B = workloads.gaussian_mixture(5000, 7000, 24, 3, clusters=9)
    p = pair_factory(A, B)
    for metric in (L1, L2):
        e = [ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(metric, T=3000, group=g, hash_seed=1, sample_seed=2))
             for g in GROUPS]
        assert e[0] == e[1]


# ------------------------------------------------------------------ sampling
def gpu_sample(ctx, D, T, seed):
    n = D.size
    Dd = dev(D.astype(np.float32))
    idx = torch.zeros(max(T, 1), dtype=torch.int64, device="cuda")
    w = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    W = ch.ch_sample(ctx, Dd, n, T, seed, idx, w, want_total=True)
    return idx.cpu().numpy()[:T], w.cpu().numpy()[:n].view(np.uint64), W


@pytest.mark.parametrize("case", ["random", "zeros_mixed", "single", "one", "wide_range", "big"])
def test_sample_bit_exact(ctx, case):
    g = np.random.default_rng(11)
    if case == "random":
        D = g.random(5003).astype(np.float32)
    elif case == "zeros_mixed":
        D = g.random(3000).astype(np.float32)
        D[g.random(3000) < 0.4] = 0
    elif case == "single":
        D = np.zeros(777, np.float32)
        D[300] = 2.5
    elif case == "one":
        D = np.array([0.25], np.float32)
    elif case == "wide_range":
        D = (10.0 ** g.uniform(-30, 30, 4000)).astype(np.float32)
    else:
        D = g.random(300_001).astype(np.float32) * 50
    T = 4097
    idx, w, W = gpu_sample(ctx, D, T, 99)
    w_o, prefix_o, W_o, _ = oracle.weights(D)
    assert W == W_o
    assert np.array_equal(w, w_o)
    if D.size <= 5003:
        assert np.array_equal(idx, oracle.draws(prefix_o, W_o, T, 99))
    else:  # linear-search oracle: check a sample of draws by big-integer arithmetic
        for l in range(0, T, 97):
            u = oracle.philox([l, 0, 3, 0], [99, 0])
            U = int(u[0]) | int(u[1]) << 32 | int(u[2]) << 64 | int(u[3]) << 96
            t = (U * W_o) >> 128
            assert idx[l] == int(np.searchsorted(prefix_o, np.uint64(t), side="right"))


def test_sample_all_zero(ctx):
    idx, w, W = gpu_sample(ctx, np.zeros(100, np.float32), 10, 1)
    assert W == 0 and np.all(idx == -1) and np.all(w == 0)


# ------------------------------------------------------------------ scans
@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("nA,nB,d,T", [(500, 2000, 16, 777), (300, 4099, 3, 301), (200, 1500, 128, 97),
                                       (120, 700, 200, 65), (64, 333, 768, 33), (50, 123, 1, 40),
                                       (400, 3000, 40, 513), (300, 2100, 96, 257), (150, 1000, 160, 70),
                                       (40, 200, 1000, 20), (900, 5000, 64, 4100), (256, 1333, 32, 300),
                                       (333, 2500, 5, 1000)])
def test_sampled_nn_exact_bit_exact(ctx, pair_factory, metric, nA, nB, d, T):
    A, B = workloads.gaussian_mixture(nA, nB, d, nA + d, clusters=9)
    p = pair_factory(A, B)
    g = np.random.default_rng(d)
    idx = g.integers(0, nA, T).astype(np.int64)
    idx[::17] = -1
    m = torch.zeros(T, dtype=torch.float32, device="cuda")
    am = torch.zeros(T, dtype=torch.int64, device="cuda")
    ch.ch_sampled_nn(ctx, p.sA, dev(idx), T, p.sB, metric, ch.CH_SCREEN_EXACT, 8, m, am)
    m, am = m.cpu().numpy(), am.cpu().numpy()
    ok = idx >= 0
    mo, amo = oracle.scan(A, idx[ok], B, metric)
    assert np.array_equal(m[ok].view(np.uint32), mo.view(np.uint32))
    assert np.array_equal(am[ok], amo)
    assert np.all(m[~ok] == 0) and np.all(am[~ok] == -1)


@pytest.mark.parametrize("dtype", [ch.CH_F32, ch.CH_BF16, ch.CH_FP8E4M3], ids=["f32", "bf16", "fp8"])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_small_d_scan_bit_exact(ctx, dtype, d):
    """The compile-time-dimension scan (d <= 4): several sample blocks and B
    chunks, duplicated points in B (ties resolved to the smallest index)."""
    keep = []
    A32, B32 = workloads.gaussian_mixture(3000, 5000, d, 40 + d, clusters=6)
    B32[4000:4500] = B32[100:600]  # exact duplicates
    sA, Ad = _typed_set(ctx, A32, dtype, keep)
    sB, Bd = _typed_set(ctx, B32, dtype, keep)
    T = 2600
    idx = np.random.default_rng(d).integers(0, 3000, T).astype(np.int64)
    idx[5::31] = -1
    for metric in (L1, L2):
        m = torch.zeros(T, dtype=torch.float32, device="cuda")
        am = torch.zeros(T, dtype=torch.int64, device="cuda")
        ch.ch_sampled_nn(ctx, sA, dev(idx), T, sB, metric, ch.CH_SCREEN_EXACT, 8, m, am)
        m, am = m.cpu().numpy(), am.cpu().numpy()
        ok = idx >= 0
        mo, amo = oracle.scan(Ad, idx[ok], Bd, metric)
        assert np.array_equal(m[ok].view(np.uint32), mo.view(np.uint32))
        assert np.array_equal(am[ok], amo)
        assert np.all(m[~ok] == 0) and np.all(am[~ok] == -1)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


@pytest.mark.parametrize("metric", [L1, L2])
def test_exact_matches_oracle(ctx, pair_factory, metric):
    A, B = workloads.uniform(1500, 1300, 16, 21)
    p = pair_factory(A, B)
    mins = torch.zeros(1500, dtype=torch.float32, device="cuda")
    v = ch.ch_exact(ctx, p.sA, p.sB, metric, 0, mins)
    vo, mo = oracle.exact_canonical(A, B, metric)
    assert np.array_equal(mins.cpu().numpy(), mo)
    assert abs(v / vo - 1) < 1e-12
    assert abs(v / oracle.exact_fp64(A, B, metric) - 1) < 1e-5
    A3, B3 = workloads.shape_surface(2100, 1900, 5)
    p3 = pair_factory(A3, B3)
    mins3 = torch.zeros(2100, dtype=torch.float32, device="cuda")
    v3 = ch.ch_exact(ctx, p3.sA, p3.sB, metric, 0, mins3)
    vo3, mo3 = oracle.exact_canonical(A3, B3, metric)
    assert np.array_equal(mins3.cpu().numpy(), mo3) and abs(v3 / vo3 - 1) < 1e-12


# ------------------------------------------------------------------ estimate
@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("seed", [0, 1])
def test_estimate_tiny_matches_oracle(ctx, pair_factory, metric, seed):
    A, B = workloads.uniform(2000, 2000, 16, seed)
    p = pair_factory(A, B)
    prm = ch.est_params(metric, 10, 16, None, seed, eps=0.2, T=2000, sample_seed=seed + 5,
                        screen=ch.CH_SCREEN_EXACT)
    eta, rep = ch.ch_estimate(ctx, p.sA, p.sB, prm, report=True)
    eta_o, det = oracle.estimate(A, B, metric, seed, seed + 5, T=2000, details=True)
    assert abs(eta / eta_o - 1) < 1e-5
    assert rep.W == det["W"] and rep.top_exp == det["top_exp"] and rep.shift_S == det["S"]
    assert abs(rep.D_total / det["D_total"] - 1) < 1e-12
    ch_x = oracle.exact_fp64(A, B, metric)
    assert abs(eta / ch_x - 1) < 0.2


@pytest.mark.parametrize("metric", [L1, L2])
def test_uniform_estimate_matches_oracle(ctx, pair_factory, metric):
    """The uniform-sampling baseline (no CrudeNN): same draws as the oracle, eta
    within 1e-5; |A| = 1 gives that point's nearest distance."""
    A, B = workloads.gaussian_mixture(3000, 2500, 12, 31, clusters=6)
    p = pair_factory(A, B)
    for seed, T in ((0, 2000), (5, 777)):
        prm = ch.est_params(metric, T=T, sample_seed=seed, screen=ch.CH_SCREEN_EXACT,
                            sampling=ch.CH_SAMPLING_UNIFORM)
        eta, rep = ch.ch_estimate(ctx, p.sA, p.sB, prm, report=True)
        eta_o = oracle.estimate_uniform(A, B, metric, seed, T)
        assert abs(eta / eta_o - 1) < 1e-5
        assert rep.D_total == 3000.0 and rep.T == T
    s1 = ch.ch_set_create(ctx, A[:1].copy(), 0, 1, 12)
    _, mins = oracle.exact_canonical(A[:1], B, metric)
    assert ch.ch_estimate(ctx, s1, p.sB, ch.est_params(metric, T=9, sampling=ch.CH_SAMPLING_UNIFORM)) == float(mins[0])
    ch.ch_set_destroy(s1)


def test_uniform_estimate_screen_and_batch(ctx, pair_factory):
    """Uniform sampling through the TF32 screen (within 1e-5 of the oracle) and
    inside a batch (equal to the single call)."""
    A, B = workloads.gaussian_mixture(20_000, 30_000, 128, 33)
    p = pair_factory(A, B)
    prm = ch.est_params(L2, T=3000, sample_seed=8, sampling=ch.CH_SAMPLING_UNIFORM)
    eta = ch.ch_estimate(ctx, p.sA, p.sB, prm)
    assert abs(eta / oracle.estimate_uniform(A, B, L2, 8, 3000) - 1) < 1e-5
    etas, st = ch.ch_estimate_batch(ctx, [p.sA, p.sB], [p.sB, p.sA], [prm, prm])
    assert st == [ch.CH_OK, ch.CH_OK] and etas[0] == eta


@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("uniform", [False, True])
def test_symmetric_estimate_matches_oracle(ctx, pair_factory, metric, uniform):
    A, B = workloads.gaussian_mixture(2500, 1800, 10, 41, clusters=7)
    p = pair_factory(A, B)
    T = 1500
    prm = ch.est_params(metric, 10, 16, None, 3, T=T, sample_seed=4, screen=ch.CH_SCREEN_EXACT,
                        sampling=ch.CH_SAMPLING_UNIFORM if uniform else ch.CH_SAMPLING_IMPORTANCE)
    tot, ab, ba = ch.ch_estimate_sym(ctx, p.sA, p.sB, prm)
    tot_o, ab_o, ba_o = oracle.estimate_sym(A, B, metric, 3, 4, T=T, uniform=uniform)
    assert abs(ab / ab_o - 1) < 1e-5 and abs(ba / ba_o - 1) < 1e-5
    assert tot == ab + ba
    # each direction equals the one-sided estimate exactly (importance sampling
    # shares the set passes between the directions; that changes no bit)
    assert ab == ch.ch_estimate(ctx, p.sA, p.sB, prm)
    prm_ba = ch.est_params(metric, 10, 16, None, 3, T=T, sample_seed=4 ^ 0x9E3779B97F4A7C15, screen=ch.CH_SCREEN_EXACT,
                           sampling=ch.CH_SAMPLING_UNIFORM if uniform else ch.CH_SAMPLING_IMPORTANCE)
    assert ba == ch.ch_estimate(ctx, p.sB, p.sA, prm_ba)


@pytest.mark.parametrize("n_a,n_b,d", [(100_000, 100_000, 128), (60_000, 300_000, 16)])
def test_symmetric_estimate_shared_passes_large(ctx, pair_factory, n_a, n_b, d):
    """The symmetric form on the l2 path with the tensor-core screen: the 100k
    mixture (one scale group, the two projections side by side) and |B| = 300k
    (two scale groups, the second in reverse for one direction): each direction
    equals its one-sided estimate bit for bit and the oracle's within 1e-5
    (T = 400 draws per direction)."""
    A, B = workloads.gaussian_mixture(n_a, n_b, d, 43, clusters=40)
    p = pair_factory(A, B)
    prm = ch.est_params(L2, 10, 16, None, 8, T=400, sample_seed=9)
    tot, ab, ba = ch.ch_estimate_sym(ctx, p.sA, p.sB, prm)
    assert ab == ch.ch_estimate(ctx, p.sA, p.sB, prm)
    prm_ba = ch.est_params(L2, 10, 16, None, 8, T=400, sample_seed=9 ^ 0x9E3779B97F4A7C15)
    assert ba == ch.ch_estimate(ctx, p.sB, p.sA, prm_ba)
    tot_o, ab_o, ba_o = oracle.estimate_sym(A, B, L2, 8, 9, T=400)
    assert abs(ab / ab_o - 1) < 1e-5 and abs(ba / ba_o - 1) < 1e-5


def test_estimate_edge_cases(ctx, pair_factory):
    A, B = workloads.uniform(10, 20, 4, 1)
    p = pair_factory(A, B)
    # A empty -> 0
    e = np.zeros((0, 4), np.float32)
    sE = ch.ch_set_create(ctx, e, 0, 0, 4)
    assert ch.ch_estimate(ctx, sE, p.sB, ch.est_params(T=10)) == 0.0
    # B empty -> EINVAL
    with pytest.raises(ch.ChamferError) as ei:
        ch.ch_estimate(ctx, p.sA, sE, ch.est_params(T=10))
    assert ei.value.status == ch.CH_EINVAL
    ch.ch_set_destroy(sE)
    # non-finite data -> EINVAL at the next synchronising call
    bad = A.copy()
    bad[3, 2] = np.nan
    sBad = ch.ch_set_create(ctx, bad, 0, 10, 4)
    with pytest.raises(ch.ChamferError) as ei:
        ch.ch_estimate(ctx, sBad, p.sB, ch.est_params(T=10))
    assert ei.value.status == ch.CH_EINVAL
    ch.ch_set_destroy(sBad)
    # bad parameters
    with pytest.raises(ch.ChamferError):
        ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(eps=1.5))
    with pytest.raises(ch.ChamferError):
        ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(levels=0, T=5))
    # |A| = 1: eta = its nearest-neighbour distance
    s1 = ch.ch_set_create(ctx, A[:1].copy(), 0, 1, 4)
    for metric in (L1, L2):
        eta = ch.ch_estimate(ctx, s1, p.sB, ch.est_params(metric, T=7))
        _, mins = oracle.exact_canonical(A[:1], B, metric)
        assert eta == float(mins[0])
    ch.ch_set_destroy(s1)
    # subset -> exactly 0
    B2 = np.vstack([B, A])
    s2 = ch.ch_set_create(ctx, B2, 0, B2.shape[0], 4)
    assert ch.ch_estimate(ctx, p.sA, s2, ch.est_params(L2, T=50)) == 0.0
    ch.ch_set_destroy(s2)


def test_host_mode_sets_match_device_sets(ctx, pair_factory):
    A, B = workloads.uniform(900, 1100, 12, 8)
    p = pair_factory(A, B)
    sA = ch.ch_set_create(ctx, A, 0, 900, 12)
    sB = ch.ch_set_create(ctx, p.B, 1, 1100, 12)
    prm = ch.est_params(L2, T=300, hash_seed=4, sample_seed=4, screen=ch.CH_SCREEN_EXACT)
    assert ch.ch_estimate(ctx, sA, sB, prm) == ch.ch_estimate(ctx, p.sA, p.sB, prm)
    ch.ch_set_destroy(sA)
    ch.ch_set_destroy(sB)


# ------------------------------------------------------------------ mid-size workload
def test_mid_workload_sampled_parity(ctx, pair_factory):
    """The benchmark's 100k x 100k, d = 128 Gaussian-mixture l2 workload: CrudeNN
    bit-exact in full; sampled scan minima checked against the oracle on a sample."""
    A, B = workloads.gaussian_mixture(100_000, 100_000, 128, 0)
    p = pair_factory(A, B)
    bidx, D, lv = gpu_crude(ctx, p, L2, 0)
    r = oracle.crude_nn(A, B, L2, hash_seed=0)
    assert np.array_equal(bidx, r["bidx"]) and np.array_equal(lv, r["level"])
    assert np.array_equal(D.view(np.uint32), r["D"].view(np.uint32))
    T = oracle.default_T(100_000, 100_000, 0.1)
    idx, w, W = gpu_sample(ctx, D, T, 1)
    w_o, prefix_o, W_o, _ = oracle.weights(r["D"])
    assert W == W_o and np.array_equal(w, w_o)
    sub = np.arange(0, T, 23)
    assert np.array_equal(idx[sub], oracle.draws(prefix_o, W_o, T, 1)[sub])
    m = torch.zeros(T, dtype=torch.float32, device="cuda")
    ch.ch_sampled_nn(ctx, p.sA, dev(idx), T, p.sB, L2, ch.CH_SCREEN_AUTO, 8, m)
    m = m.cpu().numpy()
    mo, _ = oracle.scan(A, idx[sub], B, L2)
    assert np.array_equal(m[sub], mo)
    # the estimate against the oracle's own estimate (its own scans), over the first 512 draws
    eta = ch.ch_estimate(ctx, p.sA, p.sB, ch.est_params(L2, eps=0.1, hash_seed=0, sample_seed=1, T=512))
    eta_o = oracle.estimate(A, B, L2, 0, 1, T=512)
    assert abs(eta / eta_o - 1) < 1e-5


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_resident_embedding_changes_no_bit(ctx, pair_factory, dtype):
    """ch_set_embed keeps a set's l2 embedding resident (Appendix A.2's l2
    family under one hash seed and width): CrudeNN, the estimate, the symmetric
    form, k x W and SimHash then read it instead of projecting, with the same
    results bit for bit; other seeds still project; l1 ignores it."""
    A, B = workloads.gaussian_mixture(6000, 9000, 48, 51, clusters=9)
    if dtype == "bf16":
        A = workloads.bf16_bits_to_f32(workloads.to_bf16_bits(A))
        B = workloads.bf16_bits_to_f32(workloads.to_bf16_bits(B))
        hA, hB = workloads.to_bf16_bits(A), workloads.to_bf16_bits(B)
        sA = ch.ch_set_create(ctx, hA, 0, A.shape[0], 48, ch.CH_BF16)
        sB = ch.ch_set_create(ctx, hB, 0, B.shape[0], 48, ch.CH_BF16)
    else:
        sA = ch.ch_set_create(ctx, A, 0, A.shape[0], 48)
        sB = ch.ch_set_create(ctx, B, 0, B.shape[0], 48)
    try:
        prms = [ch.est_params(L2, 10, 16, None, 12, T=900, sample_seed=2),
                ch.est_params(L2, 10, 16, None, 12, T=900, sample_seed=2, repeats=2, window=3),
                ch.est_params(L2, 10, 16, None, 12, T=900, sample_seed=2, family=ch.CH_FAMILY_SIMHASH),
                ch.est_params(L2, 10, 16, None, 13, T=900, sample_seed=2),
                ch.est_params(L1, 10, 16, None, 12, T=900, sample_seed=2)]
        before = [ch.ch_estimate(ctx, sA, sB, p) for p in prms]
        sym_before = ch.ch_estimate_sym(ctx, sA, sB, prms[0])
        bidx0 = torch.zeros(6000, dtype=torch.int64, device="cuda")
        D0 = torch.zeros(6000, dtype=torch.float32, device="cuda")
        ch.ch_crude_nn(ctx, sA, sB, ch.hash_params(L2, 10, 16, None, 12), bidx0, D0)
        for s_ in (sA, sB):
            ch.ch_set_embed(ctx, s_, ch.hash_params(L2, 10, 16, None, 12))
            ch.ch_set_embed(ctx, s_, ch.hash_params(L1, 10, 16, None, 12))  # l1: nothing to keep
        after = [ch.ch_estimate(ctx, sA, sB, p) for p in prms]
        assert after == before
        assert ch.ch_estimate_sym(ctx, sA, sB, prms[0]) == sym_before
        bidx1 = torch.zeros(6000, dtype=torch.int64, device="cuda")
        D1 = torch.zeros(6000, dtype=torch.float32, device="cuda")
        ch.ch_crude_nn(ctx, sA, sB, ch.hash_params(L2, 10, 16, None, 12), bidx1, D1)
        assert torch.equal(bidx0, bidx1) and torch.equal(D0.view(torch.int32), D1.view(torch.int32))
        r = oracle.crude_nn(A, B, L2, hash_seed=12)
        assert np.array_equal(bidx1.cpu().numpy(), r["bidx"])
    finally:
        ch.ch_set_destroy(sA)
        ch.ch_set_destroy(sB)
