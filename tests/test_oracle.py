"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every check is a published
known-answer vector, a hand-worked example, a closed form, an invariant of the
method, a special case with a textbook answer, or brute force.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2307_03043_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")
L1, L2 = oracle.L1, oracle.L2


def _hand():
    with open(os.path.join(GOLD, "hand_examples.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------- RNG primitives
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_splitmix64_published_sequence():
    want = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    s = 0
    for w in want:
        s = (s + 0x9E3779B97F4A7C15) % 2**64
        assert oracle.mix64(s) == w


# ---------------------------------------------------------------- distances
@pytest.mark.parametrize("ex", _hand()["chamfer"])
def test_exact_hand_examples(ex):
    A, B = np.array(ex["A"], np.float32), np.array(ex["B"], np.float32)
    assert oracle.exact_fp64(A, B, L1) == pytest.approx(ex["l1"], rel=1e-15)
    assert oracle.exact_fp64(A, B, L2) == pytest.approx(ex["l2"], rel=1e-15)
    v, _ = oracle.exact_canonical(A, B, L1)
    assert v == pytest.approx(ex["l1"], rel=1e-7)
    if "reverse_l1" in ex:
        assert oracle.exact_fp64(B, A, L1) == ex["reverse_l1"]


def test_canonical_tree_order_hand_example():
    h = _hand()["canonical_tree"]
    a = np.full(h["d"], h["a_rest"], np.float32)
    a[0] = h["a_first"]
    b = np.zeros(h["d"], np.float32)
    assert oracle.dist(a, b, L1) == h["l1_canonical"]
    assert oracle.dist_fp64(a, b, L1) == h["l1_exact"]


def test_distance_pythagoras_and_symmetry():
    assert oracle.dist([0, 0], [3, 4], L2) == 5.0
    assert oracle.dist([0, 0], [3, 4], L1) == 7.0
    g = np.random.default_rng(1)
    for d in (1, 3, 16, 31, 32, 33, 128, 385):
        a, b = g.standard_normal(d).astype(np.float32), g.standard_normal(d).astype(np.float32)
        for m in (L1, L2):
            assert oracle.dist(a, b, m) == oracle.dist(b, a, m)
            assert oracle.dist(a, a, m) == 0.0


@pytest.mark.parametrize("d", [1, 3, 16, 33, 128, 384])
def test_distance_within_rounding_bound_of_fp64(d):
    """|canonical - binary64| <= (d + 2) u * (sum of |terms|), u = 2^-24 (standard
    summation error bound), for both metrics."""
    g = np.random.default_rng(d)
    u = 2.0 ** -24
    for _ in range(50):
        a = (g.standard_normal(d) * 10).astype(np.float32)
        b = (g.standard_normal(d) * 10).astype(np.float32)
        c1, e1 = oracle.dist(a, b, L1), oracle.dist_fp64(a, b, L1)
        assert abs(c1 - e1) <= (d + 2) * u * e1 + 1e-30
        c2, e2 = oracle.dist(a, b, L2), oracle.dist_fp64(a, b, L2)
        assert abs(c2 * c2 - e2 * e2) <= (d + 4) * 2 * u * e2 * e2 + 1e-30


# ---------------------------------------------------------------- hash family
@pytest.mark.parametrize("case", _hand()["grid_cells"]["cases"])
def test_grid_cell_hand_examples(case):
    c = oracle.cell(case["y"], case["z"], case["e"])
    assert c == case["cell"]
    assert math.copysign(1.0, c) == 1.0 or c != 0.0


def test_shift_lattice_and_range():
    for e in (-5, 0, 3, 20):
        zs = np.array([oracle.shift(7, e, j) for j in range(4000)])
        assert np.all(zs >= 0) and np.all(zs < 2.0 ** e)
        scaled = zs * 2.0 ** (24 - e)
        assert np.all(scaled == np.floor(scaled))  # 24-bit lattice
        # uniform on [0, r): mean r/2, variance r^2/12
        assert abs(zs.mean() / 2.0 ** e - 0.5) < 4 * math.sqrt(1 / 12 / 4000)


def test_coord_multipliers_odd_and_distinct():
    ks = [oracle.coord_mult(3, j) for j in range(512)]
    assert all(k & 1 for k in ks)
    assert len(set(ks)) == 512


def test_key_equal_cells_equal_keys():
    """Points in the same grid cell share the key; reserved value 0 never appears."""
    y = np.array([0.1, 0.2, 0.3], np.float32)
    for e in (-2, 0, 4):
        zs = [oracle.shift(11, e, j) for j in range(3)]
        # move each coordinate inside its cell without crossing a boundary
        r = 2.0 ** e
        cells = [math.ceil((float(y[j]) + zs[j]) / r) for j in range(3)]
        y2 = np.array([cells[j] * r - zs[j] - r * 0.25 for j in range(3)], np.float32)
        cells2 = [oracle.cell(float(y2[j]), zs[j], e) for j in range(3)]
        assert cells2 == [float(c) for c in cells]
        assert oracle.key(y, e, 11) == oracle.key(y2, e, 11)
        assert oracle.key(y, e, 11) != 0
        assert oracle.key(y, e, 11) != oracle.key(y, e + 1, 11)


@pytest.mark.parametrize("x,y,e", [([0.0, 0.0], [0.3, 0.2], 0), ([0.0, 0.5, 1.0], [0.25, 0.25, 1.5], 1),
                                   ([1.0], [1.75], 0)])
def test_collision_probability_closed_form(x, y, e):
    """Pr[h(x) = h(y)] = prod_k max(0, 1 - |x_k - y_k| / r) (Lemma on the l1 family, App. A.2)."""
    x, y = np.array(x, np.float32), np.array(y, np.float32)
    r = 2.0 ** e
    p = float(np.prod(np.maximum(0.0, 1.0 - np.abs(x.astype(np.float64) - y) / r)))
    n = 6000
    hits = sum(oracle.key(x, e, s) == oracle.key(y, e, s) for s in range(n))
    sd = math.sqrt(max(p * (1 - p), 1e-9) / n)
    assert abs(hits / n - p) < 4.5 * sd + 1e-9
    # far points (some |x_k - y_k| > r) never collide
    far = y.copy()
    far[0] = x[0] + 1.5 * r
    assert all(oracle.key(x, e, s) != oracle.key(far, e, s) for s in range(300))


def test_gaussian_matrix_moments_and_l1_embedding():
    """Z_ij ~ N(0, 1) (Irwin-Hall reading) and E|<g, x>| = beta ||x||_2, beta = sqrt(2/pi)
    (the l2 -> l1 embedding theorem, App. A.2)."""
    G = oracle.proj_matrix(5, 256, 64).astype(np.float64)
    n = G.size
    assert abs(G.mean()) < 4 / math.sqrt(n)
    assert abs(G.var() - 1.0) < 0.04
    assert abs(np.mean(G ** 4) - 2.9) < 0.25  # Irwin-Hall(12) kurtosis 2.9
    g = np.random.default_rng(0)
    x = g.standard_normal(64)
    proj = np.abs(G @ x)
    beta = math.sqrt(2 / math.pi)
    assert abs(proj.mean() / (beta * np.linalg.norm(x)) - 1) < 0.1


def test_projection_fma_chain_close_to_fp64():
    G = oracle.proj_matrix(9, 16, 48)
    X = np.random.default_rng(2).standard_normal((30, 48)).astype(np.float32)
    Y = oracle.project(X, G)
    ref = X.astype(np.float64) @ G.astype(np.float64).T
    bound = 48 * 2.0 ** -24 * (np.abs(X).astype(np.float64) @ np.abs(G).astype(np.float64).T)
    assert np.all(np.abs(Y - ref) <= bound + 1e-30)


def test_projection_is_a_fused_chain_in_coordinate_order():
    """Reading R3 pinned by IEEE binary32 arithmetic worked by hand, with
    u = 1 + 2^-12 and v = 1 + 2^-11 (u * u = v + 2^-24, a tie between v and its
    successor that goes to the even v):
      row (-v, u) . (1, u):  acc = -v, then fma(u, u, -v) = 2^-24 exactly; rounding
        the product first, or the reverse order, gives 0;
      row (u, -v) . (u, 1):  acc = round(u * u) = v, then fma(-v, 1, v) = 0; the
        reverse order gives 2^-24;
      row (-v, u) . (u, 1):  acc = -(u v) = -(1 + 2^-11 + 2^-12 + 2^-23) exactly, then
        u - u v = -(2^-11 + 2^-23) exactly."""
    u, v = 1.0 + 2.0 ** -12, 1.0 + 2.0 ** -11
    G = np.array([[-v, u], [u, -v]], dtype=np.float32)
    y = oracle.project(np.array([[1.0, u]], dtype=np.float32), G)
    assert y[0, 0] == np.float32(2.0 ** -24)
    y2 = oracle.project(np.array([[u, 1.0]], dtype=np.float32), G)
    assert y2[0, 1] == np.float32(0.0)
    assert y2[0, 0] == np.float32(-(2.0 ** -11 + 2.0 ** -23))


@pytest.mark.parametrize("case", _hand()["top_exp"]["cases"])
def test_top_exp_hand_examples(case):
    A, B = np.array(case["A"], np.float32), np.array(case["B"], np.float32)
    assert oracle.top_exp(A, B) == case["e_top"]


# ---------------------------------------------------------------- CrudeNN
@pytest.mark.parametrize("metric", [L1, L2])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_crude_nn_bucketed_equals_brute_force(metric, seed):
    A, B = workloads.uniform(150, 170, 5, seed)
    for L in (1, 4, 10):
        r1 = oracle.crude_nn(A, B, metric, hash_seed=seed + 100, L=L, want_keys=True)
        r2 = oracle.crude_nn(A, B, metric, hash_seed=seed + 100, L=L, brute=True)
        assert np.array_equal(r1["bidx"], r2["bidx"])
        assert np.array_equal(r1["level"], r2["level"])
        assert np.array_equal(r1["D"].view(np.uint32), r2["D"].view(np.uint32))
        # b(a) is a colliding B point with the smallest index at the first colliding level
        kA, kB = r1["keysA"], r1["keysB"]
        for a in range(0, 150, 7):
            lv = r1["level"][a]
            if lv < L:
                assert kA[lv, a] == kB[lv, r1["bidx"][a]]
                assert not np.any(kB[lv, : r1["bidx"][a]] == kA[lv, a])
                assert not np.any(np.isin(kA[:lv, a], [kB[l, :] for l in range(lv)]))


@pytest.mark.parametrize("metric", [L1, L2])
def test_crude_nn_upper_bound_invariant(metric):
    """D_a >= min_b d(a, b) with probability 1 (Lemma 2, first guarantee), bitwise."""
    A, B = workloads.gaussian_mixture(400, 500, 12, 3, clusters=8)
    _, mins = oracle.exact_canonical(A, B, metric)
    for s in range(5):
        r = oracle.crude_nn(A, B, metric, hash_seed=s)
        assert np.all(r["D"] >= mins)
        assert r["D"].sum() >= mins.sum()


def test_crude_nn_single_b_and_single_scale():
    A, B = workloads.uniform(50, 1, 4, 9)
    r = oracle.crude_nn(A, B, L1, hash_seed=1)
    assert np.all(r["bidx"] == 0)
    want = [oracle.dist(a, B[0], L1) for a in A]
    assert np.array_equal(r["D"], np.array(want, np.float32))
    # one huge scale: every point shares the same cell -> b(a) = 0, level 0
    A, B = workloads.uniform(40, 60, 3, 4)
    r = oracle.crude_nn(A, B, L1, hash_seed=2, L=1, top_exp=40)
    assert np.all(r["bidx"] == 0) and np.all(r["level"] == 0)


def test_crude_nn_duplicates_collide_at_finest_scale():
    A, B = workloads.uniform(60, 80, 6, 5)
    B[10:70] = A  # every a has an exact copy in B
    r = oracle.crude_nn(A, B, L2, hash_seed=3)
    assert np.all(r["level"] == 0)
    assert oracle.exact_fp64(A, B, L2) == 0.0


def test_crude_nn_no_collision_fallback():
    """No scale collides -> b(a) = 0, level = L (reading R6)."""
    A = np.array([[0.0, 0.0]], np.float32)
    B = np.array([[1000.0, 0.0], [2000.0, 0.0]], np.float32)
    r = oracle.crude_nn(A, B, L1, hash_seed=1, L=3, top_exp=-5)
    assert r["level"][0] == 3 and r["bidx"][0] == 0
    assert r["D"][0] == 1000.0


def test_crude_quality_log_n():
    """E[D_a] <= O(log n) min_b d(a,b) (Lemma 2): lambda = D / CH stays O(log n)."""
    A, B = workloads.gaussian_mixture(1500, 1500, 16, 7, clusters=20)
    ch, _ = oracle.exact_canonical(A, B, L2)
    lam = np.mean([oracle.crude_nn(A, B, L2, hash_seed=s)["D"].sum() / ch for s in range(4)])
    assert 1.0 <= lam < 2 * math.log(3000)


# ---------------------------------------------------------------- sampling
def test_weights_hand_example():
    h = _hand()["weights"]
    w, prefix, W, S = oracle.weights(np.array(h["D"], np.float32))
    assert S == h["S"] and W == h["W"]
    assert [int(x) for x in w] == h["w"]
    assert int(prefix[-1]) == W


def test_weights_exact_rational_and_bounds():
    g = np.random.default_rng(4)
    for n in (1, 2, 3, 1000, 4097):
        D = (g.random(n) * g.choice([1e-6, 1.0, 1e6])).astype(np.float32)
        D[g.random(n) < 0.1] = 0.0
        w, prefix, W, S = oracle.weights(D)
        if D.max() == 0:
            assert W == 0
            continue
        assert W < 2**63 and W == int(np.sum(w.astype(object)))
        for a in range(0, n, max(1, n // 50)):
            exact = Fraction(float(D[a])) * Fraction(2) ** S
            assert int(w[a]) == math.ceil(exact)
            if D[a] > 0:
                assert w[a] >= 1
        # the quantised distribution is the paper's D_a / D up to tiny relative error
        p = w.astype(np.float64) / W
        q = D.astype(np.float64) / D.astype(np.float64).sum()
        big = q > 1e-6
        assert np.max(np.abs(p[big] / q[big] - 1)) < 1e-6


def test_weights_all_zero():
    w, prefix, W, S = oracle.weights(np.zeros(5, np.float32))
    assert W == 0
    assert np.all(oracle.draws(prefix, W, 10, 1) == -1)


def test_draws_exact_big_integer():
    """t = floor(u W / 2^128) checked with Python big integers; x = first a with prefix > t."""
    D = np.array([0.5, 0.0, 2.0, 1.0, 7.0], np.float32)
    w, prefix, W, _ = oracle.weights(D)
    idx = oracle.draws(prefix, W, 64, 99)
    for l in range(64):
        u = oracle.philox([l & 0xFFFFFFFF, l >> 32, 3, 0], [99, 0])
        U = int(u[0]) | int(u[1]) << 32 | int(u[2]) << 64 | int(u[3]) << 96
        t = (U * W) >> 128
        a = next(i for i in range(5) if int(prefix[i]) > t)
        assert idx[l] == a
    assert not np.any(idx == 1)  # zero weight is never drawn


def test_draws_chi_square():
    D = np.array([1, 2, 3, 4, 0, 10], np.float32)
    w, prefix, W, _ = oracle.weights(D)
    T = 60000
    idx = oracle.draws(prefix, W, T, 5)
    cnt = np.bincount(idx, minlength=6)
    p = w.astype(np.float64) / W
    nz = p > 0
    chi2 = np.sum((cnt[nz] - T * p[nz]) ** 2 / (T * p[nz]))
    assert chi2 < 20.5  # 5 degrees of freedom, p ~ 0.001
    assert cnt[4] == 0
    # uniform weights -> uniform draws; a single nonzero weight -> always drawn
    w, prefix, W, _ = oracle.weights(np.ones(8, np.float32))
    cnt = np.bincount(oracle.draws(prefix, W, 40000, 6), minlength=8)
    assert np.sum((cnt - 5000) ** 2 / 5000) < 24.3
    Dz = np.zeros(9, np.float32)
    Dz[4] = 3.0
    w, prefix, W, _ = oracle.weights(Dz)
    assert np.all(oracle.draws(prefix, W, 500, 7) == 4)


# ---------------------------------------------------------------- estimate
def test_default_T():
    for nA, nB, eps, T in _hand()["default_T"]["cases"]:
        assert oracle.default_T(nA, nB, eps) == T


def test_scan_is_canonical_minimum():
    A, B = workloads.uniform(40, 300, 17, 8)
    idx = np.arange(40, dtype=np.int64)[::-1].copy()
    for metric in (L1, L2):
        m, am = oracle.scan(A, idx, B, metric)
        _, mins = oracle.exact_canonical(A, B, metric)
        assert np.array_equal(m, mins[idx])
        for l in range(40):
            assert oracle.dist(A[idx[l]], B[am[l]], metric) == m[l]


def test_single_b_estimate_is_exact():
    """|B| = 1: D_a is the exact NN distance, so every sample returns D (Lemma 1, Var = 0)."""
    A, B = workloads.uniform(300, 1, 8, 10)
    for metric in (L1, L2):
        ch = oracle.exact_fp64(A, B, metric)
        for s in range(3):
            eta = oracle.estimate(A, B, metric, hash_seed=s, sample_seed=s, T=50)
            assert abs(eta / ch - 1) < 1e-6


def test_single_a_estimate_is_its_nn_distance():
    A, B = workloads.uniform(1, 500, 8, 11)
    for metric in (L1, L2):
        eta = oracle.estimate(A, B, metric, hash_seed=1, sample_seed=2, T=33)
        _, mins = oracle.exact_canonical(A, B, metric)
        assert eta == float(mins[0])


def test_subset_estimate_is_zero():
    A, B = workloads.uniform(80, 200, 5, 12)
    B[50:130] = A
    assert oracle.estimate(A, B, L1, hash_seed=3, sample_seed=4, T=100) == 0.0


def test_empty_a():
    A = np.zeros((0, 4), np.float32)
    B = np.ones((5, 4), np.float32)
    assert oracle.estimate(A, B, L2, 1, 1, T=10) == 0.0


def _estimates_many(A, B, metric, seeds, T, fixed_hash=None):
    """Estimator over many seeds; m_l = (per-a exact canonical NN)[x_l], which
    test_scan_is_canonical_minimum shows is what the scan returns."""
    _, mins = oracle.exact_canonical(A, B, metric)
    out = []
    for s in seeds:
        r = oracle.crude_nn(A, B, metric, hash_seed=s if fixed_hash is None else fixed_hash)
        w, prefix, W, _ = oracle.weights(r["D"])
        idx = oracle.draws(prefix, W, T, 10_000 + s)
        out.append(oracle.combine(mins[idx], idx, w, W))
    return np.array(out), r


@pytest.mark.slow
@pytest.mark.parametrize("metric", [L1, L2])
def test_unbiased_over_1000_seeds(metric):
    """E[eta] = CH (Lemma 1): mean of 1000 seeds within 1% and within 4 standard errors."""
    A, B = workloads.uniform(2000, 2000, 16, 0)
    ch = oracle.exact_fp64(A, B, metric)
    est, _ = _estimates_many(A, B, metric, range(1000), T=100)
    mean = est.mean()
    se = est.std(ddof=1) / math.sqrt(est.size)
    assert abs(mean / ch - 1) < 0.01
    assert abs(mean - ch) < 4 * se + 1e-6 * ch


@pytest.mark.slow
def test_variance_bound_lemma1():
    """Var[eta] <= CH^2 (D/CH - 1) / T for a fixed CrudeNN output (Lemma 1)."""
    A, B = workloads.gaussian_mixture(1500, 1500, 16, 2, clusters=30)
    ch_c, mins = oracle.exact_canonical(A, B, L1)
    T = 20
    est, r = _estimates_many(A, B, L1, range(600), T=T, fixed_hash=77)
    D = r["D"].astype(np.float64).sum()
    bound = ch_c ** 2 * (D / ch_c - 1) / T
    v = est.var(ddof=1)
    assert v <= bound * 1.25
    assert abs(est.mean() / ch_c - 1) < 4 * math.sqrt(bound / est.size) / ch_c + 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("metric", [L1, L2])
def test_theorem1_accuracy_tiny(metric):
    """(1 +- eps) CH in >= 99% of seeds at T = 2000, eps = 0.2 (Theorem 1)."""
    A, B = workloads.uniform(2000, 2000, 16, 1)
    ch = oracle.exact_fp64(A, B, metric)
    est, _ = _estimates_many(A, B, metric, range(200), T=2000)
    assert np.mean(np.abs(est / ch - 1) <= 0.2) >= 0.99


def test_full_estimate_matches_composed_steps():
    A, B = workloads.gaussian_mixture(300, 400, 9, 13, clusters=5)
    for metric in (L1, L2):
        eta, det = oracle.estimate(A, B, metric, hash_seed=5, sample_seed=6, T=200, details=True)
        r = oracle.crude_nn(A, B, metric, hash_seed=5)
        assert np.array_equal(r["bidx"], det["bidx"])
        w, prefix, W, _ = oracle.weights(r["D"])
        idx = oracle.draws(prefix, W, 200, 6)
        assert np.array_equal(idx, det["idx"])
        m, _ = oracle.scan(A, idx, B, metric)
        assert eta == oracle.combine(m, idx, w, W)


def test_outlier_importance_beats_uniform():
    """Outlier experiment (Section 3): importance sampling finds the far point that
    uniform sampling misses."""
    A, B = workloads.outlier_gaussian(1000, 2, 3)
    ch = oracle.exact_fp64(A, B, L1)
    T = 400
    est, _ = _estimates_many(A, B, L1, range(20), T=T)
    assert np.mean(np.abs(est / ch - 1) < 0.2) >= 0.9
    uni = np.array([oracle.estimate_uniform(A, B, L1, s, T) for s in range(20)])
    assert np.mean(np.abs(uni / ch - 1) < 0.2) < 0.5


# ------------------------------------------------------------------ uniform baseline and symmetric form
def test_uniform_draws_are_importance_draws_with_constant_weight():
    """x_l = floor(u nA / 2^128) equals the importance draw with every D_a equal
    (the weights route: w_a = 2^S, prefix (a+1) 2^S), for every l."""
    for nA, seed in ((1, 0), (7, 3), (1000, 11), (123457, 5)):
        w, prefix, W, _ = oracle.weights(np.ones(nA, np.float32))
        assert np.array_equal(oracle.draws(prefix, W, 3000, seed), oracle.draws_uniform(nA, 3000, seed))


def test_uniform_draw_frequencies():
    """Chi-square of 200k uniform draws over 10 points (p > 1e-4)."""
    from scipy import stats
    idx = oracle.draws_uniform(10, 200_000, 42)
    assert idx.min() == 0 and idx.max() == 9
    counts = np.bincount(idx, minlength=10)
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("metric", [L1, L2])
def test_uniform_estimator_unbiased(metric):
    """E[eta_unif] = sum_a min_b dist_c(a, b) exactly for the implemented draws: the
    mean over 4000 seeds lies within 5 standard errors."""
    A, B = workloads.gaussian_mixture(60, 80, 5, 9, clusters=3)
    ch_c, mins = oracle.exact_canonical(A, B, metric)
    est = np.array([oracle.estimate_uniform(A, B, metric, s, 7) for s in range(4000)])
    # the exact variance of the mean of 7 uniform draws of nA m_a
    var1 = np.var(mins.astype(np.float64) * A.shape[0])
    se = math.sqrt(var1 / 7 / est.size)
    assert abs(est.mean() - ch_c) < 5 * se
    assert abs(est.var(ddof=1) / (var1 / 7) - 1) < 0.15


def test_uniform_estimator_whole_set_and_single_point():
    A, B = workloads.uniform(50, 70, 3, 2)
    for metric in (L1, L2):
        eta, det = oracle.estimate_uniform(A, B, metric, 4, 333, details=True)
        m, _ = oracle.scan(A, det["idx"], B, metric)
        assert np.array_equal(m, det["m"])
        assert eta == sum(float(v) * 50 for v in m) / 333
        # |A| = 1: every draw is that point, eta = its nearest-neighbour distance
        _, mins = oracle.exact_canonical(A[:1], B, metric)
        assert oracle.estimate_uniform(A[:1], B, metric, 9, 17) == float(mins[0])


def test_symmetric_estimate():
    A, B = workloads.gaussian_mixture(400, 300, 6, 17, clusters=4)
    for metric in (L1, L2):
        tot, ab, ba = oracle.estimate_sym(A, B, metric, 3, 4, T=300)
        assert ab == oracle.estimate(A, B, metric, 3, 4, T=300)
        assert ba == oracle.estimate(B, A, metric, 3, 4 ^ oracle.SYM_SEED_XOR, T=300)
        assert tot == ab + ba
        # identical sets: every sample's nearest point is its copy
        assert oracle.estimate_sym(A, A.copy(), metric, 3, 4, T=50)[0] == 0.0
        assert oracle.estimate_sym(A, A.copy(), metric, 3, 4, T=50, uniform=True)[0] == 0.0


@pytest.mark.slow
def test_symmetric_estimate_unbiased():
    """Mean over 600 seeds of the symmetric estimate within 5 standard errors of
    CH(A, B) + CH(B, A) (canonical distances)."""
    A, B = workloads.gaussian_mixture(120, 90, 4, 23, clusters=3)
    for metric in (L1, L2):
        target = oracle.exact_canonical(A, B, metric)[0] + oracle.exact_canonical(B, A, metric)[0]
        est = np.array([oracle.estimate_sym(A, B, metric, s, s + 1, T=15)[0] for s in range(600)])
        assert abs(est.mean() - target) < 5 * est.std(ddof=1) / math.sqrt(est.size)


# ------------------------------------------------------------------ k x W CrudeNN (Section 3)
@pytest.mark.parametrize("metric", [L1, L2])
def test_kw_one_by_one_is_crude_nn(metric):
    A, B = workloads.gaussian_mixture(700, 900, 7, 31, clusters=6)
    for seed in (0, 5):
        r = oracle.crude_nn(A, B, metric, hash_seed=seed)
        q = oracle.crude_nn_kw(A, B, metric, hash_seed=seed, k=1, W=1)
        assert np.array_equal(r["bidx"], q["bidx"]) and np.array_equal(r["level"], q["level"])
        assert np.array_equal(r["D"].view(np.uint32), q["D"].view(np.uint32))


@pytest.mark.parametrize("metric", [L1, L2])
def test_kw_monotone_and_bounded(metric):
    """More structures or a wider window never raise D_a, and D_a never drops below
    the canonical nearest-neighbour distance (it is a distance to a point of B)."""
    A, B = workloads.gaussian_mixture(400, 500, 6, 8, clusters=4)
    _, nn = oracle.exact_canonical(A, B, metric)
    prev = None
    for k, W in ((1, 1), (1, 4), (2, 4), (4, 4), (4, 16)):
        q = oracle.crude_nn_kw(A, B, metric, hash_seed=2, k=k, W=W)
        assert np.all(q["D"] >= nn)
        for a in range(0, 400, 37):
            assert q["D"][a] == oracle.dist(A[a], B[q["bidx"][a]], metric)
        if prev is not None:
            assert np.all(q["D"] <= prev)
        prev = q["D"]


@pytest.mark.parametrize("metric", [L1, L2])
def test_kw_whole_window_is_exact(metric):
    """Scales so coarse that every point shares one bucket, and W = |B|: the window
    holds all of B, so D_a is the exact canonical minimum and b(a) its smallest argmin."""
    A, B = workloads.uniform(150, 120, 5, 6)
    B[40] = B[7]  # a duplicate: ties go to the smaller index
    q = oracle.crude_nn_kw(A, B, metric, hash_seed=1, top_exp=40, k=2, W=120)
    m, am = oracle.scan(A, np.arange(150), B, metric)
    assert np.array_equal(q["D"].view(np.uint32), m.view(np.uint32))
    assert np.array_equal(q["bidx"], am)
    assert np.all(q["level"] == 0)


def test_kw_window_restated():
    """The window rule restated in Python on tiny sets from the oracle's keys:
    per structure, buckets in scale order, points by index, first W distinct."""
    A, B = workloads.gaussian_mixture(40, 60, 3, 12, clusters=3)
    L, k, W, seed = 6, 3, 5, 9
    q = oracle.crude_nn_kw(A, B, L1, hash_seed=seed, L=L, k=k, W=W)
    best = np.full(40, np.inf, np.float32)
    arg = np.full(40, -1)
    lev = np.full(40, L)
    for r in range(k):
        s = (seed + r * 0x9E3779B97F4A7C15) % (1 << 64)
        e_lo = oracle.top_exp(A, B) - L + 1
        kA, kB = oracle.keys(A, e_lo, L, s), oracle.keys(B, e_lo, L, s)
        for a in range(40):
            taken = []
            for l in range(L):
                for b in range(60):
                    if len(taken) < W and kB[l, b] == kA[l, a] and b not in taken:
                        taken.append(b)
                        lev[a] = min(lev[a], l)
            for b in taken or [0]:
                v = oracle.dist(A[a], B[b], L1)
                if v < best[a] or (v == best[a] and b < arg[a]):
                    best[a], arg[a] = v, b
    assert np.array_equal(q["bidx"], arg) and np.array_equal(q["level"], lev)
    assert np.array_equal(q["D"], best)


# ------------------------------------------------------------------ SimHash family (Section 3)
def test_simhash_keys_are_sign_prefixes():
    """Keys agree exactly when the kept sign prefixes agree; a collision at a level
    implies one at every coarser level."""
    g = np.random.default_rng(3)
    Y = g.standard_normal((300, 16)).astype(np.float32)
    Y[100:150] = Y[:50]
    Y[150:200, :4] = Y[:50, :4]  # the same 4-bit prefix, different tails
    Y[7, 3] = 0.0                # +0 and -0 both give bit 1
    Y[8] = Y[7]
    Y[8, 3] = -0.0
    L = 6
    keys = oracle.keys_simhash(Y, L, 11)
    bits = (~(Y < 0)).astype(np.uint64)
    for l in range(L):
        t = max(1, 16 >> l)
        pref = (bits[:, :t] << np.arange(t, dtype=np.uint64)).sum(axis=1)
        same_key = keys[l][:, None] == keys[l][None, :]
        same_pref = pref[:, None] == pref[None, :]
        assert np.array_equal(same_key, same_pref)
        if l + 1 < L:
            assert np.all(~same_key | (keys[l + 1][:, None] == keys[l + 1][None, :]))
    assert np.all(keys != 0)


def test_simhash_bit_collision_probability():
    """Per hyperplane, Pr[same bit] = 1 - theta / pi for two vectors at angle theta
    (the SimHash property; the Irwin-Hall rows are nearly Gaussian): 4000 hyperplane
    draws, within 0.02."""
    d = 24
    for theta in (0.3, 1.0, 2.2):
        x = np.zeros(d, np.float32)
        x[0] = 1.0
        y = np.zeros(d, np.float32)
        y[0], y[1] = math.cos(theta), math.sin(theta)
        same = 0
        for seed in range(250):
            Y = oracle.hashed(np.stack([x, y]), L2, seed, 16)
            same += int(np.sum((Y[0] < 0) == (Y[1] < 0)))
        assert abs(same / 4000 - (1 - theta / math.pi)) < 0.02


def test_simhash_crude_nn():
    """SimHash CrudeNN: b(a) is the smallest index in the first level whose sign
    prefix matches (restated from the keys), D_a = d(a, b(a)) >= the nearest distance."""
    A, B = workloads.unit_mixture(500, 700, 12, 4)
    L, K, seed = 8, 32, 5
    r = oracle.crude_nn_simhash(A, B, L2, hash_seed=seed, L=L, K=K)
    kA = oracle.keys_simhash(oracle.hashed(A, L2, seed, K), L, seed)
    kB = oracle.keys_simhash(oracle.hashed(B, L2, seed, K), L, seed)
    _, nn = oracle.exact_canonical(A, B, L2)
    for a in range(500):
        lv, b = L, 0
        for l in range(L):
            hit = np.flatnonzero(kB[l] == kA[l, a])
            if hit.size:
                lv, b = l, int(hit[0])
                break
        assert r["level"][a] == lv and r["bidx"][a] == b
        assert r["D"][a] == oracle.dist(A[a], B[b], L2) >= nn[a]
