/*
 * oracle.c -- plain, slow CPU restatement of Chamfer-Estimate
 * (Bakshi, Indyk, Jayaram, Silwal, Waingarten, "A Near-Linear Time Algorithm
 * for the Chamfer Distance", 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA library; it
 * re-derives everything from the paper and from the published definitions of
 * Philox4x32-10 (Salmon et al., SC'11) and the splitmix64 finaliser.
 *
 * Floating point: IEEE binary32 / binary64, round-to-nearest-even, no FMA
 * contraction (built with -ffp-contract=off), fused multiply-add only where a
 * step says fmaf.  Every function names the passage it follows.
 *
 * Readings taken where the paper is silent (all listed in the design notes):
 *   R1 canonical distance summation order (32 strided partials + halving tree)
 *   R2 hash randomness from Philox4x32-10, 24-bit shift lattice
 *   R3 l2 Gaussian matrix as a 12-term Irwin-Hall sum, no 1/(beta k) factor
 *   R4 absolute scale exponents e_top-L+1 .. e_top from the joint bounding box
 *   R5 64-bit fingerprint of the integer grid cell, 0 reserved
 *   R6 first colliding level, minimum B index; no collision -> b=0, level=L
 *   R7 64-bit fixed-point weights, exact integer prefix
 *   R8 inverse-CDF draw from a 128-bit Philox word
 *   R9 estimate summed sequentially in binary64
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_L1 1
#define OR_L2 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw, "Parallel     */
/* random numbers: as easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64   */
/* multiplications, key bumped by the Weyl constants between rounds.         */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* splitmix64 output function (Steele, Lea, Flood 2014; Vigna's constants). */
uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
}

/* ------------------------------------------------------------------------ */
/* Distances.  d_X(a,b) is the l1 or l2 norm of a-b (Section 1).            */
/* ------------------------------------------------------------------------ */

/* R1: the canonical binary32 distance.  32 partial sums p[q] collect the   */
/* coordinates j with j mod 32 == q, in increasing j; then a halving tree   */
/* p[q] += p[q+s] for s = 16, 8, 4, 2, 1.  l1 adds |a_j-b_j|, l2 adds       */
/* (a_j-b_j)^2 with one fused multiply-add and takes sqrtf at the end.      */
float or_dist(const float* a, const float* b, int d, int metric)
{
    float p[32];
    for (int q = 0; q < 32; q++) p[q] = 0.0f;
    for (int j = 0; j < d; j++) {
        float t = a[j] - b[j];
        if (metric == OR_L1)
            p[j % 32] = p[j % 32] + fabsf(t);
        else
            p[j % 32] = fmaf(t, t, p[j % 32]);
    }
    for (int s = 16; s >= 1; s /= 2)
        for (int q = 0; q < s; q++) p[q] = p[q] + p[q + s];
    return metric == OR_L1 ? p[0] : sqrtf(p[0]);
}

/* The same distance evaluated in binary64 from the binary32 coordinates. */
double or_dist_fp64(const float* a, const float* b, int d, int metric)
{
    double s = 0.0;
    for (int j = 0; j < d; j++) {
        double t = (double)a[j] - (double)b[j];
        s += metric == OR_L1 ? fabs(t) : t * t;
    }
    return metric == OR_L1 ? s : sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Hashing at every scale (Definition "Hashing at every scale", Appendix A). */
/* ------------------------------------------------------------------------ */

/* l2 -> l1 embedding T(x)_i = sum_j Z_ij x_j (Theorem on the l2 embedding,  */
/* Appendix A.2).  R3: Z_ij is a 12-term Irwin-Hall approximation of a      */
/* standard normal built from Philox words (counters (j, i, 2, m), m<3),    */
/* summed exactly and rounded once to binary32.  The 1/(beta k) factor is   */
/* dropped: it only rescales the grid and the scales are absolute powers    */
/* of two chosen from the data.                                             */
void or_proj_matrix(uint64_t seed, int k, int d, float* G)
{
    uint32_t key[2];
    seed_key(seed, key);
    for (int i = 0; i < k; i++) {
        for (int j = 0; j < d; j++) {
            uint64_t sum = 0;
            for (uint32_t m = 0; m < 3; m++) {
                uint32_t ctr[4] = {(uint32_t)j, (uint32_t)i, 2u, m}, w[4];
                or_philox4x32_10(ctr, key, w);
                sum += (uint64_t)w[0] + w[1] + w[2] + w[3];
            }
            int64_t centred = (int64_t)sum - (int64_t)6 * 4294967296LL;
            double z = ldexp((double)centred, -32);
            G[(size_t)i * d + j] = (float)z;
        }
    }
}

/* y_i = fmaf chain over j = 0..d-1 starting from +0 (fixed order). */
void or_project(const float* X, int64_t n, int d, const float* G, int k, float* Y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        const float* x = X + (size_t)p * d;
        for (int i = 0; i < k; i++) {
            float acc = 0.0f;
            for (int j = 0; j < d; j++) acc = fmaf(G[(size_t)i * d + j], x[j], acc);
            Y[(size_t)p * k + i] = acc;
        }
    }
}

/* Randomly shifted grid of side r = 2^e (Lemma "Constructing a LSH at every */
/* scale", Appendix A.2): z ~ U[0, r)^d.  R2: z_{e,j} = U * 2^e with         */
/* U = (w0 >> 8) * 2^-24, w0 the first Philox word of counter (j, e, 1, 0).  */
float or_shift(uint64_t seed, int e, int j)
{
    uint32_t key[2], w[4];
    seed_key(seed, key);
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)e, 1u, 0u};
    or_philox4x32_10(ctr, key, w);
    return (float)ldexp((double)(w[0] >> 8), e - 24);
}

/* R5: odd 64-bit multiplier of coordinate j (Philox counter (j, 0, 4, 0)). */
uint64_t or_coord_mult(uint64_t seed, int j)
{
    uint32_t key[2], w[4];
    seed_key(seed, key);
    uint32_t ctr[4] = {(uint32_t)j, 0u, 4u, 0u};
    or_philox4x32_10(ctr, key, w);
    return (((uint64_t)w[1] << 32) | w[0]) | 1ull;
}

/* Grid cell coordinate: ceil((y_j + z_{e,j}) / 2^e), computed as           */
/* ceilf((y_j + z) * 2^-e) + 0.0f (the product by a power of two is exact;   */
/* adding +0 turns -0 into +0).                                             */
float or_cell(float y, float z, int e)
{
    float inv_r = (float)ldexp(1.0, -e);
    float s = y + z;
    float t = s * inv_r;
    return ceilf(t) + 0.0f;
}

/* R5: the bucket key of a point at scale 2^e is a 64-bit fingerprint of its */
/* integer cell vector h(y) = (c_0, ..., c_{d'-1}) and of e:                 */
/*   h   = sum_j bits(c_j) * K_j  (mod 2^64)                                 */
/*   key = mix64(h + mix64((uint32)e xor seed)), with 0 replaced by 1.       */
uint64_t or_key(const float* y, int dd, int e, uint64_t seed)
{
    uint64_t h = 0;
    for (int j = 0; j < dd; j++) {
        float c = or_cell(y[j], or_shift(seed, e, j), e);
        uint32_t bits;
        memcpy(&bits, &c, 4);
        h += (uint64_t)bits * or_coord_mult(seed, j);
    }
    uint64_t salt = or_mix64((uint64_t)(uint32_t)e ^ seed);
    uint64_t key = or_mix64(h + salt);
    return key == 0 ? 1 : key;
}

/* Keys of n points at the L scales e_lo .. e_lo+L-1, stored [L][n]. */
void or_keys(const float* Y, int64_t n, int dd, int e_lo, int L, uint64_t seed, uint64_t* keys)
{
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++)
        for (int l = 0; l < L; l++)
            keys[(size_t)l * n + p] = or_key(Y + (size_t)p * dd, dd, e_lo + l, seed);
}

/* smallest c with 2^c >= x, x > 0 */
static int ceil_log2_double(double x)
{
    int E;
    double m = frexp(x, &E); /* x = m 2^E, m in [0.5, 1) */
    return m == 0.5 ? E - 1 : E;
}

static int ceil_log2_i64(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n) c++;
    return c;
}

/* R4: scales r_i = 2^i of CrudeNN (Fig. 2, step 1) are taken as absolute    */
/* powers of two.  Delta = sum_j (max_j - min_j) over the joint bounding box */
/* of A and B in hashed space, summed in binary64 in coordinate order; the  */
/* top exponent is ceil(log2 Delta) + 1 (0 when Delta == 0).                 */
int or_top_exp(const float* YA, int64_t nA, const float* YB, int64_t nB, int dd)
{
    double delta = 0.0;
    for (int j = 0; j < dd; j++) {
        float lo = INFINITY, hi = -INFINITY;
        for (int64_t p = 0; p < nA; p++) {
            float v = YA[(size_t)p * dd + j];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        for (int64_t p = 0; p < nB; p++) {
            float v = YB[(size_t)p * dd + j];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        delta += (double)hi - (double)lo;
    }
    if (delta == 0.0) return 0;
    return ceil_log2_double(delta) + 1;
}

/* hashed representation y of a set: x itself for l1, T(x) for l2 */
static float* hashed_space(const float* X, int64_t n, int d, int metric, uint64_t seed, int k, int* dd)
{
    if (metric == OR_L1) {
        *dd = d;
        float* Y = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * d);
        memcpy(Y, X, sizeof(float) * (size_t)n * d);
        return Y;
    }
    *dd = k;
    float* G = (float*)malloc(sizeof(float) * (size_t)k * d);
    or_proj_matrix(seed, k, d, G);
    float* Y = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * k);
    or_project(X, n, d, G, k, Y);
    free(G);
    return Y;
}

/* ------------------------------------------------------------------------ */
/* CrudeNN(A, B)  (Fig. 2): for each a, the smallest scale at which some b  */
/* shares a's bucket; D_a = d(a, b).  R6: among the colliding b the one     */
/* with the smallest index; if no scale collides, b = 0 and level = L.      */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t idx; } or_entry;

static int entry_cmp(const void* x, const void* y)
{
    const or_entry* a = (const or_entry*)x;
    const or_entry* b = (const or_entry*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/* Buckets of B at each scale as sorted (key, index) lists; a walks the      */
/* scales in increasing order until its key is found (Fig. 2, step 3).      */
static void crude_from_keys(const uint64_t* kA, int64_t nA, const uint64_t* kB, int64_t nB, int L,
                            int64_t* bidx, uint8_t* level)
{
    or_entry* tab = (or_entry*)malloc(sizeof(or_entry) * (size_t)(nB > 0 ? nB : 1) * (L > 0 ? L : 1));
    for (int l = 0; l < L; l++) {
        or_entry* t = tab + (size_t)l * nB;
        for (int64_t b = 0; b < nB; b++) { t[b].key = kB[(size_t)l * nB + b]; t[b].idx = b; }
        qsort(t, (size_t)nB, sizeof(or_entry), entry_cmp);
    }
    #pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nA; a++) {
        bidx[a] = 0;
        level[a] = (uint8_t)L;
        for (int l = 0; l < L; l++) {
            const or_entry* t = tab + (size_t)l * nB;
            uint64_t k = kA[(size_t)l * nA + a];
            int64_t lo = 0, hi = nB; /* first entry with key >= k */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (t[mid].key < k) lo = mid + 1; else hi = mid;
            }
            if (lo < nB && t[lo].key == k) { /* sorted by (key, idx): first is min */
                bidx[a] = t[lo].idx;
                level[a] = (uint8_t)l;
                break;
            }
        }
    }
    free(tab);
}

/* Brute-force restatement of the same rule in O(|A| |B| L). */
static void crude_from_keys_brute(const uint64_t* kA, int64_t nA, const uint64_t* kB, int64_t nB, int L,
                                  int64_t* bidx, uint8_t* level)
{
    for (int64_t a = 0; a < nA; a++) {
        bidx[a] = 0;
        level[a] = (uint8_t)L;
        int found = 0;
        for (int l = 0; l < L && !found; l++) {
            for (int64_t b = 0; b < nB; b++) {
                if (kB[(size_t)l * nB + b] == kA[(size_t)l * nA + a]) {
                    bidx[a] = b;
                    level[a] = (uint8_t)l;
                    found = 1;
                    break;
                }
            }
        }
    }
}

/* Full CrudeNN.  top_exp_in == INT32_MIN picks the scales from the data    */
/* (R4).  brute != 0 uses the O(|A||B|L) restatement.  Returns the top      */
/* exponent used.                                                           */
int or_crude_nn(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric,
                uint64_t hash_seed, int L, int proj_dim, int top_exp_in, int brute,
                int64_t* bidx, float* D, uint8_t* level, uint64_t* keysA, uint64_t* keysB)
{
    int dd;
    float* YA = hashed_space(A, nA, d, metric, hash_seed, proj_dim, &dd);
    float* YB = hashed_space(B, nB, d, metric, hash_seed, proj_dim, &dd);
    int e_top = top_exp_in != INT32_MIN ? top_exp_in : or_top_exp(YA, nA, YB, nB, dd);
    int e_lo = e_top - L + 1;
    uint64_t* kA = keysA ? keysA : (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nA > 0 ? nA : 1) * L);
    uint64_t* kB = keysB ? keysB : (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nB > 0 ? nB : 1) * L);
    or_keys(YA, nA, dd, e_lo, L, hash_seed, kA);
    or_keys(YB, nB, dd, e_lo, L, hash_seed, kB);
    if (brute)
        crude_from_keys_brute(kA, nA, kB, nB, L, bidx, level);
    else
        crude_from_keys(kA, nA, kB, nB, L, bidx, level);
    #pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nA; a++)
        D[a] = or_dist(A + (size_t)a * d, B + (size_t)bidx[a] * d, d, metric);
    if (!keysA) free(kA);
    if (!keysB) free(kB);
    free(YA);
    free(YB);
    return e_top;
}

/* ------------------------------------------------------------------------ */
/* SimHash at every scale (the family Section 3 ran at scale on unit-norm    */
/* data: random hyperplanes, Charikar 2002).  R14: the hyperplanes are the   */
/* rows of the l2 embedding's Gaussian matrix (K = proj_dim <= 64 of them);  */
/* bit i of a point is 1 unless y_i < 0; level l (finest first) keeps the    */
/* first t_l = max(1, K >> l) bits, and its key is                           */
/* mix64(bits + mix64(((u64)l << 32) ^ seed)), 0 replaced by 1.  For a fixed */
/* level the key is a bijection of the kept bits, so keys collide exactly    */
/* when the sign prefixes agree, and a collision at one level implies one    */
/* at every coarser level.                                                  */
/* ------------------------------------------------------------------------ */
void or_keys_simhash(const float* Y, int64_t n, int K, int L, uint64_t seed, uint64_t* keys)
{
    for (int64_t p = 0; p < n; p++) {
        uint64_t word = 0;
        for (int i = 0; i < K; i++)
            if (!(Y[(size_t)p * K + i] < 0.0f)) word |= 1ull << i;
        for (int l = 0; l < L; l++) {
            int t = K >> l;
            if (t < 1) t = 1;
            const uint64_t bits = t >= 64 ? word : (word & ((1ull << t) - 1));
            uint64_t k = or_mix64(bits + or_mix64(((uint64_t)(uint32_t)l << 32) ^ seed));
            keys[(size_t)l * n + p] = k == 0 ? 1 : k;
        }
    }
}

/* CrudeNN (Fig. 2) with the SimHash family: buckets from or_keys_simhash on */
/* the embedding y = G x, then the same first-colliding-level rule (R6).     */
void or_crude_nn_simhash(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric,
                         uint64_t hash_seed, int L, int K, int64_t* bidx, float* D, uint8_t* level)
{
    int dd;
    float* YA = hashed_space(A, nA, d, OR_L2, hash_seed, K, &dd);
    float* YB = hashed_space(B, nB, d, OR_L2, hash_seed, K, &dd);
    uint64_t* kA = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nA > 0 ? nA : 1) * L);
    uint64_t* kB = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nB > 0 ? nB : 1) * L);
    or_keys_simhash(YA, nA, K, L, hash_seed, kA);
    or_keys_simhash(YB, nB, K, L, hash_seed, kB);
    crude_from_keys(kA, nA, kB, nB, L, bidx, level);
    for (int64_t a = 0; a < nA; a++) D[a] = or_dist(A + (size_t)a * d, B + (size_t)bidx[a] * d, d, metric);
    free(kA);
    free(kB);
    free(YA);
    free(YB);
}

/* ------------------------------------------------------------------------ */
/* k x W CrudeNN (Section 3, the large-scale variant): k independent hash    */
/* structures; in each, a's buckets are visited in increasing scale order    */
/* and the first W distinct points of B found there are retrieved; D_a is    */
/* the distance to the closest of all retrieved points.  R12: structure r     */
/* uses hash seed hash_seed + r * 0x9E3779B97F4A7C15 (r = 0 is Fig. 2's own   */
/* structure), its own scales (e_top of its own hashed space, unless fixed), */
/* and within a bucket the points in increasing index order; a structure     */
/* that retrieves nothing contributes B[0].  b(a) = the retrieved point at   */
/* the smallest canonical distance (smallest index on ties); level = the    */
/* finest scale at which any structure found a point (L if none).  k = W = 1 */
/* is or_crude_nn.  Brute force over B at every scale: small inputs only.    */
/* ------------------------------------------------------------------------ */
void or_crude_nn_kw(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric, uint64_t hash_seed,
                    int L, int proj_dim, int top_exp_in, int k, int W, int64_t* bidx, float* D, uint8_t* level)
{
    for (int64_t a = 0; a < nA; a++) {
        bidx[a] = -1;
        D[a] = INFINITY;
        level[a] = (uint8_t)L;
    }
    uint64_t* kA = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nA > 0 ? nA : 1) * L);
    uint64_t* kB = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nB > 0 ? nB : 1) * L);
    for (int r = 0; r < k; r++) {
        const uint64_t seed = hash_seed + (uint64_t)r * 0x9E3779B97F4A7C15ull;
        int dd;
        float* YA = hashed_space(A, nA, d, metric, seed, proj_dim, &dd);
        float* YB = hashed_space(B, nB, d, metric, seed, proj_dim, &dd);
        const int e_top = top_exp_in != INT32_MIN ? top_exp_in : or_top_exp(YA, nA, YB, nB, dd);
        or_keys(YA, nA, dd, e_top - L + 1, L, seed, kA);
        or_keys(YB, nB, dd, e_top - L + 1, L, seed, kB);
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t a = 0; a < nA; a++) {
            int64_t* taken = (int64_t*)malloc(sizeof(int64_t) * (size_t)W);
            int cnt = 0, first_level = L;
            for (int l = 0; l < L && cnt < W; l++) {
                for (int64_t b = 0; b < nB && cnt < W; b++) {
                    if (kB[(size_t)l * nB + b] != kA[(size_t)l * nA + a]) continue;
                    int seen = 0;
                    for (int t = 0; t < cnt; t++) seen |= taken[t] == b;
                    if (!seen) {
                        taken[cnt++] = b;
                        if (l < first_level) first_level = l;
                    }
                }
            }
            if (cnt == 0) taken[cnt++] = 0;
            for (int t = 0; t < cnt; t++) {
                const float v = or_dist(A + (size_t)a * d, B + (size_t)taken[t] * d, d, metric);
                if (v < D[a] || (v == D[a] && taken[t] < bidx[a])) {
                    D[a] = v;
                    bidx[a] = taken[t];
                }
            }
            if (first_level < level[a]) level[a] = (uint8_t)first_level;
            free(taken);
        }
        free(YA);
        free(YB);
    }
    free(kA);
    free(kB);
}

/* ------------------------------------------------------------------------ */
/* Importance distribution (Fig. 1, step 2): Pr[x = a] = D_a / D.           */
/* R7: w_a = ceil(D_a 2^S) as a 64-bit integer, S = 62 - ceil(log2 nA) - e_M */
/* with M = max D_a < 2^e_M; W = sum w_a < 2^63.  Returns S; W = 0 if M = 0.  */
/* ------------------------------------------------------------------------ */
int or_weights(const float* D, int64_t nA, uint64_t* w, uint64_t* prefix, uint64_t* W)
{
    float M = 0.0f;
    for (int64_t a = 0; a < nA; a++)
        if (D[a] > M) M = D[a];
    if (M == 0.0f) {
        for (int64_t a = 0; a < nA; a++) { w[a] = 0; prefix[a] = 0; }
        *W = 0;
        return 0;
    }
    int eM;
    frexp((double)M, &eM); /* M = m 2^eM, m in [0.5, 1): M < 2^eM */
    int S = 62 - ceil_log2_i64(nA) - eM;
    uint64_t run = 0;
    for (int64_t a = 0; a < nA; a++) {
        w[a] = D[a] > 0.0f ? (uint64_t)ceil(ldexp((double)D[a], S)) : 0;
        run += w[a];
        prefix[a] = run;
    }
    *W = run;
    return S;
}

/* Fig. 1, step 3: x_l ~ D, i.i.d.  R8: u = the 128-bit Philox output of     */
/* counter (l_lo, l_hi, 3, 0) (word 3 most significant), t = floor(u W / 2^128), */
/* x_l = the first a whose inclusive prefix exceeds t.                       */
void or_draws(const uint64_t* prefix, int64_t nA, uint64_t W, int64_t T, uint64_t seed, int64_t* idx)
{
    uint32_t key[2];
    seed_key(seed, key);
    for (int64_t l = 0; l < T; l++) {
        if (W == 0) { idx[l] = -1; continue; }
        uint32_t ctr[4] = {(uint32_t)l, (uint32_t)((uint64_t)l >> 32), 3u, 0u}, u[4];
        or_philox4x32_10(ctr, key, u);
        unsigned __int128 ulo = ((unsigned __int128)u[1] << 32) | u[0];
        unsigned __int128 uhi = ((unsigned __int128)u[3] << 32) | u[2];
        /* floor((uhi 2^64 + ulo) W / 2^128), exactly */
        unsigned __int128 plo = ulo * W;          /* < 2^128 */
        unsigned __int128 phi = uhi * W;          /* < 2^128 */
        unsigned __int128 mid = (phi & 0xFFFFFFFFFFFFFFFFull) + (plo >> 64);
        uint64_t t = (uint64_t)((phi >> 64) + (mid >> 64));
        int64_t a = 0;
        while (prefix[a] <= t) a++; /* linear search: obviously the first a with prefix > t */
        idx[l] = a;
    }
}

/* Fig. 1, step 3: min over all of B, by direct evaluation of the canonical */
/* distance; ties go to the smallest index.                                 */
void or_scan(const float* A, const int64_t* idx, int64_t T, const float* B, int64_t nB, int d, int metric,
             float* m, int64_t* argmin)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t l = 0; l < T; l++) {
        if (idx[l] < 0) { m[l] = 0.0f; if (argmin) argmin[l] = -1; continue; }
        const float* q = A + (size_t)idx[l] * d;
        float best = INFINITY;
        int64_t bi = 0;
        for (int64_t b = 0; b < nB; b++) {
            float v = or_dist(q, B + (size_t)b * d, d, metric);
            if (v < best) { best = v; bi = b; }
        }
        m[l] = best;
        if (argmin) argmin[l] = bi;
    }
}

/* Fig. 1, step 4: eta = (1/T) sum_l (D / D_{x_l}) min_b d(x_l, b), with the */
/* quantised weights w in place of D_a (R9: sequential binary64 sum).       */
double or_combine(const float* m, const int64_t* idx, const uint64_t* w, uint64_t W, int64_t T)
{
    if (W == 0 || T == 0) return 0.0;
    double s = 0.0;
    for (int64_t l = 0; l < T; l++)
        s += (double)m[l] * ((double)W / (double)w[idx[l]]);
    return s / (double)T;
}

/* Default sample count T = ceil(4 ln(max(nA, nB)) / eps^2) (Theorem 1: T = O(log n / eps^2)). */
int64_t or_default_T(int64_t nA, int64_t nB, double eps)
{
    int64_t n = nA > nB ? nA : nB;
    if (n < 2) n = 2;
    return (int64_t)ceil(4.0 * log((double)n) / (eps * eps));
}

typedef struct {
    double eta;
    double D_total;
    uint64_t W;
    int64_t T;
    int32_t top_exp;
    int32_t shift_S;
} or_report;

/* The uniform-sampling baseline (Section 2, before Fig. 1; the estimator the   */
/* paper compares importance sampling against): x_l uniform over A, drawn from */
/* the same Philox counter (l_lo, l_hi, 3, 0) as or_draws: x_l = floor(u nA /   */
/* 2^128), then eta = (1/T) sum_l nA m_l, summed in order in binary64.          */
void or_draws_uniform(int64_t nA, int64_t T, uint64_t seed, int64_t* idx)
{
    uint32_t key[2];
    seed_key(seed, key);
    for (int64_t l = 0; l < T; l++) {
        if (nA == 0) { idx[l] = -1; continue; }
        uint32_t ctr[4] = {(uint32_t)l, (uint32_t)((uint64_t)l >> 32), 3u, 0u}, u[4];
        or_philox4x32_10(ctr, key, u);
        unsigned __int128 ulo = ((unsigned __int128)u[1] << 32) | u[0];
        unsigned __int128 uhi = ((unsigned __int128)u[3] << 32) | u[2];
        unsigned __int128 plo = ulo * (uint64_t)nA;
        unsigned __int128 phi = uhi * (uint64_t)nA;
        unsigned __int128 mid = (phi & 0xFFFFFFFFFFFFFFFFull) + (plo >> 64);
        idx[l] = (int64_t)((phi >> 64) + (mid >> 64));
    }
}

double or_estimate_uniform(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric, int64_t T,
                           uint64_t sample_seed, int64_t* idx_out, float* m_out)
{
    if (nA == 0 || T == 0) return 0.0;
    int64_t* idx = idx_out ? idx_out : (int64_t*)malloc(sizeof(int64_t) * T);
    float* m = m_out ? m_out : (float*)malloc(sizeof(float) * T);
    or_draws_uniform(nA, T, sample_seed, idx);
    or_scan(A, idx, T, B, nB, d, metric, m, NULL);
    double s = 0.0;
    for (int64_t l = 0; l < T; l++) s += (double)m[l] * (double)nA;
    if (!idx_out) free(idx);
    if (!m_out) free(m);
    return s / (double)T;
}

/* Chamfer-Estimate(A, B, T) (Fig. 1) end to end; optional outputs may be NULL. */
double or_estimate(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric,
                   uint64_t hash_seed, int L, int proj_dim, int top_exp_in, int64_t T, uint64_t sample_seed,
                   int64_t* bidx_out, float* D_out, uint8_t* level_out, int64_t* idx_out, float* m_out,
                   or_report* rep)
{
    if (nA == 0) {
        if (rep) { memset(rep, 0, sizeof(*rep)); rep->T = T; }
        return 0.0;
    }
    int64_t* bidx = bidx_out ? bidx_out : (int64_t*)malloc(sizeof(int64_t) * nA);
    float* D = D_out ? D_out : (float*)malloc(sizeof(float) * nA);
    uint8_t* level = level_out ? level_out : (uint8_t*)malloc(nA);
    int e_top = or_crude_nn(A, nA, B, nB, d, metric, hash_seed, L, proj_dim, top_exp_in, 0, bidx, D, level,
                            NULL, NULL);
    uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * nA);
    uint64_t* prefix = (uint64_t*)malloc(sizeof(uint64_t) * nA);
    uint64_t W;
    int S = or_weights(D, nA, w, prefix, &W);
    int64_t* idx = idx_out ? idx_out : (int64_t*)malloc(sizeof(int64_t) * (T > 0 ? T : 1));
    float* m = m_out ? m_out : (float*)malloc(sizeof(float) * (T > 0 ? T : 1));
    or_draws(prefix, nA, W, T, sample_seed, idx);
    or_scan(A, idx, T, B, nB, d, metric, m, NULL);
    double eta = or_combine(m, idx, w, W, T);
    if (rep) {
        double Dt = 0.0;
        for (int64_t a = 0; a < nA; a++) Dt += D[a];
        rep->eta = eta;
        rep->D_total = Dt;
        rep->W = W;
        rep->T = T;
        rep->top_exp = e_top;
        rep->shift_S = S;
    }
    if (!bidx_out) free(bidx);
    if (!D_out) free(D);
    if (!level_out) free(level);
    if (!idx_out) free(idx);
    if (!m_out) free(m);
    free(w);
    free(prefix);
    return eta;
}

/* CH(A, B) = sum_a min_b d_X(a, b) (Section 1), every term in binary64. */
double or_exact_fp64(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric,
                     double* per_a)
{
    double total = 0.0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t a = 0; a < nA; a++) {
        double best = INFINITY;
        for (int64_t b = 0; b < nB; b++) {
            double v = or_dist_fp64(A + (size_t)a * d, B + (size_t)b * d, d, metric);
            if (v < best) best = v;
        }
        if (per_a) per_a[a] = best;
        total += best;
    }
    return total;
}

/* The same sum with every minimum taken over the canonical binary32 distance, */
/* summed sequentially in binary64 (the value an exact GPU brute force must give). */
double or_exact_canonical(const float* A, int64_t nA, const float* B, int64_t nB, int d, int metric,
                          float* per_a)
{
    float* mins = per_a ? per_a : (float*)malloc(sizeof(float) * (nA > 0 ? nA : 1));
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < nA; a++) {
        float best = INFINITY;
        for (int64_t b = 0; b < nB; b++) {
            float v = or_dist(A + (size_t)a * d, B + (size_t)b * d, d, metric);
            if (v < best) best = v;
        }
        mins[a] = best;
    }
    double total = 0.0;
    for (int64_t a = 0; a < nA; a++) total += (double)mins[a];
    if (!per_a) free(mins);
    return total;
}

/* Number of threads the OpenMP loops above use (1 without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
