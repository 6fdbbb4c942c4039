/*
 * chamfer.h -- C ABI of libchamfer, a GB300 (sm_103a) implementation of
 * Chamfer-Estimate from Bakshi, Indyk, Jayaram, Silwal, Waingarten,
 * "A Near-Linear Time Algorithm for the Chamfer Distance" (2023).
 *
 * CH(A, B) = sum_{a in A} min_{b in B} d_X(a, b)   (Section 1; d_X = l1 or l2,
 * not squared).  The library estimates it in three stages, each run by CUDA
 * kernels on one GPU:
 *   CrudeNN           (Fig. 2)          ch_crude_nn
 *   importance draws  (Fig. 1, steps 2-3) ch_sample
 *   exact sampled NN  (Fig. 1, step 3)  ch_sampled_nn
 *   estimate          (Fig. 1, step 4)  ch_estimate  (all of the above)
 * plus ch_exact, the O(d |A| |B|) brute force, and ch_serve_*, a request loop.
 *
 * Conventions for every entry point:
 *  - Every call returns ch_status; nothing else crosses the ABI (no C++
 *    exceptions).  On an error the outputs are left untouched and
 *    ch_last_error(ctx) describes it.
 *  - Point sets are row-major n x d (row i at data + i*d elements).
 *  - Pointers marked "device" are CUDA device pointers on the context's device;
 *    "host" pointers are ordinary host memory.  The caller owns every buffer it
 *    passes; a set owns its device copy unless it adopted the caller's memory.
 *  - Work is issued on the context's stream.  Calls on one context are
 *    stream-ordered and NOT thread-safe; ch_serve_submit/poll/wait are.
 *  - Calls that return a host value (ch_estimate, ch_exact, ch_sample's W_total,
 *    ch_top_exp) synchronise the stream; the others are asynchronous.
 *  - Results are a pure function of (data, seeds, parameters): the same call on
 *    the same inputs gives the same bits.
 */
#ifndef CHAMFER_H
#define CHAMFER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CH_OK = 0,
    CH_EINVAL = 1,   /* invalid argument (sizes, metric, dtype, eps, non-finite data, range) */
    CH_ENOMEM = 2,   /* device or pinned-host allocation failed */
    CH_ECUDA = 3,    /* a CUDA runtime call failed */
    CH_ENOTSUP = 4,  /* combination not supported by this build */
    CH_ETIMEOUT = 5, /* a bounded device or host wait gave up */
    CH_EBUSY = 6,    /* request can never be admitted (footprint above the budget) */
    CH_EAGAIN = 7    /* result not ready yet */
} ch_status;

typedef enum { CH_L1 = 1, CH_L2 = 2 } ch_metric;

/* storage type of a point set; BF16 and FP8 values are widened to binary32
 * exactly (FP8: code value times the row's binary32 scale, one rounding). */
typedef enum { CH_F32 = 0, CH_BF16 = 1, CH_FP8E4M3 = 2 } ch_dtype;

/* How the sampled l2 scan finds min_b d(q, b):
 *  EXACT  canonical binary32 distance to every b (CUDA cores);
 *  TF32/BF16/FP8  tensor-core screen of |b|^2 - 2 q.b; per sample it keeps
 *         screened entries (4 columns of B each, scored by their best column),
 *         takes the rerank_k best entries and evaluates the canonical
 *         distance on all their columns;
 *  AUTO   TF32 for F32 sets, BF16 for BF16 sets, FP8 for FP8 sets.
 * l1 always uses the exact CUDA-core scan. */
typedef enum {
    CH_SCREEN_AUTO = 0,
    CH_SCREEN_EXACT = 1,
    CH_SCREEN_TF32 = 2,
    CH_SCREEN_BF16 = 3,
    CH_SCREEN_FP8 = 4
} ch_screen;

/* CrudeNN grouping of equal bucket keys (Fig. 2, step 3):
 *  HASH  open-addressing table of B's buckets per scale, probed by each a in
 *        increasing scale order (the structure Fig. 2 describes);
 *  SORT  device radix sort of (scale, key) with segmented minima.
 * Both give bit-identical b(a). */
typedef enum { CH_GROUP_HASH = 0, CH_GROUP_SORT = 1 } ch_group;

/* LSH family at every scale:
 *  GRID     shifted grids of side 2^e on x (l1) or on the Gaussian embedding (l2), App. A.2;
 *  SIMHASH  random hyperplanes (the family Section 3 ran at scale on unit-norm data): the
 *           signs of the proj_dim-wide Gaussian embedding, the first max(1, proj_dim >> l)
 *           of them at level l (finest first); l2 only; top_exp is ignored. */
typedef enum { CH_FAMILY_GRID = 0, CH_FAMILY_SIMHASH = 1 } ch_family;

typedef struct ch_ctx ch_ctx;
typedef struct ch_set ch_set;
typedef struct ch_server ch_server;

#define CH_TOP_EXP_AUTO INT32_MIN

/* Hash family at every scale (Definition "Hashing at every scale", App. A;
 * shifted grid for l1, Gaussian l2->l1 embedding then grid for l2, App. A.2). */
typedef struct {
    int32_t metric;     /* CH_L1 or CH_L2 */
    uint32_t levels;    /* L: number of scales 2^e, e = top_exp-L+1 .. top_exp (1..64; default 10) */
    uint32_t proj_dim;  /* l2 embedding width k (1..64; default 16); ignored for l1 */
    int32_t top_exp;    /* CH_TOP_EXP_AUTO: ceil(log2 Delta)+1 from the joint bounding box */
    uint64_t hash_seed; /* Philox key of the shifts, multipliers and Gaussian matrix */
    int32_t group;      /* ch_group */
    uint32_t window;    /* W of the k x W variant (Section 3): the first W distinct points of B in a's
                           buckets, finest scale first, by index within a bucket (0 or 1: Fig. 2's first
                           point; at most 64) */
    uint32_t repeats;   /* k of the k x W variant: independent structures, structure r keyed by
                           hash_seed + r * 0x9E3779B97F4A7C15 (0 or 1: one; at most 16); D_a is the
                           distance to the closest of all retrieved points.  k x W > 1 uses the sort
                           grouping whatever `group` says. */
    int32_t family;     /* ch_family (default GRID) */
} ch_hash_params;

/* How the samples x_l are drawn:
 *  IMPORTANCE  Pr[x = a] = D_a / D from CrudeNN's upper bounds (Fig. 1);
 *  UNIFORM     x uniform over A and eta = (|A| / T) sum_l min_b d(x_l, b): the
 *              baseline the paper measures importance sampling against (Section 2),
 *              with no CrudeNN pass.  Draws use the same Philox counters (l, 3). */
typedef enum { CH_SAMPLING_IMPORTANCE = 0, CH_SAMPLING_UNIFORM = 1 } ch_sampling;

/* Chamfer-Estimate parameters (Fig. 1). */
typedef struct {
    ch_hash_params hash;
    double eps;           /* accuracy target in (0,1); used only when T == 0 */
    int64_t T;            /* samples; 0 = ceil(4 ln(max(|A|,|B|)) / eps^2) (Theorem 1) */
    uint64_t sample_seed; /* Philox key of the draws */
    int32_t screen;       /* ch_screen */
    uint32_t rerank_k;    /* screened entries reranked per sample, 4 columns each (1..32; default 8) */
    int32_t sampling;     /* ch_sampling (default IMPORTANCE) */
} ch_est_params;

typedef struct {
    double eta;       /* the estimate */
    double D_total;   /* sum_a D_a (binary64) */
    uint64_t W;       /* total fixed-point weight */
    int64_t T;        /* samples used */
    int32_t top_exp;  /* finest..coarsest scales are 2^(top_exp-L+1) .. 2^top_exp */
    int32_t shift_S;  /* weights are ceil(D_a * 2^S) */
    float t_crude_ms, t_sample_ms, t_scan_ms, t_total_ms; /* device time per stage */
    float t_kernel_ms;  /* device time of the scan's main kernel (screen or exact scan) */
    int32_t screen;     /* ch_screen the scan actually used */
} ch_est_report;

/* Fill defaults: L1, 10 levels, k = 16, auto scales, HASH grouping, seeds 0,
 * eps 0.1, T = 0 (default), AUTO screen, rerank_k 8, importance sampling. */
void ch_default_params(ch_est_params* p);

/* ------------------------------------------------------------ context
 * ch_ctx_create: device = CUDA ordinal; stream = a cudaStream_t to issue work
 * on (borrowed, must outlive the context; cudaStreamLegacy selects the legacy
 * default stream) or NULL for a non-blocking stream the context creates.  The context owns its workspace (grow-only device arena) and a
 * pinned host page for results.  *out is set on success. */
ch_status ch_ctx_create(int device, void* stream, ch_ctx** out);
void ch_ctx_destroy(ch_ctx* ctx);
/* Last error message of this context ("" if none); valid until the next call. */
const char* ch_last_error(const ch_ctx* ctx);
/* Block until all work issued on the context's stream has finished. */
ch_status ch_ctx_sync(ch_ctx* ctx);
/* Number of CUDA kernels this process has launched through the library so far
 * (all contexts); lets callers account for device work. */
int64_t ch_kernel_launches(void);
/* Bytes currently held by the context's workspace arena. */
int64_t ch_ctx_workspace_bytes(const ch_ctx* ctx);
/* Budget of every pipeline wait inside the tensor-core screen (Fig. 1 step 3's
 * l2 scan), in SM clock cycles; 0 (the default) means about 2 s.  A wait that
 * runs out stops the kernel's work; the kernel still waits, within the default
 * bound, for every copy and tensor-core operation it issued before it frees its
 * memory, and the call returns CH_ETIMEOUT with the context still usable.  A
 * small budget turns a stalled pipeline into that error quickly.  Applies to the
 * context's later calls (and to the lanes of its batched calls).  CH_EINVAL for
 * a negative value or a NULL context. */
ch_status ch_ctx_set_wait_cycles(ch_ctx* ctx, int64_t cycles);

/* ------------------------------------------------------------ point sets
 * mode 0: data is HOST memory, copied to the device;
 * mode 1: data is DEVICE memory, copied;
 * mode 2: data is DEVICE memory, adopted without a copy (must stay valid and
 *         unchanged until ch_set_destroy; rows must be 16-byte aligned).
 * n >= 0, d >= 1; dtype ch_dtype; row_scales: n binary32 scales (FP8 only, same
 * memory kind as data, copied), NULL otherwise.  The set's own passes (bounding
 * box, |x|^2, finite check) run lazily, fused into the first call that reads
 * the set for hashing or screening; a non-finite value found there makes the
 * next synchronising call on the set (ch_estimate, ch_exact, ch_top_exp)
 * return CH_EINVAL. */
ch_status ch_set_create(ch_ctx* ctx, const void* data, int mode, int64_t n, int32_t d, int32_t dtype,
                        const float* row_scales, ch_set** out);
void ch_set_destroy(ch_set* set);
/* Runs the set's lazy passes now (bounding box, |x|^2, finite check) and
 * synchronises; CH_EINVAL if the set holds a non-finite value.  A prepared set
 * is never written again, so contexts on the same device may read it
 * concurrently (every call only requires the set to live on the context's
 * device). */
ch_status ch_set_prepare(ch_ctx* ctx, ch_set* set);
/* Keeps the set's l2 embedding under hp resident (the k = proj_dim wide Gaussian
 * projection of the hashed space, Appendix A.2's l2 family, and its bounding
 * box): every later l2 call whose hash parameters have the same hash_seed and
 * proj_dim reads it instead of projecting the set again (k x W structures other
 * than the first still project under their own seeds), with the same results
 * bit for bit.  The embedding (n * proj_dim binary32 plus its boxes) is owned by
 * the set and freed with it; a second call with other parameters replaces it.
 * Synchronises (reports non-finite data as CH_EINVAL).  For hp->metric = CH_L1
 * it does nothing: the l1 family hashes the rows themselves.  Not thread-safe
 * against calls that read the set at the same time. */
ch_status ch_set_embed(ch_ctx* ctx, ch_set* set, const ch_hash_params* hp);
int64_t ch_set_size(const ch_set* set);
int32_t ch_set_dim(const ch_set* set);

/* ------------------------------------------------------------ CrudeNN (Fig. 2)
 * Scale exponents of a pair: writes the top exponent e_top (host int32) that
 * CH_TOP_EXP_AUTO would use (synchronises). */
ch_status ch_top_exp(ch_ctx* ctx, const ch_set* A, const ch_set* B, const ch_hash_params* hp, int32_t* e_top);

/* Bucket keys of every point of X at the L scales 2^e_lo .. 2^(e_lo+L-1):
 * keys = device uint64 [L][n] (scale-major).  A key is the 64-bit fingerprint
 * of the integer grid cell ceil((y_j + z_{e,j}) / 2^e) of the point's hashed
 * coordinates y (x for l1, the Gaussian embedding for l2); two points share a
 * bucket at scale e iff their keys at e are equal (Lemma on the l1 family).
 * With the SimHash family, the keys of its L sign-prefix levels (e_lo unused). */
ch_status ch_hash_keys(ch_ctx* ctx, const ch_set* X, const ch_hash_params* hp, int32_t e_lo, uint64_t* keys);

/* For each a in A: the smallest scale at which some b in B shares a's bucket,
 * b(a) = the smallest such b index, D_a = d_X(a, b(a)) (canonical binary32).
 * If no scale collides: b(a) = 0, level = L.  Outputs (device): b_idx int64
 * [|A|], D float [|A|], level uint8 [|A|] or NULL.  |B| >= 1 required. */
ch_status ch_crude_nn(ch_ctx* ctx, const ch_set* A, const ch_set* B, const ch_hash_params* hp,
                      int64_t* b_idx, float* D, uint8_t* level);

/* ------------------------------------------------------------ sampling (Fig. 1, steps 2-3)
 * Draws T i.i.d. indices with Pr[a] = w_a / W, w_a = ceil(D_a 2^S) (64-bit
 * fixed point), S = 62 - ceil(log2 nA) - e_M with max D_a < 2^e_M; each draw is
 * the first a whose inclusive prefix of w exceeds floor(u W / 2^128), u the
 * 128-bit Philox4x32-10 output of counter (l, 3, 0) under key sample_seed.
 * D: device float [nA], all finite and >= 0.  idx: device int64 [T].  w:
 * device uint64 [nA] or NULL.  W_total: host uint64 or NULL (non-NULL
 * synchronises).  All D_a = 0 gives W = 0 and idx = -1; so does a D holding
 * +Inf or NaN (outside the contract; no weight is then meaningful). */
ch_status ch_sample(ch_ctx* ctx, const float* D, int64_t nA, int64_t T, uint64_t seed, int64_t* idx,
                    uint64_t* w, uint64_t* W_total);

/* ch_sample without any device allocation (the paper has no counterpart; this
 * is a deployment variant).  For callers that cannot allocate device memory:
 * plug-ins whose host application owns every device allocation, and processes
 * held to a device-memory budget fixed at start-up, where a cudaMalloc could
 * fail or be forbidden in the middle of a run.  It needs no context: the
 * scratch lives in one fixed ~8.4 MB device array inside the library, which
 * every GPU that loads the library holds until the process exits.
 * Same arguments and results as ch_sample, bit for bit, except: nA may be at
 * most 1,048,576 (larger returns CH_EINVAL before any work); w is required;
 * W_total is a DEVICE uint64 or NULL (no host synchronisation); stream is a
 * cudaStream_t (NULL = legacy default stream).  The array's device address is
 * looked up with the device current on the first call in each CUDA context
 * (again after cudaDeviceReset), which also loads the library's device code on
 * that device: make the first call on a device before any stream capture.
 * Every call shares the one array and the call clears what must start at zero:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race; serialise them, e.g. on one stream.  Returns CH_ECUDA if a launch
 * fails. */
ch_status ch_sample_static(const float* D, int64_t nA, int64_t T, uint64_t seed, int64_t* idx, uint64_t* w,
                           uint64_t* W_total, void* stream);

/* ------------------------------------------------------------ sampled scan (Fig. 1, step 3)
 * For each l < T: min_d[l] = min_b d_X(A[idx[l]], b) with the canonical
 * binary32 distance, argmin[l] its index (smallest on ties) -- exactly, for
 * screen EXACT; for tensor-core screens, exactly whenever the true nearest b
 * is among the columns of the rerank_k best screened entries.  idx: device int64 [T] (entries < 0
 * give min_d 0, argmin -1).  min_d: device float [T]; argmin: device int64 [T]
 * or NULL. */
ch_status ch_sampled_nn(ch_ctx* ctx, const ch_set* A, const int64_t* idx, int64_t T, const ch_set* B,
                        int32_t metric, int32_t screen, uint32_t rerank_k, float* min_d, int64_t* argmin);

/* ------------------------------------------------------------ estimate (Fig. 1)
 * eta = (1/T) sum_l min_d[l] * W / w_{x_l}, summed in binary64 on the device.
 * |A| = 0 gives eta = 0.  eta: host double.  report: host or NULL. */
ch_status ch_estimate(ch_ctx* ctx, const ch_set* A, const ch_set* B, const ch_est_params* p, double* eta,
                      ch_est_report* report);

/* ------------------------------------------------------------ many estimates
 * Estimates of count independent pairs (A[i], B[i]) under params[i], in one
 * call: the pairs are spread over a few internal streams of the context, so that
 * the kernels of small pairs overlap, and the host waits once at the end.  Not in
 * the paper (a throughput form of Fig. 1 for many small pairs).  With the exact
 * scans (l1, CH_SCREEN_EXACT) each value equals ch_estimate's bit for bit.  With
 * a tensor-core screen, B is split into chunks for one stream's share of the SMs,
 * and ch_estimate splits it for all of them.  The two can then differ only where
 * a sample's nearest point misses the R reranked entries under one split but not
 * under the other.
 * A, B: arrays of count sets of this context; params: count parameter blocks;
 * eta: host double [count] (0 for failed pairs and for |A| = 0); status: host
 * ch_status [count] or NULL.  Returns CH_OK, or the first failing pair's status
 * (that pair's eta is 0; the other pairs are still computed).  Blocks until
 * every eta is on the host.  The sets' lazy passes (|x|^2, box) run first on the
 * context's stream, so one set may appear in many pairs. */
ch_status ch_estimate_batch(ch_ctx* ctx, int64_t count, const ch_set* const* A, const ch_set* const* B,
                            const ch_est_params* params, double* eta, ch_status* status);

/* ------------------------------------------------------------ symmetric estimate
 * CH(A, B) + CH(B, A) (Section 1's symmetric Chamfer distance) as two one-sided
 * estimates under the same parameters, except that the (B, A) draws use the key
 * sample_seed ^ 0x9E3779B97F4A7C15; T = 0 gives both directions the default T of
 * max(|A|, |B|).  The two directions run concurrently (as a batch of two).
 * eta: host, the sum; eta_ab / eta_ba: host, each direction, or NULL.  Errors as
 * ch_estimate (the first failing direction's status). */
ch_status ch_estimate_sym(ch_ctx* ctx, const ch_set* A, const ch_set* B, const ch_est_params* p, double* eta,
                          double* eta_ab, double* eta_ba);

/* ------------------------------------------------------------ brute force (Section 1)
 * CH(A, B) = sum_a min_b d_X(a, b).  mode 0: canonical binary32 distance for
 * every pair (exact); mode 1: tensor-core screen + canonical rerank.
 * ch: host double (binary64 sum on the device).  per_a_min: device float [|A|]
 * or NULL. */
ch_status ch_exact(ch_ctx* ctx, const ch_set* A, const ch_set* B, int32_t metric, int32_t mode, double* ch,
                   float* per_a_min);

/* ------------------------------------------------------------ serving
 * A request loop: point sets are registered once and stay resident; requests
 * (set pairs + parameters) are admitted while their device footprint fits the
 * budget and a slot is free, and run concurrently on per-slot streams. */
typedef struct {
    int64_t hbm_budget_bytes; /* device bytes requests may hold at once (sets excluded) */
    int32_t max_slots;        /* concurrent requests on the device (1..64) */
    int32_t max_queue;        /* pending requests before submit returns CH_EAGAIN */
} ch_serve_config;

typedef struct {
    double p50_us, p99_us, mean_us; /* submit -> result latency of completed requests */
    double throughput_rps;          /* completed requests per second since creation */
    int64_t completed, failed, rejected, pending;
    int64_t peak_bytes;             /* largest admitted footprint sum */
} ch_serve_stats;

ch_status ch_serve_create(ch_ctx* ctx, const ch_serve_config* cfg, ch_server** out);
/* Makes the server an index under hp: every set registered from now on keeps
 * its l2 embedding under hp resident (ch_set_embed), so requests whose hash
 * parameters share hp's hash_seed and proj_dim skip the projection of both sets
 * (their results are the same bits as without the index).  Call it before the
 * first registration; CH_EBUSY once sets are registered, CH_EINVAL for invalid
 * hash parameters. */
ch_status ch_serve_index(ch_server* s, const ch_hash_params* hp);
/* Registers a point set (same arguments as ch_set_create); *set_id identifies it. */
ch_status ch_serve_register(ch_server* s, const void* data, int mode, int64_t n, int32_t d, int32_t dtype,
                            const float* row_scales, uint64_t* set_id);
/* Queues CH(set A, set B) with parameters p; *ticket identifies the request.
 * CH_EBUSY if its footprint exceeds the whole budget, CH_EAGAIN if the queue is full. */
ch_status ch_serve_submit(ch_server* s, uint64_t setA, uint64_t setB, const ch_est_params* p, uint64_t* ticket);
/* CH_EAGAIN while pending; CH_OK with *eta and *req_status once done. */
ch_status ch_serve_poll(ch_server* s, uint64_t ticket, double* eta, int32_t* req_status);
/* Waits at most timeout_ms; CH_ETIMEOUT if still pending. */
ch_status ch_serve_wait(ch_server* s, uint64_t ticket, uint32_t timeout_ms, double* eta, int32_t* req_status);
ch_status ch_serve_stats_get(ch_server* s, ch_serve_stats* out);
/* Starts a new measurement window: clears the latency record and the completed /
 * failed / rejected counts, and restarts the throughput clock (peak_bytes kept). */
ch_status ch_serve_stats_reset(ch_server* s);
void ch_serve_destroy(ch_server* s);

#ifdef __cplusplus
}
#endif
#endif /* CHAMFER_H */
