// api.cu -- the extern "C" entry points of libchamfer (include/chamfer.h).
//
// Host-side orchestration only: argument checks, workspace layout, kernel
// launches on the context's stream, and the single device->host copy that
// ends each synchronising call.  Every arithmetic step of the method runs in
// the kernels of k_hash.cu, k_sample.cu, k_scan.cu and k_screen.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

using namespace chx;

#include <atomic>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>

namespace chx {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void Arena::reserve(size_t bytes) {
  if (bytes <= cap) return;
  if (borrowed) throw Err{CH_ENOMEM, "lent workspace smaller than the call needs"};
  if (base) {
    CHX_CUDA(cudaDeviceSynchronize());
    CHX_CUDA(cudaFree(base));
    base = nullptr;
    cap = 0;
  }
  const size_t want = bytes + bytes / 4 + (1 << 20);
  if (cudaMalloc(&base, want) != cudaSuccess) {
    cudaGetLastError();
    base = nullptr;
    throw Err{CH_ENOMEM, "workspace allocation of " + std::to_string(want) + " bytes failed"};
  }
  cap = want;
}

void Arena::release() {
  if (base && !borrowed) cudaFree(base);
  base = nullptr;
  cap = used = 0;
}

// Two-pass layout: the same sequence of take() calls first measures, then carves.
struct Layout {
  bool measure = true;
  size_t need = 0;
  Arena* a = nullptr;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (measure) {
      need += bytes;
      return nullptr;
    }
    return a->take<T>(count);
  }
};

template <class F>
static void carve(ch_ctx* c, F&& f) {
  Layout m;
  f(m);
  c->ws.reserve(m.need + 256);
  c->ws.reset();
  Layout t;
  t.measure = false;
  t.a = &c->ws;
  f(t);
}


__global__ void k_collect(ResBlock* r, const uint32_t* sa, const uint32_t* sb, const double* out2,
                          const uint64_t* W, const int32_t* S, const int32_t* e_top) {
  pdl_entry();
  if (threadIdx.x != 0) return;
  r->statusA = sa ? *sa : 0u;
  r->statusB = sb ? *sb : 0u;
  if (out2) {
    r->eta = out2[0];
    r->D_total = out2[1];
  }
  if (W) r->W = *W;
  if (S) r->S = *S;
  if (e_top) r->e_top = *e_top;
}

// raises the error a result block's status bits stand for
static void check_result(const ResBlock* hres) {
  const uint32_t st = hres->status | hres->statusA | hres->statusB;
  if (st & ST_NONFINITE) throw Err{CH_EINVAL, "point set holds a non-finite value"};
  if (st & ST_RANGE) throw Err{CH_EINVAL, "scale exponents outside [-120, 120] (data range too large or too small)"};
  if (st & ST_BAD_INDEX) throw Err{CH_EINVAL, "sample index out of range"};
  if (st & ST_TABLE_FULL) throw Err{CH_ENOMEM, "bucket table overflow"};
  if (st & ST_TIMEOUT) throw Err{CH_ETIMEOUT, "a bounded device wait gave up"};
}

static void finish(ch_ctx* c, ResBlock* dres, ResBlock* hres) {
  CHX_CUDA(cudaMemcpyAsync(hres, dres, sizeof(ResBlock), cudaMemcpyDeviceToHost, c->stream));
  CHX_CUDA(cudaStreamSynchronize(c->stream));
  check_result(hres);
}

static void check_hash(const ch_hash_params* hp) {
  CHX_CHECK(hp, CH_EINVAL, "hash params NULL");
  CHX_CHECK(hp->metric == CH_L1 || hp->metric == CH_L2, CH_EINVAL, "metric must be CH_L1 or CH_L2");
  CHX_CHECK(hp->levels >= 1 && hp->levels <= uint32_t(kMaxLevels), CH_EINVAL, "levels must be in 1..32");
  if (hp->metric == CH_L2)
    CHX_CHECK(hp->proj_dim >= 1 && hp->proj_dim <= uint32_t(kMaxProj), CH_EINVAL, "proj_dim must be in 1..64");
  CHX_CHECK(hp->group == CH_GROUP_HASH || hp->group == CH_GROUP_SORT, CH_EINVAL, "group must be HASH or SORT");
  CHX_CHECK(hp->window <= uint32_t(kWindowMax), CH_EINVAL, "window must be in 0..64 (0 = 1)");
  CHX_CHECK(hp->repeats <= 16u, CH_EINVAL, "repeats must be in 0..16 (0 = 1)");
  CHX_CHECK(hp->family == CH_FAMILY_GRID || hp->family == CH_FAMILY_SIMHASH, CH_EINVAL, "unknown family");
  CHX_CHECK(hp->family != CH_FAMILY_SIMHASH || hp->metric == CH_L2, CH_EINVAL, "SimHash hashes the l2 embedding");
}

static void check_pair(ch_ctx* c, const ch_set* A, const ch_set* B) {
  CHX_CHECK(A && B, CH_EINVAL, "set NULL");
  CHX_CHECK(A->ctx->device == c->device && B->ctx->device == c->device, CH_EINVAL,
            "sets live on another device");
  CHX_CHECK(A->d == B->d, CH_EINVAL, "sets differ in dimension");
  CHX_CHECK(A->dtype == B->dtype, CH_EINVAL, "sets differ in storage type");
  CHX_CHECK(B->n >= 1, CH_EINVAL, "B must hold at least one point");
}

// hashed space of a set under hp: the set's own rows (l1) or its l2 embedding
struct Hashed {
  HashSrc src;
  const uint32_t* box;  // [box_parts][2][dd] partial boxes of the hashed space
  int box_parts;
  float* Y;        // l2 embedding (+ Gaussian matrix tail) in the workspace
  uint32_t* boxY;  // l2 partial boxes in the workspace
};

static int proj_pad(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64; }

// k x W CrudeNN (Section 3's large-scale variant) is asked for
static bool crude_kw(const ch_hash_params* hp) { return hp->window > 1 || hp->repeats > 1; }

// the set's resident embedding serves hp (made by ch_set_embed under the same seed and width)
static bool resident_hashed(const ch_set* X, const ch_hash_params* hp) {
  return hp->metric == CH_L2 && X->hs.valid && X->hs.seed == hp->hash_seed && X->hs.k == static_cast<int>(hp->proj_dim);
}

template <class L>
static void take_hashed(L& lay, const ch_set* X, const ch_hash_params* hp, Hashed* h) {
  if (hp->metric == CH_L1) {
    h->src = HashSrc{X->data, X->dtype, X->n, X->d, X->scales};
    h->box = X->box_x;
    h->box_parts = 1;
    h->Y = nullptr;
    h->boxY = nullptr;
  } else {
    const int k = static_cast<int>(hp->proj_dim);
    // no buffers where the set's resident embedding serves every pass of the call
    // (k x W structures other than the first project under their own seeds)
    const bool resident = resident_hashed(X, hp) && !crude_kw(hp);
    h->Y = resident ? nullptr : lay.template take<float>(size_t(X->n) * k + 4 + size_t(proj_pad(k)) * X->d);
    h->boxY = resident ? nullptr : lay.template take<uint32_t>(size_t(2) * k * kMaxBoxParts);
    h->src = HashSrc{h->Y, CH_F32, X->n, k, nullptr};
    h->box = h->boxY;
    h->box_parts = 1;  // set by the projection
  }
}

// the hashed space's pass over a set: the l2 projection (which also yields
// |x|^2 and the finite check) or, for l1, the ingest pass (box of x)
// The hashed space h reads: the set's resident embedding where it serves hp,
// else the workspace buffers h->Y / h->boxY (which stay the call's own, so a
// later pass under another seed never writes into the resident one).
static void run_hashed(ch_ctx* c, const ch_set* X, const ch_hash_params* hp, Hashed* h, uint32_t* status) {
  if (resident_hashed(X, hp)) {
    h->src = HashSrc{X->hs.Y, CH_F32, X->n, X->hs.k, nullptr};
    h->box = X->hs.box;
    h->box_parts = X->hs.parts;
  } else if (hp->metric == CH_L2) {
    h->src = HashSrc{h->Y, CH_F32, X->n, static_cast<int>(hp->proj_dim), nullptr};
    h->box = h->boxY;
    h->box_parts = launch_project(X, hp->hash_seed, static_cast<int>(hp->proj_dim), h->Y, h->boxY, status,
                                  c->sm_count, c->stream);
  } else {
    ensure_ingest(const_cast<ch_set*>(X), c->stream);
  }
}

// the context's side stream and its fork / join events, made on first use
static void ensure_side(ch_ctx* c) {
  if (c->side) return;
  CHX_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CHX_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
  CHX_CUDA(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
}

// Both sets' hashed-space passes.  Where each l2 projection is bound by its
// start-up (generating the Gaussian matrix, filling the copy pipeline: sets of
// 2M to 64M coordinates) the two run side by side, A's on the context's stream
// and B's on its side stream, each on half of the SMs, so that the start-ups
// overlap (100k x 128 fp32: 8 us less per estimate).  Smaller sets would pay
// more for the fork and join than they save (4096 pairs of d = 3 surfaces:
// 162 -> 264 ms), larger ones gain nothing.
static void run_hashed_pair(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_hash_params* hp, Hashed* hA,
                            Hashed* hB, uint32_t* status) {
  const int64_t wA = A->n * A->d, wB = B->n * B->d;
  const bool side_by_side = std::min(wA, wB) >= (int64_t(1) << 21) && std::max(wA, wB) <= (int64_t(1) << 26);
  if (hp->metric != CH_L2 || c->sm_count < 2 || !side_by_side || resident_hashed(A, hp) || resident_hashed(B, hp)) {
    run_hashed(c, A, hp, hA, status);
    run_hashed(c, B, hp, hB, status);
    return;
  }
  ensure_side(c);
  const int k = static_cast<int>(hp->proj_dim);
  hA->src = HashSrc{hA->Y, CH_F32, A->n, k, nullptr};
  hA->box = hA->boxY;
  hB->src = HashSrc{hB->Y, CH_F32, B->n, k, nullptr};
  hB->box = hB->boxY;
  const int half = c->sm_count / 2;
  CHX_CUDA(cudaEventRecord(c->fork_ev, c->stream));
  CHX_CUDA(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
  hA->box_parts = launch_project(A, hp->hash_seed, k, hA->Y, hA->boxY, status, half, c->stream);
  hB->box_parts = launch_project(B, hp->hash_seed, k, hB->Y, hB->boxY, status, c->sm_count - half, c->side);
  CHX_CUDA(cudaEventRecord(c->join_ev, c->side));
  CHX_CUDA(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
}

template <class L>
static ScaleTables take_tables(L& lay, int dd, int L_) {
  ScaleTables t;
  t.e_lo = lay.template take<int32_t>(1);
  t.inv_r = lay.template take<float>(L_);
  t.salt = lay.template take<uint64_t>(L_);
  t.shift = lay.template take<float>(size_t(dd) * L_);
  t.mult = lay.template take<uint64_t>(dd);
  return t;
}

// bucket-table plan: one table of 2^log_cap 16-byte slots per scale, load <= 1/2,
// scales grouped so that a group's tables stay L2-resident
// bytes of bucket tables kept live at once (a group of scales): measured on the
// 1M-point workload, 80 MB (two 32 MB scales per pass) beat 48 MB (one) and 112 MB
static size_t table_budget() { return size_t(80) << 20; }

struct TablePlan {
  uint32_t log_cap;
  int per_group;
};
// A scale group after the first runs in reverse (the unresolved a's buckets into
// small tables, B streamed past them once) once at most this many points of A
// are left: 1M x 384 unit mixture, 46k points left after the first two scales.
constexpr int64_t kRevMax = int64_t(1) << 16;

static TablePlan table_plan(int64_t nB, int L) {
  TablePlan p;
  p.log_cap = static_cast<uint32_t>(ceil_log2_i64(std::max<int64_t>(2 * nB, 1024)));
  const size_t per_level = (size_t(1) << p.log_cap) * 16;
  const size_t budget = table_budget();
  p.per_group = static_cast<int>(std::max<size_t>(1, std::min<size_t>(L, budget / per_level)));
  return p;
}

struct CrudeBufs {
  Hashed hA, hB;
  ScaleTables tab;
  int32_t* e_top;
  ulonglong2* slots;   // CH_GROUP_HASH: bucket tables of one scale group
  // CH_GROUP_HASH scale-group control: left[0] = points of A no scale group has
  // resolved yet; mode[g] = group g's mode
  unsigned long long* left;
  int32_t* mode;
  int groups;
  // reverse groups (g >= 1, once at most rev_max points are left): small tables
  // [groups - 1][per_group][2^rev_log_cap]
  unsigned long long rev_max;
  uint32_t rev_log_cap;
  ulonglong2* rev;
  TablePlan plan;
  uint64_t *keysA, *keysB;  // CH_GROUP_SORT and k x W: keys [L][n] and the sort's scratch
  void* sort_work;
  int32_t* cand;  // k x W: [nA][k W] candidate indices
};

static int kw_k(const ch_hash_params* hp) { return hp->repeats ? static_cast<int>(hp->repeats) : 1; }
static int kw_w(const ch_hash_params* hp) { return hp->window ? static_cast<int>(hp->window) : 1; }
// hash seed of structure r (r = 0: the base structure)
static uint64_t kw_seed(uint64_t seed, int r) { return seed + uint64_t(r) * 0x9E3779B97F4A7C15ull; }

template <class L>
static void take_crude(L& lay, const ch_set* A, const ch_set* B, const ch_hash_params* hp, CrudeBufs* cb) {
  take_hashed(lay, A, hp, &cb->hA);
  take_hashed(lay, B, hp, &cb->hB);
  const int dd = hp->metric == CH_L1 ? A->d : static_cast<int>(hp->proj_dim);
  cb->tab = take_tables(lay, dd, static_cast<int>(hp->levels));
  cb->e_top = lay.template take<int32_t>(1);
  const int nl = static_cast<int>(hp->levels);
  cb->cand = nullptr;
  if (crude_kw(hp)) {
    CHX_CHECK(sort_group_supported(A->n, B->n, nl), CH_EINVAL, "k x W CrudeNN: (nA + nB) * levels must be below 2^31");
    cb->plan = TablePlan{0, 0};
    cb->slots = nullptr;
    cb->keysA = lay.template take<uint64_t>(std::max<size_t>(size_t(nl) * A->n, 1));
    cb->keysB = lay.template take<uint64_t>(size_t(nl) * B->n);
    cb->sort_work = lay.template take<char>(sort_window_workspace(A->n, B->n, nl));
    cb->cand = lay.template take<int32_t>(std::max<size_t>(size_t(A->n) * kw_k(hp) * kw_w(hp), 1));
    return;
  }
  if (hp->group == CH_GROUP_SORT || hp->family == CH_FAMILY_SIMHASH) {
    CHX_CHECK(sort_group_supported(A->n, B->n, nl), CH_EINVAL, "sort grouping: (nA + nB) * levels must be below 2^31");
    cb->plan = TablePlan{0, 0};
    cb->slots = nullptr;
    cb->keysA = lay.template take<uint64_t>(std::max<size_t>(size_t(nl) * A->n, 1));
    cb->keysB = lay.template take<uint64_t>(size_t(nl) * B->n);
    cb->sort_work = lay.template take<char>(sort_group_workspace(A->n, B->n, nl));
    return;
  }
  cb->plan = table_plan(B->n, nl);
  cb->slots = lay.template take<ulonglong2>(size_t(cb->plan.per_group) << cb->plan.log_cap);
  cb->groups = (nl + cb->plan.per_group - 1) / cb->plan.per_group;
  cb->left = lay.template take<unsigned long long>(1);
  cb->mode = lay.template take<int32_t>(cb->groups);
  // reverse groups need rows of at most 32 hashed values, at most kRevGroupMax
  // scales per group and more than one group
  cb->rev_max = (cb->groups > 1 && dd <= 32 && cb->plan.per_group <= kRevGroupMax)
                    ? static_cast<unsigned long long>(std::min<int64_t>(kRevMax, A->n))
                    : 0;
  cb->rev = nullptr;
  cb->rev_log_cap = 0;
  if (cb->rev_max) {
    cb->rev_log_cap = static_cast<uint32_t>(ceil_log2_i64(std::max<int64_t>(2 * int64_t(cb->rev_max), 1024)));
    cb->rev = lay.template take<ulonglong2>((size_t(cb->groups - 1) * cb->plan.per_group) << cb->rev_log_cap);
  }
  cb->keysA = cb->keysB = nullptr;
  cb->sort_work = nullptr;
}

// keys [L][n] of both sets into cb->keysA / keysB after their hashed passes: the
// grid family's scales and cells, or SimHash's sign prefixes (no scales)
static void bucket_keys(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_hash_params* hp, CrudeBufs* cb,
                        bool report_top, uint32_t* status) {
  const int L = static_cast<int>(hp->levels);
  cudaStream_t s = c->stream;
  if (hp->family == CH_FAMILY_SIMHASH) {
    const int K = static_cast<int>(hp->proj_dim);
    if (report_top) CHX_CUDA(cudaMemsetAsync(cb->e_top, 0, sizeof(int32_t), s));  // no scales: reported as 0
    launch_simhash_keys(static_cast<const float*>(cb->hB.src.base), B->n, K, L, hp->hash_seed, cb->keysB, s);
    launch_simhash_keys(static_cast<const float*>(cb->hA.src.base), A->n, K, L, hp->hash_seed, cb->keysA, s);
    return;
  }
  const int dd = hp->metric == CH_L1 ? A->d : static_cast<int>(hp->proj_dim);
  launch_scale_tables(cb->hA.box, cb->hA.box_parts, cb->hB.box, cb->hB.box_parts, dd, L, hp->top_exp, hp->hash_seed,
                      cb->tab, report_top ? cb->e_top : nullptr, status, s);
  launch_keys_write(cb->hB.src, L, cb->tab, cb->keysB, s);
  launch_keys_write(cb->hA.src, L, cb->tab, cb->keysA, s);
}

// CrudeNN (Fig. 2): embedding, scales, per-scale bucket tables of B, probes of A,
// then D_a = d(a, b(a)).
// With hashed_ready, cb->hA / hB already hold both sets' hashed spaces (the other
// direction of a symmetric estimate made them) and the set passes are skipped.
static void run_crude(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_hash_params* hp, CrudeBufs* cb,
                      int64_t* bidx, uint8_t* level, float* D, uint32_t* status, uint32_t* maxD = nullptr,
                      bool hashed_ready = false) {
  const int L = static_cast<int>(hp->levels);
  const int dd = hp->metric == CH_L1 ? A->d : static_cast<int>(hp->proj_dim);
  cudaStream_t s = c->stream;
  if (crude_kw(hp)) {
    // k structures in turn (own embedding seed, scales, keys), each adding its
    // window to the candidate lists; then D_a over all candidates
    const int k = kw_k(hp), W = kw_w(hp);
    for (int r = 0; r < k; ++r) {
      ch_hash_params hr = *hp;
      hr.hash_seed = kw_seed(hp->hash_seed, r);
      run_hashed(c, A, &hr, &cb->hA, status);
      run_hashed(c, B, &hr, &cb->hB, status);
      bucket_keys(c, A, B, &hr, cb, r == 0, status);
      launch_sort_window(cb->keysA, A->n, cb->keysB, B->n, L, W, r, cb->sort_work, cb->cand, k * W, level, s);
    }
    launch_cand_dist(A, B, hp->metric, cb->cand, k * W, bidx, D, maxD, s);
    return;
  }
  if (!hashed_ready) run_hashed_pair(c, A, B, hp, &cb->hA, &cb->hB, status);
  if (hp->group == CH_GROUP_SORT || hp->family == CH_FAMILY_SIMHASH) {
    bucket_keys(c, A, B, hp, cb, true, status);
    launch_sort_group(cb->keysA, A->n, cb->keysB, B->n, L, cb->sort_work, bidx, level, s);
    launch_crude_dist(A, B, hp->metric, bidx, D, maxD, c->sm_count, s);
    return;
  }
  // Small tables (one group of at most 48 MB, well inside L2) are cleared by the
  // launch that builds the scale tables, beside its work (100k x 128: CrudeNN
  // 0.117 -> 0.112 ms).  Larger ones are cleared by the driver's memset, which
  // was faster there (1M x 384: 1.38 vs 1.45 ms with the clearing in the kernel).
  const size_t cap = size_t(1) << cb->plan.log_cap;
  const size_t group_bytes0 = size_t(std::min(cb->plan.per_group, L)) * cap * sizeof(ulonglong2);
  const bool fold = group_bytes0 <= (size_t(48) << 20) && L <= cb->plan.per_group;
  // the launch that builds the scale tables also clears the single small group's
  // tables, or else the reverse groups' small tables
  void* zero = fold ? static_cast<void*>(cb->slots) : static_cast<void*>(cb->rev);
  const size_t zero_bytes = fold ? group_bytes0
                                 : cb->rev ? ((size_t(cb->groups - 1) * cb->plan.per_group) << cb->rev_log_cap) * 16 : 0;
  launch_scale_tables(cb->hA.box, cb->hA.box_parts, cb->hB.box, cb->hB.box_parts, dd, L, hp->top_exp, hp->hash_seed,
                      cb->tab, cb->e_top, status, s, zero, zero_bytes, c->sm_count, cb->left, A->n, 0);
  // Each group's kernels follow its mode (see HashTable): groups after the one
  // that resolves the last point of A return at once -- on clustered data the
  // coarse scales are rarely reached (1M x 384 unit mixture: no point past scale
  // 4 of 10) -- and once few points are left a group runs in reverse.  The crude
  // distances follow the last group in one pass over A.  (Running those of the
  // first group's points on a side stream beside the later groups was faster
  // with a distance kernel of four memory round trips per row; with the whole
  // row in flight the single pass is faster: 1M x 384 bf16, four hash seeds,
  // CrudeNN 1.06-1.28 -> 0.97-1.06 ms.)
  for (int g = 0, L0 = 0; L0 < L; ++g, L0 += cb->plan.per_group) {
    const int nl = std::min(cb->plan.per_group, L - L0);
    HashTable h{};
    h.slots = cb->slots;
    h.log_cap = cb->plan.log_cap;
    h.left = cb->left;
    h.mode = cb->mode;
    h.group = g;
    h.first = 1;
    if (g > 0 && cb->rev_max) {
      h.rev_max = cb->rev_max;
      h.rev_log_cap = cb->rev_log_cap;
      h.rev = cb->rev + ((size_t(g - 1) * cb->plan.per_group) << cb->rev_log_cap);
      launch_group_reverse(cb->hA.src, cb->hB.src, L, L0, nl, cb->tab, h, bidx, level, status, c->sm_count, s);
      h.first = 0;
    }
    if (!fold) {
      launch_table_clear(h, nl, c->sm_count, s);
      h.first = 0;
    }
    launch_group_insert(cb->hB.src, L, L0, nl, cb->tab, h, status, c->sm_count, s);
    h.first = 0;
    launch_group_probe(cb->hA.src, L, L0, nl, cb->tab, h, bidx, level, c->sm_count, s);
  }
  launch_crude_dist(A, B, hp->metric, bidx, D, maxD, c->sm_count, s);
}

struct SampleBufs {
  SampleWork sw;
  uint64_t* prefix;
};

template <class L>
static void take_sample(L& lay, int64_t nA, SampleBufs* sb) {
  sb->sw.maxD = lay.template take<uint32_t>(1);
  sb->sw.blocksum = lay.template take<uint64_t>(std::max<size_t>(sample_blocks(nA), 1));
  sb->sw.W = lay.template take<uint64_t>(1);
  sb->sw.S = lay.template take<int32_t>(1);
  sb->prefix = lay.template take<uint64_t>(std::max<int64_t>(nA, 1));
}

static int screen_choice(int screen, int metric, const ch_set* A, const ch_set* B) {
  if (metric == CH_L1) return CH_SCREEN_EXACT;
  if (screen == CH_SCREEN_AUTO)
    screen = A->dtype == CH_F32 ? CH_SCREEN_TF32 : A->dtype == CH_BF16 ? CH_SCREEN_BF16 : CH_SCREEN_FP8;
  if (screen != CH_SCREEN_EXACT && !screen_supported(screen, A, B)) screen = CH_SCREEN_EXACT;
  return screen;
}

struct ScanBufs {
  ScanPart part;
  void* screen_work;
  int screen;
};

template <class L>
static void take_scan(L& lay, ch_ctx* c, const ch_set* A, const ch_set* B, int64_t T, int metric, int screen,
                      uint32_t R, ScanBufs* sb) {
  sb->screen = screen_choice(screen, metric, A, B);
  if (sb->screen == CH_SCREEN_EXACT) {
    sb->part.chunks = scan_exact_chunks(T, B->n, A->d, A->dtype, c->sm_count);
    sb->part.val = lay.template take<float>(size_t(sb->part.chunks) * std::max<int64_t>(T, 1));
    sb->part.idx = lay.template take<int64_t>(size_t(sb->part.chunks) * std::max<int64_t>(T, 1));
    sb->screen_work = nullptr;
  } else {
    sb->part = ScanPart{nullptr, nullptr, 0};
    sb->screen_work =
        lay.template take<char>(screen_workspace(T, B->n, A->d, static_cast<int>(R), c->sm_count,
                                                 c->screen_chunk_sms, sb->screen));
  }
}

static void run_scan(ch_ctx* c, const ch_set* A, const int64_t* idx, int64_t T, const ch_set* B, int metric,
                     uint32_t R, ScanBufs* sb, float* m, int64_t* argmin, uint32_t* status,
                     const KernelTimer& timer = KernelTimer()) {
  if (T == 0) return;
  if (sb->screen == CH_SCREEN_EXACT) {
    timer.start(c->stream);
    launch_scan_exact(A, idx, T, B, metric, sb->part, c->sm_count, c->stream);
    timer.stop(c->stream);
    launch_scan_merge(sb->part, T, idx, m, argmin, c->stream);
  } else {
    ensure_norms(const_cast<ch_set*>(B), c->stream);
    launch_screen_l2(A, idx, T, B, sb->screen, static_cast<int>(R), sb->screen_work, m, argmin, status, c->sm_count,
                     c->screen_chunk_sms, c->stream, timer, c->wait_cycles);
  }
}

int64_t default_T(int64_t nA, int64_t nB, double eps) {
  int64_t n = std::max<int64_t>(std::max(nA, nB), 2);
  return static_cast<int64_t>(std::ceil(4.0 * std::log(static_cast<double>(n)) / (eps * eps)));
}

// every workspace buffer of one ch_estimate call
struct EstBufs {
  CrudeBufs cb;
  SampleBufs sb;
  ScanBufs sc;
  ResBlock* res = nullptr;
  int64_t *bidx = nullptr, *idx = nullptr;
  uint8_t* level = nullptr;
  float *D = nullptr, *m = nullptr;
  uint64_t* w = nullptr;
  double* out2 = nullptr;
};

template <class L>
static void take_estimate(L& lay, ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, int64_t T,
                          uint32_t R, EstBufs* eb) {
  const int64_t nA = A->n;
  eb->res = lay.template take<ResBlock>(1);
  eb->out2 = lay.template take<double>(kCombineDoubles);
  take_crude(lay, A, B, &p->hash, &eb->cb);
  eb->bidx = lay.template take<int64_t>(nA);
  eb->level = lay.template take<uint8_t>(nA);
  eb->D = lay.template take<float>(nA);
  take_sample(lay, nA, &eb->sb);
  eb->w = lay.template take<uint64_t>(nA);
  eb->idx = lay.template take<int64_t>(std::max<int64_t>(T, 1));
  eb->m = lay.template take<float>(std::max<int64_t>(T, 1));
  take_scan(lay, c, A, B, T, p->hash.metric, p->screen, R, &eb->sc);
}

// device workspace bytes ch_estimate(A, B, p) needs on a context like c
size_t estimate_footprint(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p) {
  const uint32_t R = p->rerank_k ? p->rerank_k : 8;
  const int64_t T = p->T > 0 ? p->T : default_T(A->n, B->n, p->eps);
  Layout m;
  EstBufs eb;
  take_estimate(m, c, A, B, p, T, R, &eb);
  return m.need + 256;
}

static ch_status fail(ch_ctx* c, const Err& e) {
  if (c) c->err = e.msg;
  return e.st;
}

}  // namespace chx

#define CHX_GUARD_BEGIN(ctxp) \
  ch_ctx* ctx_ = (ctxp);      \
  try {
#define CHX_GUARD_END                                  \
  }                                                    \
  catch (const ::chx::Err& e) {                        \
    return ::chx::fail(ctx_, e);                       \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    return ::chx::fail(ctx_, {CH_ENOMEM, "host allocation failed"}); \
  }                                                    \
  catch (...) {                                        \
    return ::chx::fail(ctx_, {CH_ECUDA, "unexpected internal error"}); \
  }

extern "C" {

int64_t ch_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void ch_default_params(ch_est_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->hash.metric = CH_L1;
  p->hash.levels = 10;
  p->hash.proj_dim = 16;
  p->hash.top_exp = CH_TOP_EXP_AUTO;
  p->hash.hash_seed = 0;
  p->hash.group = CH_GROUP_HASH;
  p->eps = 0.1;
  p->T = 0;
  p->sample_seed = 0;
  p->screen = CH_SCREEN_AUTO;
  p->rerank_k = 8;
}

ch_status ch_ctx_create(int device, void* stream, ch_ctx** out) {
  if (!out) return CH_EINVAL;
  ch_ctx* c = new (std::nothrow) ch_ctx();
  if (!c) return CH_ENOMEM;
  CHX_GUARD_BEGIN(c)
  int ndev = 0;
  CHX_CUDA(cudaGetDeviceCount(&ndev));
  CHX_CHECK(device >= 0 && device < ndev, CH_EINVAL, "no such CUDA device");
  c->device = device;
  CHX_CUDA(cudaSetDevice(device));
  CHX_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    CHX_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  CHX_CUDA(cudaMallocHost(&c->host_pin, 4096));
  {
    // sets come and go per request: a private pool that keeps freed memory
    // (release threshold = max) makes their allocation a stream-ordered reuse
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    CHX_CUDA(cudaMemPoolCreate(&c->pool, &props));
    uint64_t keep = ~uint64_t(0);
    CHX_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  for (auto& e : c->ev) CHX_CUDA(cudaEventCreate(&e));
  *out = c;
  return CH_OK;
  }
  catch (const ::chx::Err& e) {
    ch_ctx_destroy(c);
    return e.st;
  }
  catch (...) {
    ch_ctx_destroy(c);
    return CH_ECUDA;
  }
}

void ch_ctx_destroy(ch_ctx* c) {
  if (!c) return;
  for (ch_ctx* l : c->lanes) ch_ctx_destroy(l);
  c->lanes.clear();
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->batch_pin) cudaFreeHost(c->batch_pin);
  c->ws.release();
  if (c->pool) cudaMemPoolDestroy(c->pool);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->host_pin) cudaFreeHost(c->host_pin);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* ch_last_error(const ch_ctx* c) { return c ? c->err.c_str() : "null context"; }

ch_status ch_ctx_sync(ch_ctx* c) {
  if (!c) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CUDA(cudaSetDevice(c->device));
  CHX_CUDA(cudaStreamSynchronize(c->stream));
  return CH_OK;
  CHX_GUARD_END
}

int64_t ch_ctx_workspace_bytes(const ch_ctx* c) { return c ? static_cast<int64_t>(c->ws.cap) : 0; }

ch_status ch_ctx_set_wait_cycles(ch_ctx* c, int64_t cycles) {
  if (!c) return CH_EINVAL;
  if (cycles < 0) {
    c->err = "wait budget must be >= 0";
    return CH_EINVAL;
  }
  c->wait_cycles = cycles;
  return CH_OK;
}

ch_status ch_set_create(ch_ctx* c, const void* data, int mode, int64_t n, int32_t d, int32_t dtype,
                        const float* row_scales, ch_set** out) {
  if (!c || !out) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CHECK(n >= 0, CH_EINVAL, "n must be >= 0");
  CHX_CHECK(d >= 1 && d <= kMaxDim, CH_EINVAL, "d must be in 1..4096");
  CHX_CHECK(dtype == CH_F32 || dtype == CH_BF16 || dtype == CH_FP8E4M3, CH_EINVAL, "unknown dtype");
  CHX_CHECK(mode >= 0 && mode <= 2, CH_EINVAL, "mode must be 0, 1 or 2");
  CHX_CHECK(n == 0 || data, CH_EINVAL, "data NULL");
  CHX_CHECK(dtype != CH_FP8E4M3 || n == 0 || row_scales, CH_EINVAL, "FP8 sets need row scales");
  CHX_CUDA(cudaSetDevice(c->device));
  ch_set* X = new ch_set();
  X->ctx = c;
  X->n = n;
  X->d = d;
  X->dtype = dtype;
  const size_t bytes = size_t(n) * d * elem_size(dtype);
  cudaStream_t s = c->stream;
  try {
    if (mode == 2) {
      CHX_CHECK((reinterpret_cast<uintptr_t>(data) & 15) == 0, CH_EINVAL, "adopted data must be 16-byte aligned");
      X->data = const_cast<void*>(data);
      X->owned = false;
    } else {
      CHX_CUDA(cudaMallocFromPoolAsync(&X->data, std::max<size_t>(bytes, 16), c->pool, s));
      X->owned = true;
      if (bytes)
        CHX_CUDA(cudaMemcpyAsync(X->data, data, bytes, mode == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                 s));
    }
    // aux: norms [n], status, box [2d], scales [n]
    const size_t nb = (size_t(n) * 4 + 255) & ~size_t(255);
    const size_t bb = (size_t(2) * d * 4 + 255) & ~size_t(255);
    const size_t sb = dtype == CH_FP8E4M3 ? nb : 0;
    char* aux = nullptr;
    CHX_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&aux), nb + 256 + bb + sb, c->pool, s));
    X->norms = reinterpret_cast<float*>(aux);
    X->status = reinterpret_cast<uint32_t*>(aux + nb);
    X->box_x = reinterpret_cast<uint32_t*>(aux + nb + 256);
    if (sb) {
      X->scales = reinterpret_cast<float*>(aux + nb + 256 + bb);
      if (n)
        CHX_CUDA(cudaMemcpyAsync(X->scales, row_scales, size_t(n) * 4,
                                 mode == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    }
    CHX_CUDA(cudaMemsetAsync(X->status, 0, 4, s));
    // the set's passes (bounding box, |x|^2 and the finite check) run lazily with
    // the first call that needs them, fused with that call's own read of the set
  } catch (...) {
    ch_set_destroy(X);
    throw;
  }
  *out = X;
  return CH_OK;
  CHX_GUARD_END
}

void ch_set_destroy(ch_set* X) {
  if (!X) return;
  ch_ctx* c = X->ctx;
  cudaSetDevice(c->device);
  if (X->owned && X->data) cudaFreeAsync(X->data, c->stream);
  if (X->norms) cudaFreeAsync(X->norms, c->stream);
  if (X->hs.Y) cudaFreeAsync(X->hs.Y, c->stream);
  delete X;
}

ch_status ch_set_embed(ch_ctx* c, ch_set* X, const ch_hash_params* hp) {
  if (!c || !X || !hp) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_hash(hp);
  CHX_CHECK(X->ctx->device == c->device, CH_EINVAL, "set lives on another device");
  if (hp->metric != CH_L2) return CH_OK;  // l1 hashes the rows themselves; their box is cached with the set
  if (resident_hashed(X, hp)) return CH_OK;
  CHX_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int k = static_cast<int>(hp->proj_dim);
  // the projection's layout: [n][k] plus the width-padded Gaussian-matrix tail, then the partial boxes
  const size_t ybytes = ((size_t(X->n) * k + 4 + size_t(proj_pad(k)) * X->d) * 4 + 255) & ~size_t(255);
  const size_t bbytes = size_t(2) * k * kMaxBoxParts * 4;
  char* mem = nullptr;
  CHX_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&mem), ybytes + bbytes, c->pool, s));
  if (X->hs.Y) CHX_CUDA(cudaFreeAsync(X->hs.Y, s));  // an embedding under other parameters
  X->hs.valid = false;
  X->hs.Y = reinterpret_cast<float*>(mem);
  X->hs.box = reinterpret_cast<uint32_t*>(mem + ybytes);
  ResBlock* res = nullptr;
  carve(c, [&](auto& lay) { res = lay.template take<ResBlock>(1); });
  CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
  X->hs.parts = launch_project(X, hp->hash_seed, k, X->hs.Y, X->hs.box, &res->status, c->sm_count, s);
  launch_k(k_collect, 1, 32, 0, s, res, X->status, nullptr, nullptr, nullptr, nullptr, nullptr);
  launch_check("collect");
  finish(c, res, static_cast<ResBlock*>(c->host_pin));
  X->hs.seed = hp->hash_seed;
  X->hs.k = k;
  X->hs.valid = true;
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_set_prepare(ch_ctx* c, ch_set* X) {
  if (!c || !X) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CHECK(X->ctx->device == c->device, CH_EINVAL, "set lives on another device");
  CHX_CUDA(cudaSetDevice(c->device));
  ResBlock* res = nullptr;
  carve(c, [&](auto& lay) { res = lay.template take<ResBlock>(1); });
  cudaStream_t s = c->stream;
  CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
  ensure_ingest(X, s);
  ensure_norms(X, s);
  launch_k(k_collect, 1, 32, 0, s, res, X->status, nullptr, nullptr, nullptr, nullptr, nullptr);
  launch_check("collect");
  finish(c, res, static_cast<ResBlock*>(c->host_pin));
  return CH_OK;
  CHX_GUARD_END
}

int64_t ch_set_size(const ch_set* X) { return X ? X->n : -1; }
int32_t ch_set_dim(const ch_set* X) { return X ? X->d : -1; }

ch_status ch_top_exp(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_hash_params* hp, int32_t* e_top) {
  if (!c || !e_top) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_hash(hp);
  check_pair(c, A, B);
  CHX_CUDA(cudaSetDevice(c->device));
  Hashed hA, hB;
  ScaleTables tab;
  ResBlock* res = nullptr;
  const int dd = hp->metric == CH_L1 ? A->d : static_cast<int>(hp->proj_dim);
  int32_t* et = nullptr;
  carve(c, [&](auto& lay) {
    res = lay.template take<ResBlock>(1);
    take_hashed(lay, A, hp, &hA);
    take_hashed(lay, B, hp, &hB);
    tab = take_tables(lay, dd, static_cast<int>(hp->levels));
    et = lay.template take<int32_t>(1);
  });
  cudaStream_t s = c->stream;
  CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
  run_hashed(c, A, hp, &hA, &res->status);
  run_hashed(c, B, hp, &hB, &res->status);
  launch_scale_tables(hA.box, hA.box_parts, hB.box, hB.box_parts, dd, static_cast<int>(hp->levels), hp->top_exp,
                      hp->hash_seed, tab, et,
                      &res->status, s);
  launch_k(k_collect, 1, 32, 0, s, res, A->status, B->status, nullptr, nullptr, nullptr, et);
  launch_check("collect");
  ResBlock* h = static_cast<ResBlock*>(c->host_pin);
  finish(c, res, h);
  *e_top = h->e_top;
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_hash_keys(ch_ctx* c, const ch_set* X, const ch_hash_params* hp, int32_t e_lo, uint64_t* keys) {
  if (!c || !X || !keys) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_hash(hp);
  CHX_CHECK(X->ctx == c, CH_EINVAL, "set belongs to another context");
  const int L = static_cast<int>(hp->levels);
  CHX_CHECK(e_lo >= -120 && e_lo + L - 1 <= 120, CH_EINVAL, "scale exponents outside [-120, 120]");
  CHX_CUDA(cudaSetDevice(c->device));
  Hashed h;
  ScaleTables tab;
  uint32_t* st = nullptr;
  const int dd = hp->metric == CH_L1 ? X->d : static_cast<int>(hp->proj_dim);
  carve(c, [&](auto& lay) {
    st = lay.template take<uint32_t>(1);
    take_hashed(lay, X, hp, &h);
    tab = take_tables(lay, dd, L);
  });
  cudaStream_t s = c->stream;
  CHX_CUDA(cudaMemsetAsync(st, 0, 4, s));
  run_hashed(c, X, hp, &h, st);
  if (hp->family == CH_FAMILY_SIMHASH) {  // sign prefixes; e_lo does not apply
    launch_simhash_keys(h.Y, X->n, static_cast<int>(hp->proj_dim), L, hp->hash_seed, keys, s);
    return CH_OK;
  }
  launch_scale_tables(h.box, h.box_parts, h.box, h.box_parts, dd, L, e_lo + L - 1, hp->hash_seed, tab, nullptr, st,
                      s);
  launch_keys_write(h.src, L, tab, keys, s);
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_crude_nn(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_hash_params* hp, int64_t* b_idx, float* D,
                      uint8_t* level) {
  if (!c) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_hash(hp);
  check_pair(c, A, B);
  CHX_CHECK(A->n == 0 || (b_idx && D), CH_EINVAL, "output NULL");
  CHX_CUDA(cudaSetDevice(c->device));
  if (A->n == 0) return CH_OK;
  CrudeBufs cb;
  uint32_t* st = nullptr;
  uint8_t* lv = level;
  carve(c, [&](auto& lay) {
    st = lay.template take<uint32_t>(1);
    take_crude(lay, A, B, hp, &cb);
    uint8_t* tmp = lay.template take<uint8_t>(size_t(A->n));
    if (!level) lv = tmp;
  });
  CHX_CUDA(cudaMemsetAsync(st, 0, 4, c->stream));
  run_crude(c, A, B, hp, &cb, b_idx, lv, D, st);
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_sample(ch_ctx* c, const float* D, int64_t nA, int64_t T, uint64_t seed, int64_t* idx, uint64_t* w,
                    uint64_t* W_total) {
  if (!c) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CHECK(nA >= 0 && T >= 0, CH_EINVAL, "nA and T must be >= 0");
  CHX_CHECK(nA == 0 || D, CH_EINVAL, "D NULL");
  CHX_CHECK(T == 0 || idx, CH_EINVAL, "idx NULL");
  CHX_CUDA(cudaSetDevice(c->device));
  SampleBufs sb;
  uint64_t* wbuf = w;
  ResBlock* res = nullptr;
  carve(c, [&](auto& lay) {
    res = lay.template take<ResBlock>(1);
    take_sample(lay, nA, &sb);
    uint64_t* tmp = lay.template take<uint64_t>(std::max<int64_t>(nA, 1));
    if (!w) wbuf = tmp;
  });
  cudaStream_t s = c->stream;
  launch_weights(D, nA, wbuf, sb.prefix, sb.sw, s);
  if (nA == 0) {
    CHX_CUDA(cudaMemsetAsync(idx, 0xFF, size_t(T) * sizeof(int64_t), s));
  } else {
    launch_draws(sb.prefix, nA, sb.sw.W, T, seed, idx, s);
  }
  if (W_total) {
    CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
    launch_k(k_collect, 1, 32, 0, s, res, nullptr, nullptr, nullptr, sb.sw.W, sb.sw.S, nullptr);
    launch_check("collect");
    ResBlock* h = static_cast<ResBlock*>(c->host_pin);
    finish(c, res, h);
    *W_total = h->W;
  }
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_sampled_nn(ch_ctx* c, const ch_set* A, const int64_t* idx, int64_t T, const ch_set* B, int32_t metric,
                        int32_t screen, uint32_t rerank_k, float* min_d, int64_t* argmin) {
  if (!c) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_pair(c, A, B);
  CHX_CHECK(metric == CH_L1 || metric == CH_L2, CH_EINVAL, "metric must be CH_L1 or CH_L2");
  CHX_CHECK(T >= 0, CH_EINVAL, "T must be >= 0");
  CHX_CHECK(T == 0 || (idx && min_d), CH_EINVAL, "idx or min_d NULL");
  CHX_CHECK(screen >= CH_SCREEN_AUTO && screen <= CH_SCREEN_FP8, CH_EINVAL, "unknown screen");
  if (rerank_k == 0) rerank_k = 8;
  CHX_CHECK(rerank_k <= 32, CH_EINVAL, "rerank_k must be in 1..32");
  CHX_CUDA(cudaSetDevice(c->device));
  ScanBufs sc;
  uint32_t* st = nullptr;
  carve(c, [&](auto& lay) {
    st = lay.template take<uint32_t>(1);
    take_scan(lay, c, A, B, T, metric, screen, rerank_k, &sc);
  });
  CHX_CUDA(cudaMemsetAsync(st, 0, 4, c->stream));
  run_scan(c, A, idx, T, B, metric, rerank_k, &sc, min_d, argmin, st);
  return CH_OK;
  CHX_GUARD_END
}

}  // extern "C"

namespace chx {

// ------------------------------------------------------------------ batched CrudeNN
// A pair's CrudeNN runs in the batched launches when its scales fit one group of
// bucket tables, its hashed rows fit registers (<= 64 values) and it uses the default grid
// family with hash tables (the single-pair path's forward group, kernel for kernel).
static bool crude_batchable(const ch_set* A, const ch_set* B, const ch_est_params* p) {
  const ch_hash_params* hp = &p->hash;
  if (p->sampling == CH_SAMPLING_UNIFORM || crude_kw(hp)) return false;
  if (hp->group != CH_GROUP_HASH || hp->family != CH_FAMILY_GRID) return false;
  if (A->dtype != B->dtype || A->n == 0 || B->n == 0) return false;
  const int dd = hp->metric == CH_L1 ? A->d : static_cast<int>(hp->proj_dim);
  if (dd > 64) return false;
  const int L = static_cast<int>(hp->levels);
  return table_plan(B->n, L).per_group >= L;
}

// bytes of bucket tables of one batched chunk
static size_t crude_chunk_budget() { return size_t(1) << 30; }

struct CrudeChunkPair {
  int64_t i;  // index of the pair in the batch
  Hashed hA, hB;
  CrudePair d;
};

// CrudeNN of the listed pairs (all batchable, one metric, hashed type and
// width, and storage type): per chunk of pairs, the l2 projections on the
// lanes, then on c's stream one launch each of scale tables, inserts, probes and
// crude distances for the whole chunk.  D_a goes to Dp[i].
template <class OnLanes>
static void run_crude_batched(ch_ctx* c, const std::vector<int64_t>& ids, const ch_set* const* A,
                              const ch_set* const* B, const ch_est_params* params, const std::vector<float*>& Dp,
                              ResBlock* dres, OnLanes&& on_lanes_of) {
  size_t at = 0;
  while (at < ids.size()) {
    // the chunk: pairs in order until the tables reach the budget
    std::vector<CrudeChunkPair> ch;
    size_t tab_bytes = 0;
    while (at < ids.size()) {
      const int64_t i = ids[at];
      const int L = static_cast<int>(params[i].hash.levels);
      const size_t tb = (size_t(L) << table_plan(B[i]->n, L).log_cap) * sizeof(ulonglong2);
      if (!ch.empty() && tab_bytes + tb > crude_chunk_budget()) break;
      tab_bytes += tb;
      CrudeChunkPair cp;
      cp.i = i;
      ch.push_back(cp);
      ++at;
    }
    const int np = static_cast<int>(ch.size());
    // layout: descriptors and block prefixes, tables, then each pair's buffers
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    auto lay_pairs = [&](auto& lay) {
      for (auto& cp : ch) {
        const int64_t i = cp.i;
        const ch_hash_params* hp = &params[i].hash;
        const int L = static_cast<int>(hp->levels);
        const int dd = hp->metric == CH_L1 ? A[i]->d : static_cast<int>(hp->proj_dim);
        take_hashed(lay, A[i], hp, &cp.hA);
        take_hashed(lay, B[i], hp, &cp.hB);
        cp.d.t = take_tables(lay, dd, L);
        cp.d.bidx = lay.template take<int64_t>(A[i]->n);
        cp.d.level = lay.template take<uint8_t>(A[i]->n);
      }
    };
    Layout m;
    lay_pairs(m);
    // small-d projections: a ProjSet per set and a block-run prefix per (type, d) run
    const size_t proj_head = al(sizeof(ProjSet) * 2 * np) + al(sizeof(int) * (2 * np + 64));
    const size_t head = al(sizeof(CrudePair) * np) + 3 * al(sizeof(int) * (np + 1)) + proj_head;
    const size_t bytes = head + al(tab_bytes) + m.need + 256;
    char* mem = nullptr;
    CHX_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&mem), bytes, c->pool, c->stream));
    CrudePair* dP = reinterpret_cast<CrudePair*>(mem);
    int* dblk = reinterpret_cast<int*>(mem + al(sizeof(CrudePair) * np));
    const size_t blk_stride = al(sizeof(int) * (np + 1)) / sizeof(int);
    ProjSet* dS = reinterpret_cast<ProjSet*>(mem + al(sizeof(CrudePair) * np) + 3 * al(sizeof(int) * (np + 1)));
    int* dSblk = reinterpret_cast<int*>(reinterpret_cast<char*>(dS) + al(sizeof(ProjSet) * 2 * np));
    char* tables = mem + head;
    Arena ar;
    ar.base = tables + al(tab_bytes);
    ar.cap = bytes - head - al(tab_bytes);
    ar.borrowed = true;
    Layout t;
    t.measure = false;
    t.a = &ar;
    lay_pairs(t);
    // the projections (l2): sets of d <= 8 in one launch per (storage type, d),
    // resident embeddings as they are, the others on the lanes; l1 rows are the
    // sets' own
    if (params[ch[0].i].hash.metric == CH_L2) {
      std::vector<int64_t> which;  // 2 j + side: projected on a lane
      std::map<std::pair<int, int>, std::vector<std::pair<ProjSet, int>>> runs;  // (type, d) -> (set, blocks)
      const int k = static_cast<int>(params[ch[0].i].hash.proj_dim);
      for (int j = 0; j < np; ++j)
        for (int side = 0; side < 2; ++side) {
          CrudeChunkPair& cp = ch[j];
          const ch_set* X = side ? B[cp.i] : A[cp.i];
          Hashed& h = side ? cp.hB : cp.hA;
          const ch_hash_params* hp = &params[cp.i].hash;
          if (resident_hashed(X, hp)) {
            run_hashed(c, X, hp, &h, &dres[cp.i].status);  // no launch: the set's own embedding
          } else if (X->d <= 8 && k <= 16) {
            h.src = HashSrc{h.Y, CH_F32, X->n, k, nullptr};
            h.box = h.boxY;
            h.box_parts = project_small_blocks(X->n, c->sm_count);
            runs[{X->dtype, X->d}].push_back(
                {ProjSet{X->data, X->scales, X->n, hp->hash_seed, h.Y, h.boxY, X->status}, h.box_parts});
          } else {
            which.push_back(2 * int64_t(j) + side);
          }
        }
      if (!runs.empty()) {
        std::vector<ProjSet> hS;
        std::vector<int> hblk;
        std::vector<std::tuple<int, int, int, int, int>> launches;  // type, d, first set, first prefix, blocks
        for (auto& r : runs) {
          const int first = static_cast<int>(hS.size()), pre = static_cast<int>(hblk.size());
          int tot = 0;
          hblk.push_back(0);
          for (auto& e : r.second) {
            hS.push_back(e.first);
            tot += e.second;
            hblk.push_back(tot);
          }
          launches.emplace_back(r.first.first, r.first.second, first, pre, tot);
        }
        CHX_CHECK(hblk.size() <= size_t(2 * np + 64), CH_EINVAL, "internal: projection runs");
        CHX_CUDA(cudaMemcpyAsync(dS, hS.data(), sizeof(ProjSet) * hS.size(), cudaMemcpyHostToDevice, c->stream));
        CHX_CUDA(cudaMemcpyAsync(dSblk, hblk.data(), sizeof(int) * hblk.size(), cudaMemcpyHostToDevice, c->stream));
        for (auto& l : launches) {
          const int first = std::get<2>(l), pre = std::get<3>(l);
          const int ns = static_cast<int>(runs[{std::get<0>(l), std::get<1>(l)}].size());
          launch_project_small_batch(dS + first, dSblk + pre, ns, std::get<4>(l), std::get<0>(l), std::get<1>(l), k,
                                     c->stream);
        }
      }
      if (!which.empty())
        on_lanes_of(which, [&](ch_ctx* lane, int64_t js) {
          CrudeChunkPair& cp = ch[js / 2];
          const ch_hash_params* hp = &params[cp.i].hash;
          if (js % 2) run_hashed(lane, B[cp.i], hp, &cp.hB, &dres[cp.i].status);
          else run_hashed(lane, A[cp.i], hp, &cp.hA, &dres[cp.i].status);
        });
    } else {
      for (auto& cp : ch) {
        run_hashed(c, A[cp.i], &params[cp.i].hash, &cp.hA, &dres[cp.i].status);
        run_hashed(c, B[cp.i], &params[cp.i].hash, &cp.hB, &dres[cp.i].status);
      }
    }
    // descriptors and block runs
    std::vector<CrudePair> hP(np);
    std::vector<int> b_ins(np + 1, 0), b_prb(np + 1, 0), b_dst(np + 1, 0);
    char* tab = tables;
    for (int j = 0; j < np; ++j) {
      CrudeChunkPair& cp = ch[j];
      const int64_t i = cp.i;
      const ch_hash_params* hp = &params[i].hash;
      const int L = static_cast<int>(hp->levels);
      CrudePair& d = cp.d;
      d.A = cp.hA.src;
      d.B = cp.hB.src;
      d.boxA = cp.hA.box;
      d.boxB = cp.hB.box;
      d.partsA = cp.hA.box_parts;
      d.partsB = cp.hB.box_parts;
      d.log_cap = table_plan(B[i]->n, L).log_cap;
      d.slots = reinterpret_cast<ulonglong2*>(tab);
      tab += (size_t(L) << d.log_cap) * sizeof(ulonglong2);
      d.L = L;
      d.top_exp = hp->top_exp;
      d.seed = hp->hash_seed;
      d.rawA = A[i]->data;
      d.scA = A[i]->scales;
      d.rawB = B[i]->data;
      d.scB = B[i]->scales;
      d.d = A[i]->d;
      d.gx_insert = static_cast<int>(std::min<int64_t>(ceil_div(B[i]->n, 128), 64));
      d.gx_probe = static_cast<int>(std::min<int64_t>(ceil_div(A[i]->n, 128), 256));
      d.gx_dist = static_cast<int>(std::min<int64_t>(ceil_div(A[i]->n * crude_dist_lanes(A[i]->d), 256), 256));
      d.D = Dp[i];
      d.status = &dres[i].status;
      hP[j] = d;
      b_ins[j + 1] = b_ins[j] + d.gx_insert * L;
      b_prb[j + 1] = b_prb[j] + d.gx_probe;
      b_dst[j + 1] = b_dst[j] + d.gx_dist;
    }
    cudaStream_t s = c->stream;
    CHX_CUDA(cudaMemcpyAsync(dP, hP.data(), sizeof(CrudePair) * np, cudaMemcpyHostToDevice, s));
    CHX_CUDA(cudaMemcpyAsync(dblk, b_ins.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, s));
    CHX_CUDA(cudaMemcpyAsync(dblk + blk_stride, b_prb.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, s));
    CHX_CUDA(cudaMemcpyAsync(dblk + 2 * blk_stride, b_dst.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, s));
    CHX_CUDA(cudaMemsetAsync(tables, 0, tab_bytes, s));
    const ch_set* A0 = A[ch[0].i];
    const ch_hash_params* hp0 = &params[ch[0].i].hash;
    launch_scale_tables_batch(dP, np, s);
    launch_insert_batch(dP, dblk, np, b_ins[np], hP[0].B.dtype, hP[0].B.dd, s);
    launch_probe_batch(dP, dblk + blk_stride, np, b_prb[np], hP[0].A.dtype, hP[0].A.dd, s);
    launch_crude_dist_batch(dP, dblk + 2 * blk_stride, np, b_dst[np], A0->dtype, hp0->metric, s);
    CHX_CUDA(cudaFreeAsync(mem, s));
  }
}

// ------------------------------------------------------------------ batched small scans
// Chunk length of the batched small scan, tuned per (storage type, metric, d,
// size class of B) by timing candidate lengths on the first batch that needs it
// (every candidate computes the same minima, so the tuning runs are the batch's
// own scans); the choice is kept for the process.
struct ScanTuneKey {
  int dtype, metric, d, cls;
  bool operator==(const ScanTuneKey& o) const {
    return dtype == o.dtype && metric == o.metric && d == o.d && cls == o.cls;
  }
};
struct ScanTuneHash {
  size_t operator()(const ScanTuneKey& k) const {
    return (size_t(k.dtype) * 1315423911u) ^ (size_t(k.metric) << 8) ^ (size_t(k.d) << 16) ^ (size_t(k.cls) << 24);
  }
};
static std::mutex g_tune_mu;
static std::unordered_map<ScanTuneKey, int64_t, ScanTuneHash> g_tuned;
constexpr int64_t kScanChunkCandidates[] = {2048, 4096, 8192, 16384, 32768};

static int size_class(int64_t n) { return ceil_log2_i64(std::max<int64_t>(n, 1)); }

static int64_t tuned_chunk(const ScanTuneKey& k) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(k);
  return it == g_tuned.end() ? 0 : it->second;
}

static void run_small_scans(ch_ctx* c, const std::vector<int64_t>& run, const std::vector<char>& small,
                            const ch_set* const* A, const ch_set* const* B, const ch_est_params* params,
                            const std::vector<int64_t>& Ts, const std::vector<int64_t*>& idxp,
                            const std::vector<unsigned long long*>& bestp) {
  // groups of one storage type, metric and dimension
  std::map<std::tuple<int, int, int>, std::vector<int64_t>> groups;
  for (int64_t i : run)
    if (small[i]) groups[{A[i]->dtype, params[i].hash.metric, A[i]->d}].push_back(i);
  const int spi = small_scan_samples_per_item();
  for (auto& g : groups) {
    const auto& ids = g.second;
    const int dtype = std::get<0>(g.first), metric = std::get<1>(g.first), d = std::get<2>(g.first);
    int64_t sum_nB = 0;
    for (int64_t i : ids) sum_nB += B[i]->n;
    const ScanTuneKey key{dtype, metric, d, size_class(sum_nB / static_cast<int64_t>(ids.size()))};
    std::vector<SmallScanPair> pairs(ids.size());
    for (size_t j = 0; j < ids.size(); ++j) {
      const int64_t i = ids[j];
      pairs[j] = SmallScanPair{A[i]->data, A[i]->scales, A[i]->n, idxp[i], Ts[i], B[i]->data, B[i]->scales, B[i]->n,
                               bestp[i]};
    }
    auto items_for = [&](int64_t cl) {
      std::vector<SmallScanItem> it;
      for (size_t j = 0; j < ids.size(); ++j) {
        const int64_t i = ids[j];
        const int64_t sb = ceil_div(Ts[i], int64_t(spi));
        for (int64_t b0 = 0; b0 < B[i]->n; b0 += cl)
          for (int64_t q = 0; q < sb; ++q) it.push_back(SmallScanItem{int32_t(j), int32_t(q), b0});
      }
      return it;
    };
    // device buffers: the pair list and the largest item list of the candidates
    const int64_t tuned = tuned_chunk(key);
    const std::vector<int64_t> cands =
        tuned ? std::vector<int64_t>{tuned}
              : std::vector<int64_t>(std::begin(kScanChunkCandidates), std::end(kScanChunkCandidates));
    size_t max_items = 0;
    std::vector<std::vector<SmallScanItem>> lists;
    for (int64_t cl : cands) {
      lists.push_back(items_for(cl));
      max_items = std::max(max_items, lists.back().size());
    }
    char* dmem = nullptr;
    const size_t pbytes = (sizeof(SmallScanPair) * pairs.size() + 255) & ~size_t(255);
    CHX_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&dmem), pbytes + sizeof(SmallScanItem) * max_items,
                                     c->pool, c->stream));
    SmallScanPair* dp = reinterpret_cast<SmallScanPair*>(dmem);
    SmallScanItem* di = reinterpret_cast<SmallScanItem*>(dmem + pbytes);
    CHX_CUDA(cudaMemcpyAsync(dp, pairs.data(), sizeof(SmallScanPair) * pairs.size(), cudaMemcpyHostToDevice,
                             c->stream));
    float best_ms = 0.0f;
    int64_t best_cl = cands[0];
    for (size_t k = 0; k < cands.size(); ++k) {
      CHX_CUDA(cudaMemcpyAsync(di, lists[k].data(), sizeof(SmallScanItem) * lists[k].size(), cudaMemcpyHostToDevice,
                               c->stream));
      if (cands.size() > 1) CHX_CUDA(cudaEventRecord(c->ev[5], c->stream));
      launch_scan_small_batch(dp, di, static_cast<int64_t>(lists[k].size()), cands[k], dtype, metric, d, c->sm_count,
                              c->stream);
      if (cands.size() > 1) {
        CHX_CUDA(cudaEventRecord(c->ev[6], c->stream));
        CHX_CUDA(cudaEventSynchronize(c->ev[6]));
        float ms = 0.0f;
        CHX_CUDA(cudaEventElapsedTime(&ms, c->ev[5], c->ev[6]));
        if (k == 0 || ms < best_ms) {
          best_ms = ms;
          best_cl = cands[k];
        }
      }
    }
    if (cands.size() > 1) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = best_cl;
    }
    CHX_CUDA(cudaFreeAsync(dmem, c->stream));
  }
}

constexpr int kBatchLanes = 8;  // concurrent streams (and host threads) of a batched call

// argument checks of one estimate; returns (T, R)
static void check_estimate(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, int64_t* T,
                           uint32_t* R) {
  CHX_CHECK(p, CH_EINVAL, "params NULL");
  check_hash(&p->hash);
  check_pair(c, A, B);
  CHX_CHECK(p->screen >= CH_SCREEN_AUTO && p->screen <= CH_SCREEN_FP8, CH_EINVAL, "unknown screen");
  *R = p->rerank_k ? p->rerank_k : 8;
  CHX_CHECK(*R <= 32, CH_EINVAL, "rerank_k must be in 1..32");
  CHX_CHECK(p->T >= 0, CH_EINVAL, "T must be >= 0");
  CHX_CHECK(p->T > 0 || (p->eps > 0.0 && p->eps < 1.0), CH_EINVAL, "eps must be in (0, 1)");
  CHX_CHECK(p->sampling == CH_SAMPLING_IMPORTANCE || p->sampling == CH_SAMPLING_UNIFORM, CH_EINVAL,
            "unknown sampling");
  *T = p->T > 0 ? p->T : default_T(A->n, B->n, p->eps);
}

// Runs the estimate of (A, B) on c's stream in the buffers eb (carved from c's
// workspace by the caller); with hashed_ready, eb.cb.hA / hB already hold both
// sets' hashed spaces.
static ResBlock* estimate_run(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, int64_t T,
                              uint32_t R, EstBufs& eb, ResBlock* res_out, bool events, int* screen_used,
                              ResBlock* host_out, bool lone, bool hashed_ready) {
  const int64_t nA = A->n;
  if (res_out) eb.res = res_out;
  CrudeBufs& cb = eb.cb;
  SampleBufs& sb = eb.sb;
  ScanBufs& sc = eb.sc;
  ResBlock* res = eb.res;
  cudaStream_t s = c->stream;
  if (events) CHX_CUDA(cudaEventRecord(c->ev[0], s));
  CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
  const bool uniform = p->sampling == CH_SAMPLING_UNIFORM;
  if (uniform) {
    // the baseline: every D_a = 1, so the weights are equal and the draws uniform;
    // the set passes still check both sets for non-finite values
    for (const ch_set* x : {A, B}) {
      if (p->hash.metric == CH_L2) ensure_norms(const_cast<ch_set*>(x), s);
      else ensure_ingest(const_cast<ch_set*>(x), s);
    }
    launch_fill_ones(eb.D, nA, s);
  } else {
    run_crude(c, A, B, &p->hash, &cb, eb.bidx, eb.level, eb.D, &res->status, sb.sw.maxD, hashed_ready);
  }
  if (events) CHX_CUDA(cudaEventRecord(c->ev[1], s));
  launch_weights(eb.D, nA, eb.w, sb.prefix, sb.sw, s, !uniform, true);
  launch_draws(sb.prefix, nA, sb.sw.W, T, p->sample_seed, eb.idx, s, sb.sw.blocksum, lone);
  if (events) CHX_CUDA(cudaEventRecord(c->ev[2], s));
  KernelTimer kt;
  if (events) {
    kt.before = c->ev[5];
    kt.after = c->ev[6];
  }
  run_scan(c, A, eb.idx, T, B, p->hash.metric, R, &sc, eb.m, nullptr, &res->status, kt);
  if (events) CHX_CUDA(cudaEventRecord(c->ev[3], s));
  // the combine's last pass also fills the result block
  launch_combine(eb.m, eb.idx, eb.w, sb.sw.W, T, eb.D, nA, eb.out2, s,
                 CollectArgs{res, A->status, B->status, sb.sw.S, uniform ? nullptr : cb.e_top, host_out});
  if (events) CHX_CUDA(cudaEventRecord(c->ev[4], s));
  if (screen_used) *screen_used = sc.screen;
  return res;
}

// Enqueues the whole estimate of (A, B) on c's stream, carving c's workspace; the
// result block lands in res_out (or in the workspace when null).  With events,
// records stage boundaries in c->ev.  Returns the result block and the screen used.
static ResBlock* estimate_enqueue(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, int64_t T,
                                  uint32_t R, ResBlock* res_out, bool events, int* screen_used,
                                  ResBlock* host_out = nullptr, bool lone = false) {
  EstBufs eb;
  carve(c, [&](auto& lay) { take_estimate(lay, c, A, B, p, T, R, &eb); });
  return estimate_run(c, A, B, p, T, R, eb, res_out, events, screen_used, host_out, lone, false);
}

// the workspace bytes estimate_enqueue carves for (A, B, p)
static size_t estimate_need(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, int64_t T,
                            uint32_t R) {
  Layout m;
  EstBufs eb;
  take_estimate(m, c, A, B, p, T, R, &eb);
  return m.need + 256;
}

}  // namespace chx

extern "C" {

ch_status ch_estimate(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, double* eta,
                      ch_est_report* rep) {
  if (!c || !p || !eta) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  int64_t T;
  uint32_t R;
  check_estimate(c, A, B, p, &T, &R);
  CHX_CUDA(cudaSetDevice(c->device));
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->T = T;
  }
  if (A->n == 0) {
    *eta = 0.0;
    return CH_OK;
  }
  int screen = 0;
  // the combine's last block writes the finished result block into the pinned page
  ResBlock* h = static_cast<ResBlock*>(c->host_pin);
  estimate_enqueue(c, A, B, p, T, R, nullptr, rep != nullptr, &screen, h, true);
  CHX_CUDA(cudaStreamSynchronize(c->stream));
  check_result(h);
  *eta = h->eta;
  if (rep) {
    rep->eta = h->eta;
    rep->D_total = h->D_total;
    rep->W = h->W;
    rep->top_exp = h->e_top;
    rep->shift_S = h->S;
    cudaEventElapsedTime(&rep->t_crude_ms, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&rep->t_sample_ms, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&rep->t_scan_ms, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&rep->t_total_ms, c->ev[0], c->ev[4]);
    rep->t_kernel_ms = 0.0f;
    if (T > 0) cudaEventElapsedTime(&rep->t_kernel_ms, c->ev[5], c->ev[6]);
    rep->screen = screen;
  }
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_estimate_batch(ch_ctx* c, int64_t count, const ch_set* const* A, const ch_set* const* B,
                            const ch_est_params* params, double* eta, ch_status* status) {
  if (!c || count < 0 || (count > 0 && (!A || !B || !params || !eta))) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CUDA(cudaSetDevice(c->device));
  if (count == 0) return CH_OK;
  // per-pair checks; a failing pair gets its status and is skipped
  std::vector<int64_t> Ts(count);
  std::vector<uint32_t> Rs(count);
  std::vector<ch_status> st(count, CH_OK);
  for (int64_t i = 0; i < count; ++i) {
    try {
      check_estimate(c, A[i], B[i], &params[i], &Ts[i], &Rs[i]);
      CHX_CHECK(A[i]->ctx == c && B[i]->ctx == c, CH_EINVAL, "batched sets must belong to the context");
    } catch (const Err& e) {
      st[i] = e.st;
    }
  }
  // lanes: sub-contexts with their own streams and workspaces
  const int K = static_cast<int>(std::min<int64_t>(kBatchLanes, count));
  while (static_cast<int>(c->lanes.size()) < K) {
    ch_ctx* l = nullptr;
    const ch_status cs = ch_ctx_create(c->device, nullptr, &l);
    CHX_CHECK(cs == CH_OK, cs, "batch lane creation failed");
    c->lanes.push_back(l);
  }
  // K lanes run at once, so each screen splits B for its share of the SMs only
  // (fewer chunks, fewer rerank candidates per sample)
  for (int k = 0; k < K; ++k) {
    c->lanes[k]->screen_chunk_sms = std::max(1, c->sm_count / K);
    c->lanes[k]->wait_cycles = c->wait_cycles;
  }
  // the lazy set passes run here, on c's stream, so that no two lanes race on them
  for (int64_t i = 0; i < count; ++i) {
    if (st[i] != CH_OK) continue;
    const ch_set* X[2] = {A[i], B[i]};
    for (const ch_set* x : X) {
      if (params[i].hash.metric == CH_L2) ensure_norms(const_cast<ch_set*>(x), c->stream);
      else ensure_ingest(const_cast<ch_set*>(x), c->stream);
    }
  }
  // The pairs run in four phases, so that the small per-pair steps become one
  // launch each for the whole batch:
  //   1. CrudeNN of every pair on the lanes (pair i on lane i mod K);
  //   2. one launch: weights, prefix, W and draws of every pair (a CTA per pair);
  //   3. the sampled scans on the lanes;
  //   4. one launch: the combine of every pair, in the single-pair summation order.
  // Each pair's D, w, prefix, draws and minima live in one batch allocation; a
  // lane's workspace holds the scratch of one pair's CrudeNN or scan at a time.
  std::vector<int64_t> run;
  for (int64_t i = 0; i < count; ++i)
    if (st[i] == CH_OK && A[i]->n > 0) run.push_back(i);
  // pairs whose sampled scan is the exact scan of d <= 4: one persistent launch
  // for all of them (per storage type and metric) instead of a scan per pair
  std::vector<char> small(count, 0);
  for (int64_t i : run)
    small[i] = A[i]->d <= kBatchScanMaxD && Ts[i] > 0 && B[i]->n < (int64_t(1) << 32) - 1 &&
               screen_choice(params[i].screen, params[i].hash.metric, A[i], B[i]) == CH_SCREEN_EXACT;
  // pairs whose CrudeNN runs in the batched launches (the others on the lanes)
  std::vector<char> bcr(count, 0);
  for (int64_t i : run) bcr[i] = crude_batchable(A[i], B[i], &params[i]);
  std::vector<size_t> need(K, 0);
  for (int64_t i : run) {
    const ch_est_params* p = &params[i];
    ch_ctx* lane = c->lanes[i % K];
    Layout mc, ms;
    CrudeBufs cb;
    if (!bcr[i]) {
      take_crude(mc, A[i], B[i], &p->hash, &cb);
      mc.template take<int64_t>(A[i]->n);  // b(a)
      mc.template take<uint8_t>(A[i]->n);  // level
    }
    ScanBufs sc;
    if (!small[i]) take_scan(ms, lane, A[i], B[i], Ts[i], p->hash.metric, p->screen, Rs[i], &sc);
    need[i % K] = std::max(need[i % K], std::max(mc.need, ms.need) + 256);
  }
  for (int k = 0; k < K; ++k) c->lanes[k]->ws.reserve(need[k]);
  // the batch allocation: result blocks, the work list, then each pair's arrays
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t arena = al(sizeof(ResBlock) * count) + al(sizeof(BatchItem) * std::max<size_t>(run.size(), 1));
  size_t best_bytes = 0;  // the small pairs' minima (distance bits << 32), one block (cleared together)
  for (int64_t i : run) {
    arena += al(size_t(A[i]->n) * 4) + 2 * al(size_t(A[i]->n) * 8) + al(size_t(Ts[i]) * 8) + al(size_t(Ts[i]) * 4);
    if (small[i]) best_bytes += al(size_t(Ts[i]) * 8);
  }
  arena += best_bytes;
  char* mem = nullptr;
  CHX_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&mem), arena, c->pool, c->stream));
  ResBlock* dres = reinterpret_cast<ResBlock*>(mem);
  BatchItem* ditems = reinterpret_cast<BatchItem*>(mem + al(sizeof(ResBlock) * count));
  char* cur = mem + al(sizeof(ResBlock) * count) + al(sizeof(BatchItem) * std::max<size_t>(run.size(), 1));
  std::vector<BatchItem> items(run.size());
  std::vector<float*> Dp(count, nullptr), mp(count, nullptr);
  std::vector<int64_t*> idxp(count, nullptr);
  std::vector<unsigned long long*> bestp(count, nullptr);
  char* best_base = cur;
  cur += best_bytes;
  {
    char* b = best_base;
    for (int64_t i : run)
      if (small[i]) {
        bestp[i] = reinterpret_cast<unsigned long long*>(b);
        b += al(size_t(Ts[i]) * 8);
      }
  }
  for (size_t j = 0; j < run.size(); ++j) {
    const int64_t i = run[j];
    BatchItem& it = items[j];
    float* D = reinterpret_cast<float*>(cur);
    cur += al(size_t(A[i]->n) * 4);
    it.w = reinterpret_cast<uint64_t*>(cur);
    cur += al(size_t(A[i]->n) * 8);
    it.prefix = reinterpret_cast<uint64_t*>(cur);
    cur += al(size_t(A[i]->n) * 8);
    it.idx = reinterpret_cast<int64_t*>(cur);
    cur += al(size_t(Ts[i]) * 8);
    float* m = reinterpret_cast<float*>(cur);
    cur += al(size_t(Ts[i]) * 4);
    it.D = D;
    it.m = m;
    it.mpk = bestp[i];
    it.res = dres + i;
    it.statusA = A[i]->status;
    it.statusB = B[i]->status;
    it.nA = A[i]->n;
    it.T = Ts[i];
    it.seed = params[i].sample_seed;
    Dp[i] = D;
    mp[i] = m;
    idxp[i] = it.idx;
  }
  CHX_CUDA(cudaMemsetAsync(dres, 0, sizeof(ResBlock) * count, c->stream));
  if (!items.empty())
    CHX_CUDA(cudaMemcpyAsync(ditems, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                             c->stream));
  // c's stream -> every lane, and back
  auto fork = [&] {
    CHX_CUDA(cudaEventRecord(c->ev[7], c->stream));
    for (int k = 0; k < K; ++k) CHX_CUDA(cudaStreamWaitEvent(c->lanes[k]->stream, c->ev[7], 0));
  };
  auto join = [&] {
    for (int k = 0; k < K; ++k) {
      CHX_CUDA(cudaEventRecord(c->lanes[k]->ev[7], c->lanes[k]->stream));
      CHX_CUDA(cudaStreamWaitEvent(c->stream, c->lanes[k]->ev[7], 0));
    }
  };
  // one host thread per lane enqueues that lane's pairs (kernel launches are the
  // host-side cost of small pairs); the sets' lazy state is already final
  auto on_lanes = [&](auto&& body) {
    std::vector<std::thread> th;
    for (int k = 0; k < K; ++k)
      th.emplace_back([&, k] {
        cudaSetDevice(c->device);
        for (int64_t i : run) {
          if (i % K != k || st[i] != CH_OK) continue;
          try {
            body(c->lanes[k], i);
          } catch (const Err& e) {
            st[i] = e.st;
          } catch (...) {
            st[i] = CH_ECUDA;
          }
        }
      });
    for (auto& t : th) t.join();
  };
  fork();
  on_lanes([&](ch_ctx* lane, int64_t i) {  // 1. CrudeNN (or the uniform baseline's equal weights)
    const ch_est_params* p = &params[i];
    if (bcr[i]) return;  // below, in the batched launches
    if (p->sampling == CH_SAMPLING_UNIFORM) {
      launch_fill_ones(Dp[i], A[i]->n, lane->stream);
      return;
    }
    CrudeBufs cb;
    int64_t* bidx = nullptr;
    uint8_t* level = nullptr;
    carve(lane, [&](auto& lay) {
      take_crude(lay, A[i], B[i], &p->hash, &cb);
      bidx = lay.template take<int64_t>(A[i]->n);
      level = lay.template take<uint8_t>(A[i]->n);
    });
    run_crude(lane, A[i], B[i], &p->hash, &cb, bidx, level, Dp[i], &dres[i].status, nullptr);
  });
  join();
  {
    // the batched CrudeNN, one run per (metric, hashed type and width, storage type)
    std::map<std::tuple<int, int, int, int>, std::vector<int64_t>> groups;
    for (int64_t i : run) {
      if (!bcr[i]) continue;
      const ch_hash_params* hp = &params[i].hash;
      const int dd = hp->metric == CH_L1 ? A[i]->d : static_cast<int>(hp->proj_dim);
      const int hdt = hp->metric == CH_L1 ? A[i]->dtype : CH_F32;
      groups[{hp->metric, hdt, dd, A[i]->dtype}].push_back(i);
    }
    // body(lane, j) for j in which, j on lane j mod K; c's stream -> lanes -> c's stream
    auto on_lanes_of = [&](const std::vector<int64_t>& which, auto&& body) {
      fork();
      std::vector<std::thread> th;
      std::vector<ch_status> err(K, CH_OK);
      for (int k = 0; k < K; ++k)
        th.emplace_back([&, k] {
          cudaSetDevice(c->device);
          try {
            for (int64_t j : which)
              if (j % K == k) body(c->lanes[k], j);
          } catch (const Err& e) {
            err[k] = e.st;
          } catch (...) {
            err[k] = CH_ECUDA;
          }
        });
      for (auto& t : th) t.join();
      join();
      for (int k = 0; k < K; ++k) CHX_CHECK(err[k] == CH_OK, err[k], "batched CrudeNN: a projection failed");
    };
    for (auto& g : groups) run_crude_batched(c, g.second, A, B, params, Dp, dres, on_lanes_of);
  }
  launch_batch_sample(ditems, static_cast<int64_t>(run.size()), c->stream);  // 2.
  fork();
  on_lanes([&](ch_ctx* lane, int64_t i) {  // 3. the sampled scans (the small pairs' below)
    if (small[i]) return;
    const ch_est_params* p = &params[i];
    ScanBufs sc;
    carve(lane, [&](auto& lay) { take_scan(lay, lane, A[i], B[i], Ts[i], p->hash.metric, p->screen, Rs[i], &sc); });
    run_scan(lane, A[i], idxp[i], Ts[i], B[i], p->hash.metric, Rs[i], &sc, mp[i], nullptr, &dres[i].status);
  });
  if (best_bytes) {
    CHX_CUDA(cudaMemsetAsync(best_base, 0xFF, best_bytes, c->stream));
    run_small_scans(c, run, small, A, B, params, Ts, idxp, bestp);
  }
  join();
  launch_batch_combine(ditems, static_cast<int64_t>(run.size()), c->stream);  // 4.
  const size_t bytes = sizeof(ResBlock) * count;
  if (c->batch_pin_cap < bytes) {
    if (c->batch_pin) cudaFreeHost(c->batch_pin);
    c->batch_pin = nullptr;
    c->batch_pin_cap = 0;
    CHX_CUDA(cudaMallocHost(&c->batch_pin, bytes));
    c->batch_pin_cap = bytes;
  }
  ResBlock* h = static_cast<ResBlock*>(c->batch_pin);
  CHX_CUDA(cudaMemcpyAsync(h, dres, bytes, cudaMemcpyDeviceToHost, c->stream));
  CHX_CUDA(cudaFreeAsync(mem, c->stream));
  CHX_CUDA(cudaStreamSynchronize(c->stream));
  ch_status first = CH_OK;
  for (int64_t i = 0; i < count; ++i) {
    eta[i] = 0.0;
    if (st[i] == CH_OK && A[i]->n > 0) {
      try {
        check_result(&h[i]);
        eta[i] = h[i].eta;
      } catch (const Err& e) {
        st[i] = e.st;
      }
    }
    if (status) status[i] = st[i];
    if (first == CH_OK && st[i] != CH_OK) first = st[i];
  }
  if (first != CH_OK) c->err = "one or more pairs failed (see the per-pair status)";
  return first;
  CHX_GUARD_END
}

ch_status ch_estimate_sym(ch_ctx* c, const ch_set* A, const ch_set* B, const ch_est_params* p, double* eta,
                          double* eta_ab, double* eta_ba) {
  if (!c || !p || !eta) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  CHX_CHECK(A && B, CH_EINVAL, "set NULL");
  ch_est_params pb = *p;  // the (B, A) direction: its own draws
  pb.sample_seed ^= 0x9E3779B97F4A7C15ull;
  const bool shared = p->sampling != CH_SAMPLING_UNIFORM && !crude_kw(&p->hash) && p->hash.group == CH_GROUP_HASH &&
                      p->hash.family != CH_FAMILY_SIMHASH && A->n > 0 && B->n > 0;
  if (!shared) {
    // the variants without shared set passes: the two directions as a batch of two
    const ch_set* As[2] = {A, B};
    const ch_set* Bs[2] = {B, A};
    ch_est_params ps[2] = {*p, pb};
    double e[2] = {0.0, 0.0};
    ch_status st[2] = {CH_OK, CH_OK};
    const ch_status r = ch_estimate_batch(c, 2, As, Bs, ps, e, st);
    if (r != CH_OK) {
      if (st[0] != CH_OK || st[1] != CH_OK) {
        c->err = st[0] != CH_OK ? "direction (A, B) failed" : "direction (B, A) failed";
        return st[0] != CH_OK ? st[0] : st[1];
      }
      return r;
    }
    *eta = e[0] + e[1];
    if (eta_ab) *eta_ab = e[0];
    if (eta_ba) *eta_ba = e[1];
    return CH_OK;
  }
  // CH(A, B) + CH(B, A) sharing the set passes: both directions use the same hash
  // parameters, so A's and B's hashed spaces (the l2 embedding under the one
  // Gaussian matrix, or the rows and boxes for l1), the joint box and the scales
  // are the same; they are computed once, then each direction builds its own
  // bucket tables, draws and scans.
  int64_t Tab, Tba;
  uint32_t R, Rb;
  check_estimate(c, A, B, p, &Tab, &R);
  check_estimate(c, B, A, &pb, &Tba, &Rb);
  CHX_CUDA(cudaSetDevice(c->device));
  EstBufs e1, e2;
  carve(c, [&](auto& lay) {
    take_estimate(lay, c, A, B, p, Tab, R, &e1);
    take_estimate(lay, c, B, A, &pb, Tba, Rb, &e2);
  });
  ResBlock* h = static_cast<ResBlock*>(c->host_pin);  // [0]: (A, B), [1]: (B, A)
  estimate_run(c, A, B, p, Tab, R, e1, nullptr, false, nullptr, h, true, false);
  e2.cb.hA = e1.cb.hB;
  e2.cb.hB = e1.cb.hA;
  estimate_run(c, B, A, &pb, Tba, Rb, e2, nullptr, false, nullptr, h + 1, true, true);
  CHX_CUDA(cudaStreamSynchronize(c->stream));
  check_result(h);
  check_result(h + 1);
  *eta = h[0].eta + h[1].eta;
  if (eta_ab) *eta_ab = h[0].eta;
  if (eta_ba) *eta_ba = h[1].eta;
  return CH_OK;
  CHX_GUARD_END
}

ch_status ch_exact(ch_ctx* c, const ch_set* A, const ch_set* B, int32_t metric, int32_t mode, double* ch,
                   float* per_a_min) {
  if (!c || !ch) return CH_EINVAL;
  CHX_GUARD_BEGIN(c)
  check_pair(c, A, B);
  CHX_CHECK(metric == CH_L1 || metric == CH_L2, CH_EINVAL, "metric must be CH_L1 or CH_L2");
  CHX_CHECK(mode == 0 || mode == 1, CH_EINVAL, "mode must be 0 or 1");
  CHX_CUDA(cudaSetDevice(c->device));
  const int64_t nA = A->n;
  ScanBufs sc;
  ResBlock* res = nullptr;
  float* mins = per_a_min;
  double* out2 = nullptr;
  carve(c, [&](auto& lay) {
    res = lay.template take<ResBlock>(1);
    out2 = lay.template take<double>(kCombineDoubles);
    take_scan(lay, c, A, B, nA, metric, mode == 0 ? CH_SCREEN_EXACT : CH_SCREEN_AUTO, 8, &sc);
    float* tmp = lay.template take<float>(std::max<int64_t>(nA, 1));
    if (!per_a_min) mins = tmp;
  });
  cudaStream_t s = c->stream;
  CHX_CUDA(cudaMemsetAsync(res, 0, sizeof(ResBlock), s));
  CHX_CUDA(cudaMemsetAsync(out2, 0, 2 * sizeof(double), s));
  ensure_ingest(const_cast<ch_set*>(A), s);  // finite check of both sets
  ensure_ingest(const_cast<ch_set*>(B), s);
  if (nA > 0) {
    run_scan(c, A, nullptr, nA, B, metric, 8, &sc, mins, nullptr, &res->status);
    launch_sum_f32(mins, nA, out2, s);
  }
  launch_k(k_collect, 1, 32, 0, s, res, A->status, B->status, out2, nullptr, nullptr, nullptr);
  launch_check("collect");
  ResBlock* h = static_cast<ResBlock*>(c->host_pin);
  finish(c, res, h);
  *ch = h->D_total;
  return CH_OK;
  CHX_GUARD_END
}

}  // extern "C"
