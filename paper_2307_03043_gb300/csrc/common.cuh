// common.cuh -- shared definitions of libchamfer's CUDA sources.
//
// Exactness rules for every kernel whose result must match the canonical
// definition bit for bit: binary32 round-to-nearest intrinsics only
// (__fadd_rn, __fsub_rn, __fmul_rn, __fmaf_rn, __fsqrt_rn), which the
// compiler never contracts or reassociates; no fast-math; denormals kept
// (the library is built with -ftz=false -prec-div=true -prec-sqrt=true).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include <string>
#include <vector>

#include "../../include/chamfer.h"

namespace chx {

constexpr int kMaxLevels = 32;   // L <= 32 (keys kept in registers in blocks of 16)
constexpr int kMaxProj = 64;     // l2 embedding width k <= 64
constexpr int kMaxDim = 4096;    // point dimension supported by the kernels
constexpr int kLevelBlock = 16;  // scales handled per register block

// ------------------------------------------------------------------ errors
struct Err {
  ch_status st;
  std::string msg;
};

#define CHX_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::chx::Err{CH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define CHX_CHECK(cond, code, text)                 \
  do {                                              \
    if (!(cond)) throw ::chx::Err{(code), (text)};  \
  } while (0)

// kernels launched by this process through the library (for launch accounting)
void count_launch();

inline void launch_check(const char* what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Err{CH_ECUDA, std::string("launch ") + what + ": " + cudaGetErrorString(e)};
}

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_entry(): it waits until the kernel launched before it on the stream has
// completed and its writes are visible (a no-op when there is no such
// dependency), then lets the next kernel be scheduled.  Launched through
// launch_k, a kernel's launch and block scheduling thus overlap the tail of its
// predecessor while its own work still starts after the predecessor's ends.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... P, class... A>
inline void launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
  if (e != cudaSuccess) throw Err{CH_ECUDA, std::string("launch: ") + cudaGetErrorString(e)};
}

// device status bits (written by kernels, read back by synchronising calls)
enum : uint32_t {
  ST_NONFINITE = 1u << 0,   // a set holds NaN or Inf
  ST_RANGE = 1u << 1,       // scale exponents outside the supported range
  ST_TABLE_FULL = 1u << 2,  // a hash table probe sequence exceeded its bound
  ST_TIMEOUT = 1u << 3,     // a bounded device wait gave up
  ST_BAD_INDEX = 1u << 4,   // an index argument was out of range
};

// ------------------------------------------------------------------ workspace
// Grow-only device arena; one per context (and one per serving slot).
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool borrowed = false;  // base is lent by the caller: never freed or regrown here
  void reserve(size_t bytes);  // synchronises the device if it must grow
  void release();
  void reset() { used = 0; }
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (used + bytes > cap) throw Err{CH_ENOMEM, "workspace arena overflow (internal sizing error)"};
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

}  // namespace chx

// a set's resident l2 embedding under one (hash seed, width k), made by ch_set_embed
struct chx_hashed {
  bool valid = false;
  uint64_t seed = 0;
  int k = 0;
  float* Y = nullptr;         // projection [n][k] (+ the width-padded Gaussian-matrix tail), owned by the set
  uint32_t* box = nullptr;    // ordered-encoded partial boxes [parts][2][k] of Y
  int parts = 0;
};

struct ch_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  int screen_chunk_sms = 0;  // SMs the screen's B split aims to fill (0: all); a batch lane's share
  long long wait_cycles = 0;  // budget of the tensor-core screen's pipeline waits, SM cycles (0: about 2 s)
  chx::Arena ws;
  cudaMemPool_t pool = nullptr;  // stream-ordered pool for sets; keeps freed memory
  void* host_pin = nullptr;   // pinned page for small readbacks
  std::string err;
  cudaEvent_t ev[8] = {};
  std::vector<ch_ctx*> lanes;  // sub-contexts (own streams) of batched calls, made on first use
  cudaStream_t side = nullptr;  // second stream for work that runs beside the main one, made on first use
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  void* batch_pin = nullptr;   // pinned result blocks of batched calls
  size_t batch_pin_cap = 0;
};

struct ch_set {
  ch_ctx* ctx = nullptr;
  void* data = nullptr;
  bool owned = false;
  int64_t n = 0;
  int32_t d = 0;
  int32_t dtype = CH_F32;
  float* scales = nullptr;     // FP8 row scales (device, owned)
  float* norms = nullptr;      // |x|^2 per row (device, owned), binary32
  uint32_t* status = nullptr;  // device status word (ST_* bits)
  uint32_t* box_x = nullptr;   // ordered-encoded [2][d] bounding box of x (l1 hashed space)
  chx_hashed hs;               // cached l2 embedding
  uint32_t ready = 0;          // READY_* passes already enqueued on the context's stream
};

namespace chx {
enum : uint32_t {
  READY_BOX_X = 1u << 0,  // box_x computed (and the finite check done)
  READY_NORMS = 1u << 1,  // norms computed (and the finite check done)
};
// ingest pass (box of x, finite check) unless already done
void ensure_ingest(ch_set* X, cudaStream_t s);
// |x|^2 per row (sequential fmaf chain over j) unless already done
void ensure_norms(ch_set* X, cudaStream_t s);
}  // namespace chx

namespace chx {

// ------------------------------------------------------------------ RNG
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with the published
// multipliers, the key advancing by the Weyl constants between rounds.
struct P4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline P4 philox10(P4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2511F53ull * c.x;
    const uint64_t m1 = 0xCD9E8D57ull * c.z;
    P4 n;
    n.x = static_cast<uint32_t>(m1 >> 32) ^ c.y ^ k0;
    n.y = static_cast<uint32_t>(m1);
    n.z = static_cast<uint32_t>(m0 >> 32) ^ c.w ^ k1;
    n.w = static_cast<uint32_t>(m0);
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014; Vigna's variant constants)
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ float helpers
// order-preserving map binary32 -> uint32 (for atomic min / max of floats)
__host__ __device__ inline uint32_t ord_enc(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float ord_dec(uint32_t u) {
  uint32_t v = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
  float f;
  memcpy(&f, &v, 4);
  return f;
}

// exact 2^e as binary32 for -126 <= e <= 127
__device__ inline float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// E4M3 (OCP FP8, no infinities) code -> binary32, exact: the hardware conversion
// to binary16 (every E4M3 value, subnormals included, is a binary16 value; the two
// NaN codes give NaN), then binary16 -> binary32, also exact
__device__ inline float e4m3_to_f32(uint8_t b) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(b), __NV_E4M3);
  return __half2float(__half(h));
}

__device__ inline float bf16_to_f32(uint16_t h) { return __int_as_float(static_cast<uint32_t>(h) << 16); }

// element j of row r of a set stored as DT, widened to binary32 exactly
template <int DT>
__device__ inline float load_elem(const void* base, int64_t r, int d, int j, const float* scales) {
  if constexpr (DT == CH_F32) {
    return static_cast<const float*>(base)[r * d + j];
  } else if constexpr (DT == CH_BF16) {
    return bf16_to_f32(static_cast<const uint16_t*>(base)[r * d + j]);
  } else {
    return __fmul_rn(e4m3_to_f32(static_cast<const uint8_t*>(base)[r * d + j]), scales[r]);
  }
}

__host__ __device__ inline int ceil_log2_i64(int64_t n) {
  int c = 0;
  while ((int64_t(1) << c) < n) ++c;
  return c;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__device__ inline int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Packed binary32 pairs (sm_100 and later): fma.rn.f32x2 and mul.rn.f32x2 round
// each half exactly as fmaf and __fmul_rn do (IEEE, round to nearest even), at one
// issue slot per two lanes of work.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
// c = a * b + c, per half
__device__ __forceinline__ void f2_fma(uint64_t& c, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
}
// a * b, per half
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// min(a, b, c) in one instruction (sm_100 and later); like fminf, a NaN operand
// is ignored when another is a number
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
inline uint32_t next_pow2_u32(uint64_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

size_t elem_size(int dtype);

// ------------------------------------------------------------------ launchers
// (defined in the kernel .cu files; all enqueue on `s` and never synchronise)

// ingest: finite check, |x|^2, bounding box of x (ordered-encoded, [2][d])
void launch_ingest(const ch_set* X, cudaStream_t s);

// l2 embedding of X with G = Irwin-Hall Gaussian (k x d): Y [n][k] and the box
// of Y as P partial boxes [P][2][k] (ordered-encoded; P <= kMaxBoxParts), whose
// elementwise min / max is the box.  Returns P.
constexpr int kMaxBoxParts = 256;
int launch_project(const ch_set* X, uint64_t seed, int k, float* Y, uint32_t* box, uint32_t* status,
                   int sm_count, cudaStream_t s);

// Tables of one CrudeNN call (device): scales, shifts, multipliers
struct ScaleTables {
  int32_t* e_lo;         // [1] finest exponent
  float* inv_r;          // [L] 2^-e
  uint64_t* salt;        // [L] mix64((uint32)e ^ seed)
  float* shift;          // [dd][L] z_{e,j}, coordinate-major
  uint64_t* mult;        // [dd] odd multipliers
};

// computes e_top from the two boxes, each given as partial boxes [parts][2][dd]
// (or uses top_exp), then fills the tables; with zero (16-byte aligned), further
// blocks of the same launch set zero_bytes (a multiple of 16) there to zero; with
// left, left[0] = n_left (the count of points of A not yet resolved by a scale)
// and left[1 .. n_zero_words] = 0
void launch_scale_tables(const uint32_t* boxA, int partsA, const uint32_t* boxB, int partsB, int dd, int L,
                         int top_exp_in, uint64_t seed, ScaleTables t, int32_t* e_top_out, uint32_t* status,
                         cudaStream_t s, void* zero = nullptr, size_t zero_bytes = 0, int sm_count = 1,
                         unsigned long long* left = nullptr, int64_t n_left = 0, int n_zero_words = 0);

// hashed-space source of a set: DT-typed rows (l1) or the binary32 embedding (l2)
struct HashSrc {
  const void* base;
  int dtype;
  int64_t n;
  int dd;
  const float* scales;
};

struct HashTable {
  ulonglong2* slots;  // [nl][cap] : x = key (0 = empty), y = ~min b index
  uint32_t log_cap;
  // Scale-group control (left = NULL: none; every group runs forward).
  // left: points of A that no scale so far resolved.  The group's first kernel
  // (first != 0) turns it into the group's mode, mode[group], which its later
  // kernels read: nothing left (skip), more than rev_max left (forward: B into
  // the tables above), else reverse (below).
  unsigned long long* left;
  int32_t* mode;
  int group;
  int first;
  unsigned long long rev_max;  // 0: no reverse groups
  // reverse groups: small tables [nl][2^rev_log_cap] of the unresolved a's
  // buckets, cleared before the groups run
  ulonglong2* rev;
  uint32_t rev_log_cap;
};

// reverse groups hold at most this many scales
constexpr int kRevGroupMax = 16;

// zeroes the tables of nl scales (forward groups only)
void launch_table_clear(HashTable h, int nl, int sm_count, cudaStream_t s);
// bucket tables of the scales [L0, L0+nl) (one table of 2^log_cap slots per scale)
void launch_group_insert(HashSrc B, int L, int L0, int nl, ScaleTables t, HashTable h, uint32_t* status, int sm_count,
                         cudaStream_t s);
void launch_group_probe(HashSrc A, int L, int L0, int nl, ScaleTables t, HashTable h, int64_t* bidx,
                        uint8_t* level, int sm_count, cudaStream_t s);
// the reverse form of a scale group (its three kernels return unless the group's mode is reverse)
void launch_group_reverse(HashSrc A, HashSrc B, int L, int L0, int nl, ScaleTables t, HashTable h, int64_t* bidx,
                          uint8_t* level, uint32_t* status, int sm_count, cudaStream_t s);
void launch_keys_write(HashSrc X, int L, ScaleTables t, uint64_t* keys, cudaStream_t s);
// SimHash keys [L][n] of embedded rows Y [n][K] (K <= 64)
void launch_simhash_keys(const float* Y, int64_t n, int K, int L, uint64_t seed, uint64_t* keys, cudaStream_t s);

// radix-sort grouping (CH_GROUP_SORT): keys [L][nA] and [L][nB] -> bidx, level
size_t sort_group_workspace(int64_t nA, int64_t nB, int L);
bool sort_group_supported(int64_t nA, int64_t nB, int L);

// k x W CrudeNN (Section 3): structure r's window of W points per a, by the same
// sort, into cand[a * stride + r * W + q] (-1 past the retrieved points); level[a]
// = the finest scale any structure so far found a point at (set by r = 0)
constexpr int kWindowMax = 64;
size_t sort_window_workspace(int64_t nA, int64_t nB, int L);
void launch_sort_window(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L, int W, int r,
                        void* work, int32_t* cand, int stride, uint8_t* level, cudaStream_t s);
// D_a = min over a's candidates of the canonical distance, b(a) its argmin
// (smallest index on ties); with maxD, max_a D_a (ordered-encoded)
void launch_cand_dist(const ch_set* A, const ch_set* B, int metric, const int32_t* cand, int stride, int64_t* bidx,
                      float* D, uint32_t* maxD, cudaStream_t s);
void launch_sort_group(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L,
                       void* work, int64_t* bidx, uint8_t* level, cudaStream_t s);

// D_a = canonical d(a, B[b(a)]); with maxD non-null also max_a D_a (ordered-encoded;
// *maxD is cleared first unless keep_max)
void launch_crude_dist(const ch_set* A, const ch_set* B, int metric, const int64_t* bidx, float* D, uint32_t* maxD,
                       int sm_count, cudaStream_t s);

// CrudeNN of many pairs in one launch per step (batched estimates): every pair's
// scales fit one group of bucket tables, its hashed rows fit registers (dd <= 64)
// and A and B share one storage type.  Each kernel's blocks are cut into
// consecutive runs, one per pair (blk0[p] .. blk0[p + 1] - 1); a block finds its
// pair by binary search and then does exactly what the single-pair kernel's
// block of the same index does.
struct CrudePair {
  HashSrc A, B;                      // hashed rows of the two sets
  const uint32_t* boxA;              // [partsA][2][dd] partial boxes of A's hashed rows
  const uint32_t* boxB;
  int partsA, partsB;
  ScaleTables t;
  ulonglong2* slots;                 // [L][2^log_cap] bucket tables, zeroed before the launches
  uint32_t log_cap;
  int L, top_exp;
  uint64_t seed;
  const void* rawA;                  // the stored rows, for D_a
  const float* scA;
  const void* rawB;
  const float* scB;
  int d;
  int gx_insert, gx_probe, gx_dist;  // blocks per pair: insert (per scale), probe, crude distance
  int64_t* bidx;
  uint8_t* level;
  float* D;
  uint32_t* status;
};
// the pair whose run of blocks holds block b: the largest p with blk0[p] <= b
__device__ __forceinline__ int find_pair(const int* __restrict__ blk0, int np, int b) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&blk0[mid]) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// l2 embeddings of many sets of d <= 8 in one launch (batched estimates)
struct ProjSet {
  const void* X;
  const float* scales;
  int64_t n;
  uint64_t seed;
  float* Y;          // [n][k]
  uint32_t* box;     // [blocks of the set][2][k] partial boxes
  uint32_t* status;  // the set's status word (non-finite data)
};
// blocks (= partial boxes) of a set's small projection
int project_small_blocks(int64_t n, int sm_count);
void launch_project_small_batch(const ProjSet* S, const int* blk0, int ns, int blocks, int dtype, int d, int k,
                                cudaStream_t s);
// scale tables of every pair (a block per pair; e_top is not reported)
void launch_scale_tables_batch(const CrudePair* P, int np, cudaStream_t s);
// B into the tables at every scale, then A's probes: blk0 [np + 1] prefix of
// the per-pair block counts (insert: gx_insert * L, probe: gx_probe)
void launch_insert_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int dd, cudaStream_t s);
void launch_probe_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int dd, cudaStream_t s);
// D_a of every pair (G lanes per a, as launch_crude_dist's lane form; blocks gx_dist)
void launch_crude_dist_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int metric,
                             cudaStream_t s);
// lanes per a of the batched crude distance for dimension d
int crude_dist_lanes(int d);

// sampling
struct SampleWork {
  uint32_t* maxD;        // [1] ordered-encoded max
  uint64_t* blocksum;    // [nblocks]
  uint64_t* W;           // [1]
  int32_t* S;            // [1]
};
// the weight scan works in blocks of kSampleScanTile points (256 threads x 4)
constexpr int kSampleScanTile = 1024;
constexpr int64_t sample_blocks_c(int64_t nA) { return (nA + kSampleScanTile - 1) / kSampleScanTile; }
size_t sample_blocks(int64_t nA);
// D[0..n) = 1 (the uniform-sampling baseline's weights)
void launch_fill_ones(float* D, int64_t n, cudaStream_t s);

// weights and their prefix; max_ready: *sw.maxD already holds max_a D_a;
// local_prefix: leave prefix block-local (sw.blocksum then holds the blocks'
// exclusive offsets, which launch_draws takes as blockoff)
void launch_weights(const float* D, int64_t nA, uint64_t* w, uint64_t* prefix, SampleWork sw, cudaStream_t s,
                    bool max_ready = false, bool local_prefix = false);
// warp_search: a warp per draw (for a lone estimate, whose few draws are
// latency-bound) instead of a thread per draw (for many concurrent estimates)
void launch_draws(const uint64_t* prefix, int64_t nA, const uint64_t* W, int64_t T, uint64_t seed,
                  int64_t* idx, cudaStream_t s, const uint64_t* blockoff = nullptr, bool warp_search = false);

// optional CUDA events recorded around a stage's main kernel
struct KernelTimer {
  cudaEvent_t before = nullptr, after = nullptr;
  void start(cudaStream_t s) const {
    if (before) cudaEventRecord(before, s);
  }
  void stop(cudaStream_t s) const {
    if (after) cudaEventRecord(after, s);
  }
};

// canonical rerank of screened entries: part_s / part_i [parts][T][per] (score,
// first column or -1); an entry stands for columns first + o * stride, o < occ
constexpr int kRerankMaxCand = 1024;  // parts * per
constexpr int kRerankMaxOcc = 4;
void launch_rerank(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, const float* part_s,
                   const int32_t* part_i, int parts, int per, int occ, int stride, int R, float* min_d,
                   int64_t* argmin, cudaStream_t s);

// exact scan: per (sample, chunk) minima, then merge
struct ScanPart {
  float* val;
  int64_t* idx;
  int chunks;
};
void launch_scan_exact(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int metric, ScanPart part,
                       int sm_count, cudaStream_t s);
void launch_scan_merge(ScanPart part, int64_t T, const int64_t* qidx, float* min_d, int64_t* argmin,
                       cudaStream_t s);
int scan_exact_chunks(int64_t T, int64_t nB, int d, int dtype, int sm_count);

// ---- batched exact scan of small dimensions (d <= 4) over many pairs at once
constexpr int kBatchScanMaxD = 4;
struct SmallScanPair {
  const void* A;
  const float* scA;
  int64_t nA;
  const int64_t* qidx;  // [T] draws (< 0: none)
  int64_t T;
  const void* B;
  const float* scB;
  int64_t nB;
  unsigned long long* best;  // [T] min over B of canonical distance bits << 32, preset to all ones
};
struct SmallScanItem {
  int32_t pair;    // index into the pair list
  int32_t sblock;  // block of samples
  int64_t b0;      // first point of B of the item's chunk
};
// samples per item of the batched small scan
int small_scan_samples_per_item();
// one persistent launch over every item (all pairs of one storage type, metric
// and dimension d <= 4); each item's minimum distances fold into best[] by atomicMin
void launch_scan_small_batch(const SmallScanPair* pairs, const SmallScanItem* items, int64_t n_items,
                             int64_t chunk_len, int dtype, int metric, int d, int sm_count, cudaStream_t s);

// tensor-core screen + rerank (l2)
bool screen_supported(int screen, const ch_set* A, const ch_set* B);
// chunk_sms: the SM count the split of B into chunks aims to fill (the grid still
// spans up to sm_count SMs); concurrent batch lanes pass their share
size_t screen_workspace(int64_t T, int64_t nB, int d, int R, int sm_count, int chunk_sms, int screen);
void launch_screen_l2(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int screen, int R,
                      void* work, float* min_d, int64_t* argmin, uint32_t* status, int sm_count, int chunk_sms,
                      cudaStream_t s, const KernelTimer& timer, long long wait_cycles = 0);

// result block copied to the host at the end of a synchronising call
struct ResBlock {
  double eta;
  double D_total;
  uint64_t W;
  int32_t e_top;
  int32_t S;
  uint32_t status;   // call status bits
  uint32_t statusA;  // set A status bits
  uint32_t statusB;  // set B status bits
  uint32_t pad;
};

// what the combine's final pass copies into a result block (null fields skipped)
struct CollectArgs {
  ResBlock* res = nullptr;
  const uint32_t* statusA = nullptr;
  const uint32_t* statusB = nullptr;
  const int32_t* S = nullptr;
  const int32_t* e_top = nullptr;
  ResBlock* host = nullptr;  // pinned host page that also receives the finished block (no copy afterwards)
};

// combine: eta = (1/T) sum m_l W / w_{x_l} (binary64) and sum D (binary64).
// out must hold kCombineDoubles doubles: out[0] = eta, out[1] = sum D, then
// per-block partials.  The block count is fixed, so the summation order (and
// the result's bits) do not depend on the GPU.
constexpr int kCombineBlocks = 128;
constexpr int kCombineDoubles = 2 + 2 * kCombineBlocks;

// One pair of a batched call in the work lists of the batched sampling and
// combine kernels (device memory; one CTA per entry).
struct BatchItem {
  const float* D;    // [nA] crude distances
  uint64_t* w;       // [nA] weights
  uint64_t* prefix;  // [nA] inclusive prefix of w
  int64_t* idx;      // [T] draws
  const float* m;    // [T] sampled minima (the combine's input), or
  const unsigned long long* mpk;  // [T] the minima packed by the batched small scan (distance bits in the high word)
  ResBlock* res;     // the pair's result block (W, S, eta, D_total, set status words)
  const uint32_t* statusA;
  const uint32_t* statusB;
  int64_t nA, T;
  uint64_t seed;
};
// weights, their exact inclusive prefix, W and the T draws of every listed pair
// (the same integers as launch_weights + launch_draws)
void launch_batch_sample(const BatchItem* items, int64_t count, cudaStream_t s);
// eta and sum D of every listed pair, in the summation order of launch_combine
// (so the same bits), into its result block
void launch_batch_combine(const BatchItem* items, int64_t count, cudaStream_t s);
void launch_combine(const float* m, const int64_t* idx, const uint64_t* w, const uint64_t* W, int64_t T,
                    const float* D, int64_t nA, double* out, cudaStream_t s, CollectArgs collect = CollectArgs());
// sum of per-a minima (binary64): out[1] = sum (same layout as launch_combine)
void launch_sum_f32(const float* v, int64_t n, double* out, cudaStream_t s);

}  // namespace chx
