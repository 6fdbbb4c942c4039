// k_sort.cu -- CrudeNN grouping by a device radix sort (CH_GROUP_SORT).
//
// Entries (key, tag) of every scale: tag = isA<<31 | scale<<26 | index.  In the
// initial order each scale lists B (ascending index) before A.  A stable LSD
// radix sort by the 64-bit key (8 passes of 8 bits) and then by the scale
// (a 9th pass) leaves every (scale, key) run starting with its smallest-index
// B, followed by the rest of B and by A.  A segmented scan of run-head
// positions then gives each A entry its run head; when that head is a B, the
// entry proposes (scale, b) and an atomicMin of the packed pair over the
// scales keeps the smallest scale (Fig. 2, step 3).  Same b(a) as the bucket
// tables, by definition.
#include "common.cuh"

namespace chx {

namespace {

constexpr int kST = 256;               // threads per sort block
constexpr int kSItems = 32;            // rounds of kST entries per tile
constexpr int kSTile = kST * kSItems;  // 8192 entries per tile
constexpr int kSWarps = kST / 32;
constexpr int kIdxBits = 26;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1;
constexpr int kHeadPer = 16;                       // entries per thread in the head scan
constexpr int kHeadBlock = kST * kHeadPer;         // 4096 entries per head-scan block

__device__ inline uint32_t tag_scale(uint32_t t) { return (t >> kIdxBits) & 31u; }

__global__ void k_sort_build(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L,
                             uint64_t* key, uint32_t* tag) {
  pdl_entry();
  const int64_t N = nA + nB, total = N * L;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t l = i / N, p = i - l * N;
    const uint32_t sc = static_cast<uint32_t>(l) << kIdxBits;
    if (p < nB) {
      key[i] = keysB[l * nB + p];
      tag[i] = sc | static_cast<uint32_t>(p);
    } else {
      key[i] = keysA[l * nA + (p - nB)];
      tag[i] = 0x80000000u | sc | static_cast<uint32_t>(p - nB);
    }
  }
}

__device__ inline uint32_t sort_digit(uint64_t k, uint32_t t, int pass) {
  return pass < 8 ? static_cast<uint32_t>(k >> (8 * pass)) & 0xFFu : tag_scale(t);
}

// per-tile digit histogram, stored digit-major: hist[digit * ntiles + tile]
__global__ void __launch_bounds__(kST) k_sort_hist(const uint64_t* key, const uint32_t* tag, int64_t n, int pass,
                                                   uint32_t* hist, int ntiles) {
  pdl_entry();
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSTile;
  for (int r = 0; r < kSItems; ++r) {
    const int64_t i = base + r * kST + threadIdx.x;
    const bool ok = i < n;
    const uint32_t dg = ok ? sort_digit(key[i], tag[i], pass) : 256u;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
    if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[dg], __popc(peers));
  }
  __syncthreads();
  hist[size_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of the digit-major histogram (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* hist, int64_t M) {
  pdl_entry();
  __shared__ uint32_t s[1024];
  const int64_t per = (M + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = min(M, b + per);
  uint32_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += hist[i];
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - sum;
  for (int64_t i = b; i < e; ++i) {
    const uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// stable scatter: rounds in entry order, warps in order, lanes in order
__global__ void __launch_bounds__(kST) k_sort_scatter(const uint64_t* kin, const uint32_t* tin, uint64_t* kout,
                                                      uint32_t* tout, int64_t n, int pass, const uint32_t* hist,
                                                      int ntiles) {
  pdl_entry();
  __shared__ uint32_t off[256], run[256];
  __shared__ uint32_t wc[kSWarps][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  off[tid] = hist[size_t(tid) * ntiles + blockIdx.x];
  run[tid] = 0;
  const int64_t base = int64_t(blockIdx.x) * kSTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSItems; ++r) {
    for (int k = tid; k < kSWarps * 256; k += kST) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t i = base + r * kST + tid;
    const bool ok = i < n;
    uint64_t kv = 0;
    uint32_t tv = 0, dg = 256u;
    if (ok) {
      kv = kin[i];
      tv = tin[i];
      dg = sort_digit(kv, tv, pass);
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
    const uint32_t lrank = __popc(peers & lt);
    if (ok && lrank == 0) wc[warp][dg] = __popc(peers);
    __syncthreads();
    uint32_t total = 0;  // digit tid: exclusive prefix over warps
    for (int w = 0; w < kSWarps; ++w) {
      const uint32_t c = wc[w][tid];
      wc[w][tid] = total;
      total += c;
    }
    __syncthreads();
    if (ok) {
      const uint32_t pos = off[dg] + run[dg] + wc[warp][dg] + lrank;
      kout[pos] = kv;
      tout[pos] = tv;
    }
    __syncthreads();
    run[tid] += total;
  }
}

// run-head positions: hp[i] = last j <= i that starts a (scale, key) run, within
// this block (-1 if the block's prefix holds none); block_last = the block's last head
__global__ void __launch_bounds__(kST) k_sort_heads(const uint64_t* key, const uint32_t* tag, int64_t n, int32_t* hp,
                                                    int32_t* block_last) {
  pdl_entry();
  __shared__ int32_t s[kST];
  const int64_t b = int64_t(blockIdx.x) * kHeadBlock + int64_t(threadIdx.x) * kHeadPer;
  int32_t cur = -1;
  int32_t loc[kHeadPer];
#pragma unroll
  for (int j = 0; j < kHeadPer; ++j) {
    const int64_t i = b + j;
    if (i < n) {
      const bool head = i == 0 || key[i] != key[i - 1] || tag_scale(tag[i]) != tag_scale(tag[i - 1]);
      if (head) cur = static_cast<int32_t>(i);
    }
    loc[j] = cur;
  }
  s[threadIdx.x] = cur;
  __syncthreads();
  for (int o = 1; o < kST; o <<= 1) {  // inclusive max-scan over threads
    const int32_t v = threadIdx.x >= o ? s[threadIdx.x - o] : -1;
    __syncthreads();
    s[threadIdx.x] = max(s[threadIdx.x], v);
    __syncthreads();
  }
  const int32_t before = threadIdx.x > 0 ? s[threadIdx.x - 1] : -1;
#pragma unroll
  for (int j = 0; j < kHeadPer; ++j) {
    const int64_t i = b + j;
    if (i < n) hp[i] = max(loc[j], before);
  }
  if (threadIdx.x == kST - 1) block_last[blockIdx.x] = s[kST - 1];
}

// exclusive max-scan of the blocks' last heads (one block)
__global__ void __launch_bounds__(1024) k_sort_carry(int32_t* block_last, int64_t nb) {
  pdl_entry();
  __shared__ int32_t s[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = -1;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
    const int64_t i = c0 + threadIdx.x;
    const int32_t v = i < nb ? block_last[i] : -1;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int32_t u = threadIdx.x >= o ? s[threadIdx.x - o] : -1;
      __syncthreads();
      s[threadIdx.x] = max(s[threadIdx.x], u);
      __syncthreads();
    }
    const int32_t c = carry;
    if (i < nb) block_last[i] = max(c, threadIdx.x > 0 ? s[threadIdx.x - 1] : -1);
    __syncthreads();
    if (threadIdx.x == 1023) carry = max(c, s[1023]);
    __syncthreads();
  }
}

// each A entry whose run starts with a B proposes (scale, b)
__global__ void k_sort_assign(const uint32_t* tag, const int32_t* hp, const int32_t* carry, int64_t n,
                              unsigned long long* packed) {
  pdl_entry();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t t = tag[i];
    if (!(t & 0x80000000u)) continue;
    int32_t h = hp[i];
    if (h < 0) h = carry[i / kHeadBlock];
    const uint32_t ht = tag[h];
    if (ht & 0x80000000u) continue;  // the run holds no b
    const unsigned long long cand = (static_cast<unsigned long long>(tag_scale(t)) << 32) | (ht & kIdxMask);
    atomicMin(&packed[t & kIdxMask], cand);
  }
}

__global__ void k_sort_finish(const unsigned long long* packed, int64_t nA, int L, int64_t* bidx, uint8_t* level) {
  pdl_entry();
  const int64_t a = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a >= nA) return;
  const unsigned long long p = packed[a];
  if (p == ~0ull) {
    bidx[a] = 0;
    level[a] = static_cast<uint8_t>(L);
  } else {
    bidx[a] = static_cast<int64_t>(p & 0xFFFFFFFFull);
    level[a] = static_cast<uint8_t>(p >> 32);
  }
}

struct SortWork {
  uint64_t *k0, *k1;
  uint32_t *t0, *t1, *hist;
  int32_t *hp, *blast;
  unsigned long long* packed;
  int ntiles;
  int64_t nhb;
};

SortWork carve_sort(void* work, int64_t nA, int64_t nB, int L) {
  const int64_t n = (nA + nB) * L;
  SortWork w;
  w.ntiles = static_cast<int>(ceil_div(n, kSTile));
  w.nhb = ceil_div(n, kHeadBlock);
  char* p = static_cast<char*>(work);
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) & ~size_t(255);
    return q;
  };
  w.k0 = reinterpret_cast<uint64_t*>(take(n * 8));
  w.k1 = reinterpret_cast<uint64_t*>(take(n * 8));
  w.t0 = reinterpret_cast<uint32_t*>(take(n * 4));
  w.t1 = reinterpret_cast<uint32_t*>(take(n * 4));
  w.hist = reinterpret_cast<uint32_t*>(take(size_t(256) * w.ntiles * 4));
  w.hp = reinterpret_cast<int32_t*>(take(n * 4));
  w.blast = reinterpret_cast<int32_t*>(take(w.nhb * 4));
  w.packed = reinterpret_cast<unsigned long long*>(take(nA * 8));
  return w;
}

}  // namespace

size_t sort_group_workspace(int64_t nA, int64_t nB, int L) {
  const int64_t n = (nA + nB) * L;
  const size_t r = 256;
  return size_t(n) * 8 * 2 + size_t(n) * 4 * 3 + size_t(256) * ceil_div(n, kSTile) * 4 +
         size_t(ceil_div(n, kHeadBlock)) * 4 + size_t(nA) * 8 + 8 * r;
}

bool sort_group_supported(int64_t nA, int64_t nB, int L) {
  return nA < (int64_t(1) << kIdxBits) && nB < (int64_t(1) << kIdxBits) && L <= 32 &&
         (nA + nB) * L < (int64_t(1) << 31);
}

// the stable sort and the run heads; returns the sorted tags
static const uint32_t* sort_core(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L,
                                 const SortWork& w, cudaStream_t s) {
  const int64_t n = (nA + nB) * L;
  const int gb = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 152 * 16));
  launch_k(k_sort_build, gb, 256, 0, s, keysA, nA, keysB, nB, L, w.k0, w.t0);
  launch_check("sort_build");
  uint64_t *kin = w.k0, *kout = w.k1;
  uint32_t *tin = w.t0, *tout = w.t1;
  for (int pass = 0; pass < 9; ++pass) {
    launch_k(k_sort_hist, w.ntiles, kST, 0, s, kin, tin, n, pass, w.hist, w.ntiles);
    launch_check("sort_hist");
    launch_k(k_sort_scan, 1, 1024, 0, s, w.hist, int64_t(256) * w.ntiles);
    launch_check("sort_scan");
    launch_k(k_sort_scatter, w.ntiles, kST, 0, s, kin, tin, kout, tout, n, pass, w.hist, w.ntiles);
    launch_check("sort_scatter");
    std::swap(kin, kout);
    std::swap(tin, tout);
  }
  launch_k(k_sort_heads, static_cast<int>(w.nhb), kST, 0, s, kin, tin, n, w.hp, w.blast);
  launch_check("sort_heads");
  launch_k(k_sort_carry, 1, 1024, 0, s, w.blast, w.nhb);
  launch_check("sort_carry");
  return tin;
}

void launch_sort_group(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L, void* work,
                       int64_t* bidx, uint8_t* level, cudaStream_t s) {
  if (nA == 0) return;
  const int64_t n = (nA + nB) * L;
  SortWork w = carve_sort(work, nA, nB, L);
  const uint32_t* tin = sort_core(keysA, nA, keysB, nB, L, w, s);
  const int gb = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 152 * 16));
  CHX_CUDA(cudaMemsetAsync(w.packed, 0xFF, size_t(nA) * 8, s));
  launch_k(k_sort_assign, gb, 256, 0, s, tin, w.hp, w.blast, n, w.packed);
  launch_check("sort_assign");
  launch_k(k_sort_finish, static_cast<int>(ceil_div(nA, 256)), 256, 0, s, w.packed, nA, L, bidx, level);
  launch_check("sort_finish");
}

// ------------------------------------------------------------------ k x W window
namespace {

// pos[scale * nA + a] = sorted position of a's entry at that scale
__global__ void k_sort_pos(const uint32_t* tag, int64_t n, int64_t nA, int32_t* pos) {
  pdl_entry();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t t = tag[i];
    if (t & 0x80000000u) pos[int64_t(tag_scale(t)) * nA + (t & kIdxMask)] = static_cast<int32_t>(i);
  }
}

// Structure r's window for each a: scales in increasing order; in a's run the B
// entries come first, in increasing index (initial order + stable sort), so the
// first W distinct of them, over the scales, are read off directly.  A structure
// that finds nothing contributes B[0].
__global__ void k_window(const uint32_t* tag, const int32_t* hp, const int32_t* carry, const int32_t* pos,
                         int64_t n, int64_t nA, int L, int W, int r, int stride, int32_t* cand, uint8_t* level) {
  pdl_entry();
  const int64_t a = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a >= nA) return;
  int32_t taken[kWindowMax];
  int cnt = 0, first = L;
  for (int l = 0; l < L && cnt < W; ++l) {
    const int64_t i = pos[int64_t(l) * nA + a];
    int64_t j = hp[i];
    if (j < 0) j = carry[i / kHeadBlock];
    for (; j < n && cnt < W; ++j) {
      const uint32_t t = tag[j];
      if (t & 0x80000000u) break;  // the run's B entries are over
      const int32_t b = static_cast<int32_t>(t & kIdxMask);
      bool seen = false;
      for (int q = 0; q < cnt; ++q) seen |= taken[q] == b;
      if (!seen) {
        taken[cnt++] = b;
        first = min(first, l);
      }
    }
  }
  if (cnt == 0) taken[cnt++] = 0;
  int32_t* out = cand + a * stride + int64_t(r) * W;
  for (int q = 0; q < W; ++q) out[q] = q < cnt ? taken[q] : -1;
  if (r == 0 || first < level[a]) level[a] = static_cast<uint8_t>(first);
}

}  // namespace

size_t sort_window_workspace(int64_t nA, int64_t nB, int L) {
  return sort_group_workspace(nA, nB, L) + size_t(nA) * L * 4 + 256;
}

void launch_sort_window(const uint64_t* keysA, int64_t nA, const uint64_t* keysB, int64_t nB, int L, int W, int r,
                        void* work, int32_t* cand, int stride, uint8_t* level, cudaStream_t s) {
  if (nA == 0) return;
  CHX_CHECK(W >= 1 && W <= kWindowMax, CH_EINVAL, "window must be in 1..64");
  const int64_t n = (nA + nB) * L;
  SortWork w = carve_sort(work, nA, nB, L);
  int32_t* pos = reinterpret_cast<int32_t*>(static_cast<char*>(work) +
                                            ((sort_group_workspace(nA, nB, L) + 255) & ~size_t(255)));
  const uint32_t* tin = sort_core(keysA, nA, keysB, nB, L, w, s);
  const int gb = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 152 * 16));
  launch_k(k_sort_pos, gb, 256, 0, s, tin, n, nA, pos);
  launch_check("sort_pos");
  launch_k(k_window, static_cast<int>(ceil_div(nA, 128)), 128, 0, s, tin, w.hp, w.blast, pos, n, nA, L, W, r, stride, cand,
                                                               level);
  launch_check("window");
}

}  // namespace chx
