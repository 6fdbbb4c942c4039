// k_sample.cu -- importance sampling (Fig. 1, steps 2-3) and the estimate
// (Fig. 1, step 4) on the device.
//
// Pr[x = a] = D_a / D is realised with 64-bit fixed-point weights
// w_a = ceil(D_a 2^S), S = 62 - ceil(log2 nA) - e_M (max D_a < 2^e_M), an exact
// integer inclusive prefix, and inverse-CDF draws from 128-bit Philox words.
#include "common.cuh"

namespace chx {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // elements per block
static_assert(kScanTile == kSampleScanTile, "the weight-scan tile is declared in common.cuh");

size_t sample_blocks(int64_t nA) { return static_cast<size_t>(sample_blocks_c(nA)); }

__global__ void k_max_d(const float* D, int64_t n, uint32_t* maxD) {
  pdl_entry();
  uint32_t m = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = max(m, ord_enc(D[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxD, m);
}

// A non-finite maximum (D holding Inf or NaN, outside the contract) is treated
// like an all-zero D: W = 0, every weight 0 and every draw -1.
__device__ inline int weight_shift(const uint32_t* maxD, int64_t nA, bool* zero) {
  const float M = ord_dec(*maxD);
  if (!(M > 0.0f) || !(M <= 3.402823466e38f)) {
    *zero = true;
    return 0;
  }
  *zero = false;
  int eM;
  frexp(static_cast<double>(M), &eM);
  return 62 - ceil_log2_i64(nA) - eM;
}

// ceil(Da 2^S) for a finite Da > 0, exactly, from the bits of Da (the same
// integer as ceil(ldexp(double(Da), S)), without the FP64 pipe): Da = m 2^(e-150)
// with a 24-bit m, so the scaled value is m shifted by e - 150 + S, rounded up.
// S keeps every weight below 2^63, so a left shift never overflows.
__device__ __forceinline__ uint64_t ceil_scaled(float Da, int S) {
  const uint32_t bits = __float_as_uint(Da);
  int e = static_cast<int>((bits >> 23) & 0xFFu);
  uint64_t m = bits & 0x7FFFFFu;
  if (e == 0)
    e = 1;  // subnormal
  else
    m |= 0x800000u;
  const int sh = e - 150 + S;
  if (sh >= 0) return m << sh;
  const int k = -sh;
  if (k >= 32) return 1;  // 0 < m 2^-k < 1
  return (m + (uint64_t(1) << k) - 1) >> k;
}

// block-local inclusive scan of u64 weights; writes w, the local prefix and the block sum
__global__ void __launch_bounds__(kScanThreads) k_weights(const float* D, int64_t nA, const uint32_t* maxD,
                                                          uint64_t* w, uint64_t* prefix, uint64_t* blocksum,
                                                          int32_t* S_out) {
  pdl_entry();
  __shared__ uint64_t s_warp[kScanThreads / 32];
  bool zero;
  const int S = weight_shift(maxD, nA, &zero);
  if (blockIdx.x == 0 && threadIdx.x == 0) *S_out = S;
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
  uint64_t v[kScanItems];
  uint64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t a = base + i;
    uint64_t wa = 0;
    if (a < nA && !zero) {
      const float Da = D[a];
      if (Da > 0.0f) wa = ceil_scaled(Da, S);
    }
    if (a < nA) w[a] = wa;
    run += wa;
    v[i] = run;
  }
  // exclusive offset of this thread within the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint64_t woff = 0;
  for (int i = 0; i < warp; ++i) woff += s_warp[i];
  const uint64_t off = woff + x - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t a = base + i;
    if (a < nA) prefix[a] = v[i] + off;
  }
  if (threadIdx.x == kScanThreads - 1) blocksum[blockIdx.x] = off + run;
}

// exclusive scan of the block sums (one block, sequential chunks of 1024)
__global__ void k_scan_blocksums(uint64_t* blocksum, int64_t nb, uint64_t* W) {
  pdl_entry();
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const uint64_t v = i < nb ? blocksum[i] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint64_t woff = 0;
    for (int k = 0; k < warp; ++k) woff += s_warp[k];
    const uint64_t carry = s_carry;
    if (i < nb) blocksum[i] = carry + woff + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + woff + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *W = s_carry;
}

__global__ void k_add_offsets(uint64_t* prefix, int64_t nA, const uint64_t* blockoff) {
  pdl_entry();
  const int64_t a = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a < nA) prefix[a] += blockoff[a / kScanTile];
}

__global__ void k_fill_ones(float* D, int64_t n) {
  pdl_entry();
  const int64_t a = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a < n) D[a] = 1.0f;
}

void launch_fill_ones(float* D, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  launch_k(k_fill_ones, static_cast<int>(ceil_div(n, 256)), 256, 0, s, D, n);
  launch_check("fill_ones");
}

void launch_weights(const float* D, int64_t nA, uint64_t* w, uint64_t* prefix, SampleWork sw, cudaStream_t s,
                    bool max_ready, bool local_prefix) {
  if (nA == 0) {
    CHX_CUDA(cudaMemsetAsync(sw.W, 0, sizeof(uint64_t), s));
    CHX_CUDA(cudaMemsetAsync(sw.S, 0, sizeof(int32_t), s));
    return;
  }
  if (!max_ready) {
    CHX_CUDA(cudaMemsetAsync(sw.maxD, 0, sizeof(uint32_t), s));
    const int gmax = static_cast<int>(std::min<int64_t>(ceil_div(nA, 256), 152 * 4));
    launch_k(k_max_d, gmax, 256, 0, s, D, nA, sw.maxD);
    launch_check("max_d");
  }
  const int64_t nb = static_cast<int64_t>(sample_blocks(nA));
  launch_k(k_weights, static_cast<int>(nb), kScanThreads, 0, s, D, nA, sw.maxD, w, prefix, sw.blocksum, sw.S);
  launch_check("weights");
  launch_k(k_scan_blocksums, 1, 1024, 0, s, sw.blocksum, nb, sw.W);
  launch_check("scan_blocksums");
  if (nb > 1 && !local_prefix) {
    launch_k(k_add_offsets, static_cast<int>(ceil_div(nA, 256)), 256, 0, s, prefix, nA, sw.blocksum);
    launch_check("add_offsets");
  }
}

// x_l = first a with prefix_a > floor(u W / 2^128), u = Philox(l_lo, l_hi, 3, 0).
// With blockoff, prefix holds the block-local inclusive sums of kScanTile-point
// blocks and blockoff their exclusive offsets: the search first finds the block
// whose inclusive end exceeds t, then the point inside it -- the same a.
// First index in [lo, hi) whose predicate holds (monotone: false ... false
// true ... true), or hi: a 32-ary search by one warp.  Each round the lanes
// test the last element of 32 equal segments and the first true segment is
// kept, so a range of n takes about log32(n) dependent loads instead of
// log2(n).  The whole warp calls it with the same range.
template <class Pred>
__device__ __forceinline__ int64_t warp_first_true(int64_t lo, int64_t hi, int lane, Pred pred) {
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t probe = min(hi - 1, lo + (lane + 1) * step - 1);
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred(probe));
    if (bal == 0) return hi;
    const int j = __ffs(bal) - 1;
    const int64_t nlo = lo + int64_t(j) * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  const int64_t e = lo + lane;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, e < hi && pred(e));
  return bal == 0 ? hi : lo + (__ffs(bal) - 1);
}

// t = floor(u W) for draw l, u = Philox(l, 3) read as a 128-bit fraction
__device__ __forceinline__ uint64_t draw_point(int64_t l, uint64_t seed, uint64_t W) {
  const P4 u = philox10(P4{uint32_t(l), uint32_t(uint64_t(l) >> 32), 3u, 0u}, uint32_t(seed), uint32_t(seed >> 32));
  const uint64_t ulo = (uint64_t(u.y) << 32) | u.x;
  const uint64_t uhi = (uint64_t(u.w) << 32) | u.z;
  const uint64_t plo_hi = __umul64hi(ulo, W);
  const uint64_t phi_lo = uhi * W;
  const uint64_t phi_hi = __umul64hi(uhi, W);
  const uint64_t mid = phi_lo + plo_hi;
  return phi_hi + (mid < phi_lo ? 1 : 0);
}

// Draw l by one thread: x_l = the first a whose inclusive prefix exceeds t,
// by binary search (the form for many draws, where loads in flight, not their
// latency, set the pace)
__global__ void k_draws(const uint64_t* prefix, int64_t nA, const uint64_t* Wp, int64_t T, uint64_t seed,
                        int64_t* idx, const uint64_t* blockoff) {
  pdl_entry();
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= T) return;
  const uint64_t W = *Wp;
  if (W == 0) {
    idx[l] = -1;
    return;
  }
  const uint64_t t = draw_point(l, seed, W);
  if (blockoff) {
    const int64_t nb = ceil_div_dev(nA, kScanTile);
    int64_t lo = 0, hi = nb;  // first block whose inclusive end (next block's offset, or W) exceeds t
    while (lo < hi) {
      const int64_t m = lo + ((hi - lo) >> 1);
      const uint64_t end = m + 1 < nb ? blockoff[m + 1] : W;
      if (end > t)
        hi = m;
      else
        lo = m + 1;
    }
    const uint64_t off = blockoff[lo];
    int64_t a0 = lo * kScanTile, a1 = min(nA, a0 + kScanTile);
    while (a0 < a1) {  // first a in the block with off + local prefix > t
      const int64_t m = a0 + ((a1 - a0) >> 1);
      if (off + prefix[m] > t)
        a1 = m;
      else
        a0 = m + 1;
    }
    idx[l] = a0;
    return;
  }
  int64_t lo = 0, hi = nA;  // first a with prefix[a] > t
  while (lo < hi) {
    const int64_t m = lo + ((hi - lo) >> 1);
    if (prefix[m] > t)
      hi = m;
    else
      lo = m + 1;
  }
  idx[l] = lo;
}

// Draw l by one warp with the 32-ary search: about 4 dependent loads instead of
// 17, for few draws, where their latency sets the pace
__global__ void k_draws_warp(const uint64_t* prefix, int64_t nA, const uint64_t* Wp, int64_t T, uint64_t seed,
                             int64_t* idx, const uint64_t* blockoff) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t l = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (l >= T) return;  // whole warps
  const uint64_t W = *Wp;
  if (W == 0) {
    if (lane == 0) idx[l] = -1;
    return;
  }
  const uint64_t t = draw_point(l, seed, W);
  int64_t a;
  if (blockoff) {
    // the first block whose inclusive end (the next block's offset, or W) exceeds
    // t, then the first a in it with offset + local prefix > t
    const int64_t nb = ceil_div_dev(nA, kScanTile);
    const int64_t blk = warp_first_true(0, nb, lane, [&](int64_t m) {
      const uint64_t end = m + 1 < nb ? blockoff[m + 1] : W;
      return end > t;
    });
    const uint64_t off = blockoff[blk];
    const int64_t a0 = blk * kScanTile, a1 = min(nA, a0 + kScanTile);
    a = warp_first_true(a0, a1, lane, [&](int64_t m) { return off + prefix[m] > t; });
  } else {
    a = warp_first_true(0, nA, lane, [&](int64_t m) { return prefix[m] > t; });
  }
  if (lane == 0) idx[l] = a;
}

void launch_draws(const uint64_t* prefix, int64_t nA, const uint64_t* W, int64_t T, uint64_t seed, int64_t* idx,
                  cudaStream_t s, const uint64_t* blockoff, bool warp_search) {
  if (T == 0) return;
  // a warp per draw for a lone estimate of up to 16384 draws (100k x 128: 2 us
  // less); a thread per draw otherwise, where the warp form's extra loads cost
  // throughput (4096 concurrent pairs of d = 3, l1: 114 vs 128 ms per batch)
  if (warp_search && T <= 16384)
    launch_k(k_draws_warp, static_cast<int>(ceil_div(T, 8)), 256, 0, s, prefix, nA, W, T, seed, idx, blockoff);
  else
    launch_k(k_draws, static_cast<int>(ceil_div(T, 256)), 256, 0, s, prefix, nA, W, T, seed, idx, blockoff);
  launch_check("draws");
}

// ------------------------------------------------------------------ combine
// Two fixed-shape passes (kCombineBlocks blocks of 256, then one block), so the
// binary64 summation order is the same on every GPU:
//   out[0] = (1/T) sum_l m_l W / w_{x_l};  out[1] = sum_a D_a.
// Block b sums the contiguous slices [b*len, (b+1)*len) of the samples and of D.
__device__ inline void block_sum2(double& a, double& b, double* sa, double* sb) {
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sa[threadIdx.x] += sa[threadIdx.x + st];
      sb[threadIdx.x] += sb[threadIdx.x + st];
    }
    __syncthreads();
  }
  a = sa[0];
  b = sb[0];
}

// the result block from the summed partials (thread 0)
__device__ inline void combine_write(double a, double b, const uint64_t* Wp, int64_t T, double* out,
                                     const CollectArgs& c) {
  const uint64_t W = Wp ? *Wp : 0;
  out[0] = (W != 0 && T > 0) ? a / static_cast<double>(T) : 0.0;
  out[1] = b;
  if (c.res) {
    c.res->eta = out[0];
    c.res->D_total = b;
    c.res->W = W;
    if (c.statusA) c.res->statusA = *c.statusA;
    if (c.statusB) c.res->statusB = *c.statusB;
    if (c.S) c.res->S = *c.S;
    if (c.e_top) c.res->e_top = *c.e_top;
    if (c.host) {  // the whole block, status words included, straight into host memory
      *c.host = *c.res;
      __threadfence_system();
    }
  }
}

// With ticket (a zeroed counter): the block that finishes last also sums the
// kCombineBlocks partials, with the same tree as k_combine_final (256 threads,
// the upper half adding exact zeros), so one launch does both passes.
__global__ void __launch_bounds__(256) k_combine_part(const float* m, const int64_t* idx, const uint64_t* w,
                                                      const uint64_t* Wp, int64_t T, const float* D, int64_t nA,
                                                      double* out, uint32_t* ticket, CollectArgs collect) {
  pdl_entry();
  __shared__ double s_a[256], s_b[256];
  __shared__ bool s_last;
  const uint64_t W = Wp ? *Wp : 0;
  const int64_t lt = ceil_div_dev(T, kCombineBlocks), la = ceil_div_dev(nA, kCombineBlocks);
  double acc = 0.0, accD = 0.0;
  if (W != 0) {
    const double Wd = static_cast<double>(W);
    const int64_t end = min(T, (blockIdx.x + 1) * lt);
    for (int64_t l = blockIdx.x * lt + threadIdx.x; l < end; l += blockDim.x)
      acc += static_cast<double>(m[l]) * (Wd / static_cast<double>(w[idx[l]]));
  }
  if (D) {
    const int64_t end = min(nA, (blockIdx.x + 1) * la);
    for (int64_t a = blockIdx.x * la + threadIdx.x; a < end; a += blockDim.x) accD += static_cast<double>(D[a]);
  }
  block_sum2(acc, accD, s_a, s_b);
  if (threadIdx.x == 0) {
    out[2 + 2 * blockIdx.x] = acc;
    out[3 + 2 * blockIdx.x] = accD;
  }
  if (!ticket) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == kCombineBlocks - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  if (threadIdx.x < kCombineBlocks) {
    a = __ldcg(&out[2 + 2 * threadIdx.x]);
    b = __ldcg(&out[3 + 2 * threadIdx.x]);
  }
  __syncthreads();  // s_a / s_b are reused
  block_sum2(a, b, s_a, s_b);
  if (threadIdx.x == 0) combine_write(a, b, Wp, T, out, collect);
}

__global__ void __launch_bounds__(kCombineBlocks) k_combine_final(const uint64_t* Wp, int64_t T, double* out,
                                                                  CollectArgs c) {
  pdl_entry();
  __shared__ double s_a[kCombineBlocks], s_b[kCombineBlocks];
  double a = out[2 + 2 * threadIdx.x], b = out[3 + 2 * threadIdx.x];
  block_sum2(a, b, s_a, s_b);
  if (threadIdx.x == 0) combine_write(a, b, Wp, T, out, c);
}

void launch_combine(const float* m, const int64_t* idx, const uint64_t* w, const uint64_t* W, int64_t T,
                    const float* D, int64_t nA, double* out, cudaStream_t s, CollectArgs collect) {
  if (collect.res) {  // the result block's spare word, zeroed with the block, counts the finished blocks
    launch_k(k_combine_part, kCombineBlocks, 256, 0, s, m, idx, w, W, T, D, nA, out, &collect.res->pad, collect);
    launch_check("combine");
    return;
  }
  launch_k(k_combine_part, kCombineBlocks, 256, 0, s, m, idx, w, W, T, D, nA, out, static_cast<uint32_t*>(nullptr),
           collect);
  launch_check("combine_part");
  launch_k(k_combine_final, 1, kCombineBlocks, 0, s, W, T, out, collect);
  launch_check("combine_final");
}

// ------------------------------------------------------------------ batched work lists
// One CTA per listed pair (a work list of BatchItem): the pairs of a batched call
// take their weights, prefix and draws in one launch, and their combine in
// another, instead of five launches each.

constexpr int kBatchThreads = 1024;

// block-wide max of non-negative ordered-encoded values (every thread calls it)
__device__ inline uint32_t block_max_u32(uint32_t v, uint32_t* s_w) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  v = 0;
  for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) v = max(v, s_w[i]);
  __syncthreads();
  return v;
}

// Per pair: S from max D (as k_max_d + weight_shift), w_a = ceil(D_a 2^S), the
// inclusive prefix in chunks of blockDim x kScanItems points carried across
// chunks (exact integers, so any grouping gives the same sums), W, then the draws
// by binary search over the whole prefix.
__global__ void __launch_bounds__(kBatchThreads) k_batch_sample(const BatchItem* items) {
  pdl_entry();
  __shared__ uint32_t s_m[32];
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  const BatchItem it = items[blockIdx.x];
  const int64_t nA = it.nA;
  uint32_t mx = 0;
  for (int64_t a = threadIdx.x; a < nA; a += blockDim.x) mx = max(mx, ord_enc(it.D[a]));
  const uint32_t maxD = block_max_u32(mx, s_m);
  bool zero;
  const int S = weight_shift(&maxD, nA, &zero);
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = int64_t(blockDim.x) * kScanItems;
  for (int64_t c0 = 0; c0 < nA; c0 += tile) {
    const int64_t base = c0 + int64_t(threadIdx.x) * kScanItems;
    uint64_t v[kScanItems];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t a = base + i;
      uint64_t wa = 0;
      if (a < nA && !zero) {
        const float Da = it.D[a];
        if (Da > 0.0f) wa = ceil_scaled(Da, S);
      }
      if (a < nA) it.w[a] = wa;
      run += wa;
      v[i] = run;
    }
    uint64_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint64_t woff = 0;
    for (int i = 0; i < warp; ++i) woff += s_warp[i];
    const uint64_t carry = s_carry;
    const uint64_t off = carry + woff + x - run;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t a = base + i;
      if (a < nA) it.prefix[a] = v[i] + off;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = off + run;
    __syncthreads();
  }
  const uint64_t W = nA > 0 ? s_carry : 0;
  if (threadIdx.x == 0) {
    it.res->W = W;
    it.res->S = nA > 0 ? S : 0;
  }
  // the prefix written above is read back by other threads of this CTA
  __threadfence_block();
  __syncthreads();
  for (int64_t l = threadIdx.x; l < it.T; l += blockDim.x) {
    if (W == 0) {
      it.idx[l] = -1;
      continue;
    }
    const uint64_t t = draw_point(l, it.seed, W);
    int64_t lo = 0, hi = nA;  // first a with prefix[a] > t
    while (lo < hi) {
      const int64_t m = lo + ((hi - lo) >> 1);
      if (it.prefix[m] > t)
        hi = m;
      else
        lo = m + 1;
    }
    it.idx[l] = lo;
  }
}

// Per pair, 256 threads: the kCombineBlocks partial sums of k_combine_part (block
// b's thread t sums the strided elements of slice b, then the block's tree), and
// their final tree with the upper half of the threads adding zeros: the same
// binary64 operations in the same order, so the same bits.
__global__ void __launch_bounds__(256) k_batch_combine(const BatchItem* items) {
  pdl_entry();
  __shared__ double s_a[256], s_b[256];
  __shared__ double p_a[kCombineBlocks], p_b[kCombineBlocks];
  const BatchItem it = items[blockIdx.x];
  const uint64_t W = it.res->W;
  const int64_t T = it.T, nA = it.nA;
  const int64_t lt = ceil_div_dev(T, kCombineBlocks), la = ceil_div_dev(nA, kCombineBlocks);
  const double Wd = static_cast<double>(W);
  for (int b = 0; b < kCombineBlocks; ++b) {
    double acc = 0.0, accD = 0.0;
    if (W != 0) {
      const int64_t end = min(T, (b + 1) * lt);
      for (int64_t l = b * lt + threadIdx.x; l < end; l += blockDim.x) {
        const float ml = it.mpk ? __uint_as_float(static_cast<uint32_t>(it.mpk[l] >> 32)) : it.m[l];
        acc += static_cast<double>(ml) * (Wd / static_cast<double>(it.w[it.idx[l]]));
      }
    }
    const int64_t endA = min(nA, (b + 1) * la);
    for (int64_t a = b * la + threadIdx.x; a < endA; a += blockDim.x) accD += static_cast<double>(it.D[a]);
    block_sum2(acc, accD, s_a, s_b);
    if (threadIdx.x == 0) {
      p_a[b] = acc;
      p_b[b] = accD;
    }
    __syncthreads();  // s_a / s_b are reused
  }
  double a = 0.0, bsum = 0.0;
  if (threadIdx.x < kCombineBlocks) {
    a = p_a[threadIdx.x];
    bsum = p_b[threadIdx.x];
  }
  __syncthreads();
  block_sum2(a, bsum, s_a, s_b);
  if (threadIdx.x == 0) {
    ResBlock* r = it.res;
    r->eta = (W != 0 && T > 0) ? a / static_cast<double>(T) : 0.0;
    r->D_total = bsum;
    if (it.statusA) r->statusA = *it.statusA;
    if (it.statusB) r->statusB = *it.statusB;
  }
}

void launch_batch_sample(const BatchItem* items, int64_t count, cudaStream_t s) {
  if (count == 0) return;
  launch_k(k_batch_sample, static_cast<int>(count), kBatchThreads, 0, s, items);
  launch_check("batch_sample");
}

void launch_batch_combine(const BatchItem* items, int64_t count, cudaStream_t s) {
  if (count == 0) return;
  launch_k(k_batch_combine, static_cast<int>(count), 256, 0, s, items);
  launch_check("batch_combine");
}

void launch_sum_f32(const float* v, int64_t n, double* out, cudaStream_t s) {
  // out[1] = sum v (binary64), out[0] = 0: the combine reduction with no samples
  launch_combine(nullptr, nullptr, nullptr, nullptr, 0, v, n, out, s);
}

}  // namespace chx
