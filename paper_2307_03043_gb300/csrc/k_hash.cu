// k_hash.cu -- CrudeNN on the device (Fig. 2 of the paper): set ingest, the
// l2 -> l1 Gaussian embedding, the shifted grids at every scale, bucket
// tables of B probed by A in increasing scale order, and D_a = d(a, b(a)).
#include <cstring>
#include <type_traits>

#include "tma.cuh"

namespace chx {

size_t elem_size(int dtype) { return dtype == CH_F32 ? 4 : dtype == CH_BF16 ? 2 : 1; }

// ------------------------------------------------------------------ ingest
// One warp per row: finite check and per-coordinate min/max of x (the l1 hashed
// space's bounding box).  CB = column blocks of 32 kept in registers (0 =
// shared-memory atomics for large d).
template <int DT, int CB>
__global__ void __launch_bounds__(256) k_ingest(const void* X, const float* scales, int64_t n, int d,
                                                float* norms, uint32_t* box, uint32_t* status) {
  pdl_entry();
  extern __shared__ uint32_t s_box[];  // [2][d]
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    s_box[c] = 0xFFFFFFFFu;
    s_box[d + c] = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  uint32_t lo[CB > 0 ? CB : 1], hi[CB > 0 ? CB : 1];
#pragma unroll
  for (int b = 0; b < (CB > 0 ? CB : 1); ++b) {
    lo[b] = 0xFFFFFFFFu;
    hi[b] = 0u;
  }
  bool bad = false;
  if constexpr (CB > 0) {
    // four rows per warp iteration; every load of the four rows is issued first
    constexpr int RPW = 4;
    for (int64_t r0 = (int64_t(blockIdx.x) * warps + warp) * RPW; r0 < n; r0 += int64_t(gridDim.x) * warps * RPW) {
      float v[RPW][CB];
#pragma unroll
      for (int q = 0; q < RPW; ++q)
#pragma unroll
        for (int b = 0; b < CB; ++b) {
          const int c = b * 32 + lane;
          v[q][b] = (r0 + q < n && c < d) ? load_elem<DT>(X, r0 + q, d, c, scales) : 0.0f;
        }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
#pragma unroll
        for (int b = 0; b < CB; ++b) {
          const int c = b * 32 + lane;
          if (r0 + q < n && c < d) {
            const float x = v[q][b];
            bad |= !isfinite(x);
            const uint32_t o = ord_enc(x);
            lo[b] = min(lo[b], o);
            hi[b] = max(hi[b], o);
          }
        }
      }
    }
  }
  for (int64_t r = int64_t(blockIdx.x) * warps + warp; CB == 0 && r < n; r += int64_t(gridDim.x) * warps) {
    for (int c = lane; c < d; c += 32) {
      const float v = load_elem<DT>(X, r, d, c, scales);
      bad |= !isfinite(v);
      const uint32_t o = ord_enc(v);
      atomicMin(&s_box[c], o);
      atomicMax(&s_box[d + c], o);
    }
  }
  if constexpr (CB > 0) {
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int c = b * 32 + lane;
      if (c < d && lo[b] <= hi[b]) {
        atomicMin(&s_box[c], lo[b]);
        atomicMax(&s_box[d + c], hi[b]);
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    if (s_box[c] <= s_box[d + c]) {
      atomicMin(&box[c], s_box[c]);
      atomicMax(&box[d + c], s_box[d + c]);
    }
  }
}

template <int DT>
static void ingest_dt(const ch_set* X, cudaStream_t s, int grid) {
  const int d = X->d;
  const size_t smem = size_t(2) * d * sizeof(uint32_t);
  const int cb = (d + 31) / 32;
#define CHX_INGEST(CBV) \
  launch_k(k_ingest<DT, CBV>, grid, 256, smem, s, X->data, X->scales, X->n, d, X->norms, X->box_x, X->status)
  if (cb <= 1) CHX_INGEST(1);
  else if (cb <= 2) CHX_INGEST(2);
  else if (cb <= 4) CHX_INGEST(4);
  else if (cb <= 8) CHX_INGEST(8);
  else if (cb <= 16) CHX_INGEST(16);
  else CHX_INGEST(0);
#undef CHX_INGEST
}

void launch_ingest(const ch_set* X, cudaStream_t s) {
  CHX_CUDA(cudaMemsetAsync(X->box_x, 0xFF, size_t(X->d) * 4, s));
  CHX_CUDA(cudaMemsetAsync(X->box_x + X->d, 0, size_t(X->d) * 4, s));
  if (X->n == 0) return;
  const int grid = static_cast<int>(std::min<int64_t>(ceil_div(X->n, 8), 152 * 8));
  switch (X->dtype) {
    case CH_F32: ingest_dt<CH_F32>(X, s, grid); break;
    case CH_BF16: ingest_dt<CH_BF16>(X, s, grid); break;
    default: ingest_dt<CH_FP8E4M3>(X, s, grid); break;
  }
  launch_check("ingest");
}

void ensure_ingest(ch_set* X, cudaStream_t s) {
  if (X->ready & READY_BOX_X) return;
  launch_ingest(X, s);
  X->ready |= READY_BOX_X;
}

// |x|^2 per row as the fmaf chain over j in increasing order (the order the l2
// projection pass uses, so the norms never depend on which pass made them)
template <int DT>
__global__ void __launch_bounds__(256) k_norms(const void* X, const float* scales, int64_t n, int d, float* norms,
                                               uint32_t* status) {
  pdl_entry();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  bool bad = false;
  if (r < n) {
    float sq = 0.0f;
    for (int j = 0; j < d; ++j) {
      const float x = load_elem<DT>(X, r, d, j, scales);
      bad |= !isfinite(x);
      sq = fmaf(x, x, sq);
    }
    norms[r] = sq;
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

void ensure_norms(ch_set* X, cudaStream_t s) {
  if (X->ready & READY_NORMS) return;
  X->ready |= READY_NORMS;
  if (X->n == 0) return;
  const int grid = static_cast<int>(ceil_div(X->n, 256));
  switch (X->dtype) {
    case CH_F32: launch_k(k_norms<CH_F32>, grid, 256, 0, s, X->data, X->scales, X->n, X->d, X->norms, X->status); break;
    case CH_BF16: launch_k(k_norms<CH_BF16>, grid, 256, 0, s, X->data, X->scales, X->n, X->d, X->norms, X->status); break;
    default: launch_k(k_norms<CH_FP8E4M3>, grid, 256, 0, s, X->data, X->scales, X->n, X->d, X->norms, X->status); break;
  }
  launch_check("norms");
}

// ------------------------------------------------------------------ l2 embedding
// Z_ij: 12-term Irwin-Hall normal from Philox counters (j, i, 2, m), m < 3,
// summed exactly, centred, scaled by 2^-32 and rounded once to binary32
// (the l2 -> l1 embedding theorem of App. A.2 with the 1/(beta k) factor left out).
// entry (j, i) of the Gaussian matrix: Irwin-Hall sum of 12 Philox words
// (counter (j, i, 2, m), m = 0..2), centred, times 2^-32, rounded once to
// binary32; zero for i >= k
__device__ inline float gauss_entry(uint64_t seed, int k, int j, int i) {
  if (i >= k) return 0.0f;
  uint64_t sum = 0;
  for (uint32_t m = 0; m < 3; ++m) {
    const P4 w = philox10(P4{uint32_t(j), uint32_t(i), 2u, m}, uint32_t(seed), uint32_t(seed >> 32));
    sum += uint64_t(w.x) + w.y + w.z + w.w;
  }
  const int64_t centred = static_cast<int64_t>(sum) - int64_t(6) * 4294967296LL;
  // one round-to-nearest of the integer to binary32, then an exact scaling by
  // 2^-32 (|centred| >= 1 keeps it normal): the single rounding of
  // centred * 2^-32, without binary64 arithmetic
  return __ll2float_rn(centred) * 0x1p-32f;
}

__global__ void k_gauss(uint64_t seed, int k, int kp, int d, float* G /* [d][kp], zero rows i >= k */) {
  pdl_entry();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(kp) * d) return;
  G[t] = gauss_entry(seed, k, static_cast<int>(t / kp), static_cast<int>(t % kp));
}

// Thread per row; rows staged through shared memory 32 coordinates at a time
// (coalesced 128-byte row segments), y_i = fmaf chain over j in increasing order.
// The same pass also writes |x|^2 (norms, when non-null) and raises ST_NONFINITE
// in the set's status word, so an l2 set is read from HBM once.
template <int DT, int KP>
__global__ void __launch_bounds__(128) k_project(const void* X, const float* scales, int64_t n, int d,
                                                 const float* G, int k, float* Y, uint32_t* box, float* norms,
                                                 uint32_t* status) {
  pdl_entry();
  // RPT rows per thread (rows tid and tid + 128) so that each G value read from
  // shared memory feeds RPT fused multiply-adds
  constexpr int RPT = KP <= 16 ? 2 : 1;
  __shared__ float s_x[128 * RPT][33];
  __shared__ __align__(16) float s_g[32][KP];
  const int64_t r0 = int64_t(blockIdx.x) * 128 * RPT;
  const int tid = threadIdx.x;
  float acc[RPT][KP];
  float sq[RPT];
  bool bad = false;
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    sq[p] = 0.0f;
#pragma unroll
    for (int i = 0; i < KP; ++i) acc[p][i] = 0.0f;
  }
  for (int j0 = 0; j0 < d; j0 += 32) {
    const int jn = min(32, d - j0);
    __syncthreads();
    // stage: warp w holds rows w, w+4, ..., lane = coordinate within the 32-wide
    // segment (coalesced); the 32 loads of a pass are issued before any store
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int p = 0; p < RPT; ++p) {
      float v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int64_t row = r0 + p * 128 + warp + 4 * q;
        v[q] = (row < n && lane < jn) ? load_elem<DT>(X, row, d, j0 + lane, scales) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) s_x[p * 128 + warp + 4 * q][lane] = v[q];
    }
    for (int t = tid; t < 32 * KP; t += 128) {
      const int jj = t / KP, ii = t % KP;
      s_g[jj][ii] = (jj < jn) ? G[int64_t(j0 + jj) * KP + ii] : 0.0f;
    }
    __syncthreads();
    for (int jj = 0; jj < jn; ++jj) {
      float xv[RPT];
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        xv[p] = s_x[p * 128 + tid][jj];
        sq[p] = fmaf(xv[p], xv[p], sq[p]);
        bad |= !isfinite(xv[p]);
      }
      const float4* g4 = reinterpret_cast<const float4*>(&s_g[jj][0]);
#pragma unroll
      for (int i4 = 0; i4 < KP / 4; ++i4) {
        const float4 g = g4[i4];
#pragma unroll
        for (int p = 0; p < RPT; ++p) {
          acc[p][4 * i4 + 0] = __fmaf_rn(g.x, xv[p], acc[p][4 * i4 + 0]);
          acc[p][4 * i4 + 1] = __fmaf_rn(g.y, xv[p], acc[p][4 * i4 + 1]);
          acc[p][4 * i4 + 2] = __fmaf_rn(g.z, xv[p], acc[p][4 * i4 + 2]);
          acc[p][4 * i4 + 3] = __fmaf_rn(g.w, xv[p], acc[p][4 * i4 + 3]);
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    const int64_t r = r0 + p * 128 + tid;
    if (r < n) {
#pragma unroll
      for (int i = 0; i < KP; ++i)
        if (i < k) Y[r * k + i] = acc[p][i];
      if (norms) norms[r] = sq[p];
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (tid & 31) == 0) atomicOr(status, ST_NONFINITE);
  // bounding box of the embedding
  const int lane = tid & 31;
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    if (i < k) {
      uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        if (r0 + p * 128 + tid < n) {
          lo = min(lo, ord_enc(acc[p][i]));
          hi = max(hi, ord_enc(acc[p][i]));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
      }
      if (lane == 0 && lo <= hi) {
        atomicMin(&box[i], lo);
        atomicMax(&box[k + i], hi);
      }
    }
  }
}

// Small dimensions (d <= 8, known at compile time): one fused launch per set.
// Each block generates its own copy of G (d x KP entries, at most one per
// thread) in shared memory, a thread keys rows in grid-stride order with the
// same fmaf chains in coordinate order as k_project, and the block writes one
// partial box (as k_project_tma does), so neither a separate G launch nor the
// box initialisation is needed.
constexpr int kProjSmallMaxD = 8;
// block bx of gx blocks over one set's rows; writes partial box bx
template <int DT, int KP, int D>
__device__ __forceinline__ void project_small_block(const void* X, const float* scales, int64_t n, uint64_t seed,
                                                    int k, float* Y, uint32_t* box, float* norms, uint32_t* status,
                                                    int bx, int gx) {
  static_assert(D * KP <= 128, "one G entry per thread");
  __shared__ __align__(16) float s_g[D][KP];
  __shared__ uint32_t s_box[2 * KP];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < D * KP) s_g[tid / KP][tid % KP] = gauss_entry(seed, k, tid / KP, tid % KP);
  if (tid < 2 * KP) s_box[tid] = tid < KP ? 0xFFFFFFFFu : 0u;
  __syncthreads();
  uint32_t lo[KP], hi[KP];  // ordered-encoded, as k_project keeps them
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    lo[i] = 0xFFFFFFFFu;
    hi[i] = 0u;
  }
  bool bad = false;
  for (int64_t r = int64_t(bx) * blockDim.x + tid; r < n; r += int64_t(gx) * blockDim.x) {
    float xv[D];
#pragma unroll
    for (int j = 0; j < D; ++j) xv[j] = load_elem<DT>(X, r, D, j, scales);
    float acc[KP], sq = 0.0f;
#pragma unroll
    for (int i = 0; i < KP; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      sq = fmaf(xv[j], xv[j], sq);
      bad |= !isfinite(xv[j]);
#pragma unroll
      for (int i = 0; i < KP; ++i) acc[i] = __fmaf_rn(s_g[j][i], xv[j], acc[i]);
    }
    if (KP == 16 && k == 16) {
      float4* y4 = reinterpret_cast<float4*>(Y + r * 16);
#pragma unroll
      for (int i4 = 0; i4 < 4; ++i4) y4[i4] = make_float4(acc[4 * i4], acc[4 * i4 + 1], acc[4 * i4 + 2], acc[4 * i4 + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < KP; ++i)
        if (i < k) Y[r * k + i] = acc[i];
    }
    if (norms) norms[r] = sq;
#pragma unroll
    for (int i = 0; i < KP; ++i) {
      lo[i] = min(lo[i], ord_enc(acc[i]));
      hi[i] = max(hi[i], ord_enc(acc[i]));
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    if (i < k) {
      uint32_t l = lo[i], h = hi[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        l = min(l, __shfl_xor_sync(0xFFFFFFFFu, l, o));
        h = max(h, __shfl_xor_sync(0xFFFFFFFFu, h, o));
      }
      if (lane == 0 && l <= h) {
        atomicMin(&s_box[i], l);
        atomicMax(&s_box[KP + i], h);
      }
    }
  }
  __syncthreads();
  if (tid < 2 * k) {
    const int i = tid < k ? tid : KP + tid - k;
    box[size_t(bx) * 2 * k + tid] = s_box[i];
  }
}

template <int DT, int KP, int D>
__global__ void __launch_bounds__(128) k_project_small(const void* X, const float* scales, int64_t n, uint64_t seed,
                                                       int k, float* Y, uint32_t* box, float* norms,
                                                       uint32_t* status) {
  pdl_entry();
  project_small_block<DT, KP, D>(X, scales, n, seed, k, Y, box, norms, status, blockIdx.x, gridDim.x);
}

// every listed set of one storage type and d in one launch: the block run of set
// i (blk0[i] .. blk0[i + 1] - 1) does what k_project_small's grid does for it
template <int DT, int KP, int D>
__global__ void __launch_bounds__(128) k_project_small_batch(const ProjSet* S, const int* blk0, int ns, int k) {
  pdl_entry();
  const int si = find_pair(blk0, ns, blockIdx.x);
  const ProjSet& p = S[si];
  const int local = blockIdx.x - __ldg(&blk0[si]);
  project_small_block<DT, KP, D>(p.X, p.scales, p.n, p.seed, k, p.Y, p.box, nullptr, p.status, local,
                                 __ldg(&blk0[si + 1]) - __ldg(&blk0[si]));
}

int project_small_blocks(int64_t n, int sm_count) {
  return static_cast<int>(std::min<int64_t>(ceil_div(n, 128), std::min(sm_count, kMaxBoxParts)));
}

void launch_project_small_batch(const ProjSet* S, const int* blk0, int ns, int blocks, int dtype, int d, int k,
                                cudaStream_t s) {
  if (ns == 0 || blocks == 0) return;
  CHX_CHECK(d >= 1 && d <= kProjSmallMaxD && k <= 16, CH_EINVAL, "batched small projection: d <= 8, k <= 16");
  auto go = [&](auto dtc) {
    constexpr int DTV = decltype(dtc)::value;
    switch (d) {
#define CHX_PSB(DV)                                                                                          \
  case DV:                                                                                                   \
    if (k <= 8) launch_k(k_project_small_batch<DTV, 8, DV>, blocks, 128, 0, s, S, blk0, ns, k);              \
    else launch_k(k_project_small_batch<DTV, 16, DV>, blocks, 128, 0, s, S, blk0, ns, k);                    \
    break;
      CHX_PSB(1) CHX_PSB(2) CHX_PSB(3) CHX_PSB(4) CHX_PSB(5) CHX_PSB(6) CHX_PSB(7) CHX_PSB(8)
#undef CHX_PSB
      default: break;
    }
  };
  switch (dtype) {
    case CH_F32: go(std::integral_constant<int, CH_F32>{}); break;
    case CH_BF16: go(std::integral_constant<int, CH_BF16>{}); break;
    default: go(std::integral_constant<int, CH_FP8E4M3>{}); break;
  }
  launch_check("project_small_batch");
}

// Asynchronous variant for rows whose byte length is a multiple of 16: each
// 32-coordinate slice of the block's rows (and of G) is copied with 16-byte
// cp.async into a double buffer, so the next slice is in flight while the
// current one is multiplied.  Same arithmetic and order as k_project.
constexpr int kProjThreads = 64;  // small blocks: ~5 resident per SM, about one wave

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(
                   __cvta_generic_to_shared(smem))),
               "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int DT, int KP>
__global__ void __launch_bounds__(kProjThreads) k_project_async(const void* X, const float* scales, int64_t n, int d,
                                                       const float* G, int k, float* Y, uint32_t* box, float* norms,
                                                       uint32_t* status) {
  pdl_entry();
  constexpr int RPT = KP <= 16 ? 2 : 1;
  constexpr int ROWS = kProjThreads * RPT;
  constexpr int ES = DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1;
  constexpr int PER = 16 / ES;       // coordinates per 16-byte chunk
  constexpr int CH = 32 / PER;       // chunks per 32-coordinate slice of a row
  constexpr int STR = CH + 1;        // padded row stride in chunks (odd: conflict-free)
  extern __shared__ __align__(16) uint4 dyn[];
  uint4* s_x = dyn;                                                    // [2][ROWS][STR]
  float* s_g = reinterpret_cast<float*>(dyn + 2 * ROWS * STR);         // [2][32][KP]
  const int64_t r0 = int64_t(blockIdx.x) * ROWS;
  const int tid = threadIdx.x;
  const int row_bytes = d * ES;
  const int slices = (d + 31) / 32;
  auto issue = [&](int sl, int buf) {
    const int j0 = sl * 32;
    // rows: ROWS x CH chunks; chunk (rr, c) covers coordinates j0 + c*PER .. +PER
    for (int t = tid; t < ROWS * CH; t += kProjThreads) {
      const int rr = t / CH, c = t % CH;
      const int64_t row = r0 + rr;
      const int jb = (j0 + c * PER) * ES;
      const bool ok = row < n && jb < row_bytes;
      const char* src = static_cast<const char*>(X) + (ok ? row * row_bytes + jb : 0);
      cp_async16(&s_x[(buf * ROWS + rr) * STR + c], src, ok ? 16u : 0u);
    }
    // G rows j0 .. j0+31 (KP floats each), zero past d
    for (int t = tid; t < 32 * KP / 4; t += kProjThreads) {
      const int jj = t / (KP / 4), c = t % (KP / 4);
      const bool ok = j0 + jj < d;
      const float* src = G + (ok ? int64_t(j0 + jj) * KP + c * 4 : 0);
      cp_async16(&s_g[(buf * 32 + jj) * KP + c * 4], src, ok ? 16u : 0u);
    }
    cp_async_commit();
  };

  float acc[RPT][KP];
  float sq[RPT];
  bool bad = false;
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    sq[p] = 0.0f;
#pragma unroll
    for (int i = 0; i < KP; ++i) acc[p][i] = 0.0f;
  }
  float scl[RPT];
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    const int64_t r = r0 + p * kProjThreads + tid;
    scl[p] = (DT == CH_FP8E4M3 && r < n) ? scales[r] : 1.0f;
  }
  issue(0, 0);
  for (int sl = 0; sl < slices; ++sl) {
    const int buf = sl & 1;
    if (sl + 1 < slices) {
      issue(sl + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int jn = min(32, d - sl * 32);
    const float* g = s_g + buf * 32 * KP;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      float xv[RPT][PER];
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        const uint4 raw = s_x[(buf * ROWS + p * kProjThreads + tid) * STR + c];
        if constexpr (DT == CH_F32) {
          xv[p][0] = __uint_as_float(raw.x);
          xv[p][1] = __uint_as_float(raw.y);
          xv[p][2] = __uint_as_float(raw.z);
          xv[p][3] = __uint_as_float(raw.w);
        } else if constexpr (DT == CH_BF16) {
          const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xv[p][2 * e] = bf16_to_f32(static_cast<uint16_t>(w4[e] & 0xFFFFu));
            xv[p][2 * e + 1] = bf16_to_f32(static_cast<uint16_t>(w4[e] >> 16));
          }
        } else {
          const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int e = 0; e < 16; ++e)
            xv[p][e] = __fmul_rn(e4m3_to_f32(static_cast<uint8_t>(w4[e / 4] >> (8 * (e % 4)))), scl[p]);
        }
      }
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int jj = c * PER + e;
        if (jj < jn) {
#pragma unroll
          for (int p = 0; p < RPT; ++p) {
            sq[p] = fmaf(xv[p][e], xv[p][e], sq[p]);
            bad |= !isfinite(xv[p][e]);
          }
          const float4* g4 = reinterpret_cast<const float4*>(g + jj * KP);
#pragma unroll
          for (int i4 = 0; i4 < KP / 4; ++i4) {
            const float4 gv = g4[i4];
#pragma unroll
            for (int p = 0; p < RPT; ++p) {
              acc[p][4 * i4 + 0] = __fmaf_rn(gv.x, xv[p][e], acc[p][4 * i4 + 0]);
              acc[p][4 * i4 + 1] = __fmaf_rn(gv.y, xv[p][e], acc[p][4 * i4 + 1]);
              acc[p][4 * i4 + 2] = __fmaf_rn(gv.z, xv[p][e], acc[p][4 * i4 + 2]);
              acc[p][4 * i4 + 3] = __fmaf_rn(gv.w, xv[p][e], acc[p][4 * i4 + 3]);
            }
          }
        }
      }
    }
    __syncthreads();  // the buffer is refilled two slices from now
  }
  const int lane = tid & 31;
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    const int64_t r = r0 + p * kProjThreads + tid;
    if (r < n) {
#pragma unroll
      for (int i = 0; i < KP; ++i)
        if (i < k) Y[r * k + i] = acc[p][i];
      if (norms) norms[r] = sq[p];
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    if (i < k) {
      uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        if (r0 + p * kProjThreads + tid < n) {
          lo = min(lo, ord_enc(acc[p][i]));
          hi = max(hi, ord_enc(acc[p][i]));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
      }
      if (lane == 0 && lo <= hi) {
        atomicMin(&box[i], lo);
        atomicMax(&box[k + i], hi);
      }
    }
  }
}

template <int DT, int KP>
static size_t project_async_smem() {
  constexpr int RPT = KP <= 16 ? 2 : 1;
  constexpr int ES = DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1;
  constexpr int CH = 32 * ES / 16;
  return size_t(2) * kProjThreads * RPT * (CH + 1) * 16 + size_t(2) * 32 * KP * 4;
}

// TMA-streamed projection (rows whose byte length is a multiple of 16, KP <= 16).
// A persistent grid of one block per SM; every warp is its own pipeline over
// 64-row tiles: lane 0 streams 128-byte slices of the tile's rows (one TMA box
// of 64 rows x 128 bytes, 128-byte swizzle) through two stages; lane l owns rows
// l and l + 32, so every Gaussian-matrix load from shared memory feeds two rows.
// The matrix is generated into shared memory by each block (same entries as
// k_gauss) while the first slices are in flight.  Per row: y_i = fmaf chain over
// j in increasing order, |x|^2 likewise, so the results are those of k_project
// bit for bit.  The box of y: after each tile a transposing butterfly leaves
// lane l the tile's min and max of output l / (32 / KP), kept across tiles in
// two registers; one partial box per block at the end.
template <int DT>
constexpr int pt_max_warps() { return 13; }
constexpr int kPTBox = 128;            // bytes of a row per slice
constexpr int kPTRows = 64;            // rows per tile (two per lane)
constexpr int kPTStage = kPTRows * kPTBox;

// butterfly over the warp that reduces KP values per lane to one value per lane:
// afterwards lane l holds the min (MIN) or max over all lanes of value l / (32 / KP)
template <int KP, bool MIN>
__device__ __forceinline__ float pt_xreduce(float (&v)[KP], int lane) {
  int x = 16;
#pragma unroll
  for (int w = KP / 2; w >= 1; w >>= 1, x >>= 1) {
    const bool up = (lane & x) != 0;
#pragma unroll
    for (int q = 0; q < w; ++q) {
      const float keep = up ? v[q + w] : v[q];
      const float send = up ? v[q] : v[q + w];
      const float got = __shfl_xor_sync(0xFFFFFFFFu, send, x);
      v[q] = MIN ? fminf(keep, got) : fmaxf(keep, got);
    }
  }
  float r = v[0];
  for (; x >= 1; x >>= 1) {
    const float got = __shfl_xor_sync(0xFFFFFFFFu, r, x);
    r = MIN ? fminf(r, got) : fmaxf(r, got);
  }
  return r;
}


template <int DT, int KP>
__global__ void __launch_bounds__(pt_max_warps<DT>() * 32, 1)
    k_project_tma(const __grid_constant__ CUtensorMap map, const void* X, const float* scales, int64_t n, int d,
                  uint64_t seed, int k, float* Y, uint32_t* box, float* norms, uint32_t* status) {
  pdl_entry();
  constexpr int ES = DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1;
  constexpr int PER = 16 / ES;          // coordinates per 16-byte chunk
  constexpr int SLICE = kPTBox / ES;    // coordinates per slice
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned by an offset from the shared array itself, so that the
  // compiler keeps every access below in the shared state space
  unsigned char* base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* stage = base + size_t(warp) * 2 * kPTStage;
  float* sG = reinterpret_cast<float*>(base + size_t(warps) * 2 * kPTStage);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sG + size_t(d) * KP) + 2 * warp;

  const int64_t ntiles = (n + kPTRows - 1) / kPTRows;
  const int slices = (d + SLICE - 1) / SLICE;
  // tiles go round-robin over the blocks first, so that the blocks' loads differ by one tile at most
  const int64_t gw = int64_t(warp) * gridDim.x + blockIdx.x, stride = int64_t(gridDim.x) * warps;
  const int64_t my_tiles = gw < ntiles ? (ntiles - gw + stride - 1) / stride : 0;
  const int64_t items = my_tiles * slices;

  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncwarp();
  // item it = (tile gw + (it / slices) * stride, slice it % slices); the
  // producer (lane 0) runs two items ahead of the consumers
  int64_t pt = gw;  // producer's next tile and slice
  int psl = 0;
  // the set streams through once: its lines go first, so that the embeddings
  // and bucket tables that follow keep their place in L2
  const uint64_t pol = l2_evict_first_policy();
  auto issue = [&](int64_t it) {  // lane 0: item it -> stage it & 1
    uint64_t* b = &bar[it & 1];
    mbar_expect_tx(b, kPTStage);
    tma_load_2d_hint(stage + (it & 1) * kPTStage, &map, psl * kPTBox, static_cast<int>(pt * kPTRows), b, pol);
    if (++psl == slices) {
      psl = 0;
      pt += stride;
    }
  };
  if (lane == 0) {
    if (items > 0) issue(0);
    if (items > 1) issue(1);
  }
  __shared__ uint32_t s_box[2 * KP];  // the block's box of y, ordered-encoded
  if (threadIdx.x < 2 * KP) s_box[threadIdx.x] = threadIdx.x < KP ? 0xFFFFFFFFu : 0u;
  for (int t = threadIdx.x; t < d * KP; t += blockDim.x) sG[t] = gauss_entry(seed, k, t / KP, t % KP);
  __syncthreads();

  // acc2[r][h] holds outputs 2h and 2h + 1 of row r; sq2 holds |x|^2 of rows 0 and 1
  uint64_t acc2[2][KP / 2], sq2 = 0;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int h = 0; h < KP / 2; ++h) acc2[r][h] = 0;
  float run_lo = __int_as_float(0x7F800000), run_hi = __int_as_float(0xFF800000);
  bool ok = true;
  int64_t it = 0;
  int64_t t = gw;  // consumer's tile and slice
  int sl = 0;
  for (; it < items; ++it) {
    float scl[2] = {1.0f, 1.0f};
    if constexpr (DT == CH_FP8E4M3) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int64_t row = t * kPTRows + lane + 32 * r;
        scl[r] = row < n ? scales[row] : 1.0f;
      }
    }
    ok = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(&bar[it & 1], static_cast<uint32_t>((it >> 1) & 1)));
    if (!ok) break;
    const uint4* rows[2] = {reinterpret_cast<const uint4*>(stage + (it & 1) * kPTStage + lane * kPTBox),
                            reinterpret_cast<const uint4*>(stage + (it & 1) * kPTStage + (lane + 32) * kPTBox)};
    const int j0 = sl * SLICE;
    const int jn = min(SLICE, d - j0);
    auto chunk = [&](int c, int lim) {
      float xv[2][PER];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const uint4 raw = rows[r][c ^ (lane & 7)];
        if constexpr (DT == CH_F32) {
          xv[r][0] = __uint_as_float(raw.x);
          xv[r][1] = __uint_as_float(raw.y);
          xv[r][2] = __uint_as_float(raw.z);
          xv[r][3] = __uint_as_float(raw.w);
        } else if constexpr (DT == CH_BF16) {
          const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xv[r][2 * e] = __uint_as_float(w4[e] << 16);
            xv[r][2 * e + 1] = __uint_as_float(w4[e] & 0xFFFF0000u);
          }
        } else {
          const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int e = 0; e < 16; ++e)
            xv[r][e] = __fmul_rn(e4m3_to_f32(static_cast<uint8_t>(w4[e / 4] >> (8 * (e % 4)))), scl[r]);
        }
      }
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        if (e < lim) {
          const uint64_t xx = f2_pack(xv[0][e], xv[1][e]);
          f2_fma(sq2, xx, xx);
          const uint64_t xb[2] = {f2_pack(xv[0][e], xv[0][e]), f2_pack(xv[1][e], xv[1][e])};
          const ulonglong2* g2 = reinterpret_cast<const ulonglong2*>(sG + (j0 + c * PER + e) * KP);
#pragma unroll
          for (int i4 = 0; i4 < KP / 4; ++i4) {
            const ulonglong2 gv = g2[i4];  // outputs 4 i4 .. 4 i4 + 3 of G's row j
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              f2_fma(acc2[r][2 * i4], gv.x, xb[r]);
              f2_fma(acc2[r][2 * i4 + 1], gv.y, xb[r]);
            }
          }
        }
      }
    };
    if (jn == SLICE) {
      // two chunks per loop body (one for fp8, whose chunk decodes 16 codes): the
      // fully unrolled slice overflowed the instruction cache (no_instruction
      // stalls); two projections, fp8 300k x 384: 368 us fully unrolled, 289 us
      // at two chunks, 274 us at one; bf16 1M x 384: 611 / 602 / 624 us at 1 / 2 / 4
      if constexpr (DT == CH_FP8E4M3) {
#pragma unroll 1
        for (int c = 0; c < 8; ++c) chunk(c, PER);
      } else {
#pragma unroll 2
        for (int c = 0; c < 8; ++c) chunk(c, PER);
      }
    } else {
      for (int c = 0; c * PER < jn; ++c) chunk(c, min(PER, jn - c * PER));
    }
    __syncwarp();
    if (lane == 0 && it + 2 < items) {
      fence_proxy_async_smem();
      issue(it + 2);
    }
    if (sl == slices - 1) {  // the tile's rows are complete
      float acc[2][KP], sq[2];
      {
        const float2 q = f2_unpack(sq2);
        sq[0] = q.x;
        sq[1] = q.y;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int h = 0; h < KP / 2; ++h) {
          const float2 q = f2_unpack(acc2[r][h]);
          acc[r][2 * h] = q.x;
          acc[r][2 * h + 1] = q.y;
        }
      float tlo[KP], thi[KP];
#pragma unroll
      for (int i = 0; i < KP; ++i) {
        tlo[i] = __int_as_float(0x7F800000);
        thi[i] = __int_as_float(0xFF800000);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int64_t row = t * kPTRows + lane + 32 * r;
        if (row < n) {
          if (KP == 16 && k == 16) {
            float4* y4 = reinterpret_cast<float4*>(Y + row * 16);
#pragma unroll
            for (int i4 = 0; i4 < 4; ++i4)
              y4[i4] = make_float4(acc[r][4 * i4], acc[r][4 * i4 + 1], acc[r][4 * i4 + 2], acc[r][4 * i4 + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < KP; ++i)
              if (i < k) Y[row * k + i] = acc[r][i];
          }
          if (norms) norms[row] = sq[r];
#pragma unroll
          for (int i = 0; i < KP; ++i) {
            tlo[i] = fminf(tlo[i], acc[r][i]);
            thi[i] = fmaxf(thi[i], acc[r][i]);
          }
          if (!isfinite(sq[r])) {  // a non-finite coordinate, or only an overflowing square: look again
            bool bad = false;
            for (int j = 0; j < d; ++j) bad |= !isfinite(load_elem<DT>(X, row, d, j, scales));
            if (bad) atomicOr(status, ST_NONFINITE);
          }
        }
#pragma unroll
        for (int h = 0; h < KP / 2; ++h) acc2[r][h] = 0;
      }
      sq2 = 0;
      run_lo = fminf(run_lo, pt_xreduce<KP, true>(tlo, lane));
      run_hi = fmaxf(run_hi, pt_xreduce<KP, false>(thi, lane));
    }
    if (++sl == slices) {
      sl = 0;
      t += stride;
    }
  }
  if (!ok) {
    if (lane == 0) atomicOr(status, ST_TIMEOUT);
    // let the copies still in flight (items it and it + 1) land before the
    // block's shared memory is released
    for (int64_t j = it; j < items && j < it + 2; ++j)
      mbar_wait_bounded(&bar[j & 1], static_cast<uint32_t>((j >> 1) & 1));
  }
  // lane l holds output o = l / (32 / KP); one lane per output merges into the block's box
  const int o = lane / (32 / KP);
  if (lane % (32 / KP) == 0 && o < k && run_lo <= run_hi) {
    atomicMin(&s_box[o], ord_enc(run_lo));
    atomicMax(&s_box[KP + o], ord_enc(run_hi));
  }
  __syncthreads();
  if (threadIdx.x < 2 * k) {
    const int i = threadIdx.x < k ? threadIdx.x : KP + threadIdx.x - k;
    box[size_t(blockIdx.x) * 2 * k + threadIdx.x] = s_box[i];
  }
}

template <int DT>
static size_t project_tma_smem(int warps, int d, int kp) {
  return 1024 + size_t(warps) * 2 * kPTStage + size_t(d) * kp * 4 + size_t(warps) * 16;
}

// the launch shape for the TMA projection, or 0 warps when it does not apply
template <int DT>
static int project_tma_warps(const ch_set* X, int kp) {
  if (kp > 16) return 0;
  if ((int64_t(X->d) * int64_t(elem_size(DT))) % 16 != 0 || (reinterpret_cast<uintptr_t>(X->data) & 15) != 0) return 0;
  if (X->n >= (int64_t(1) << 31) - kPTRows) return 0;
  const size_t budget = 226 * 1024;  // leaves room for the kernel's static shared memory
  for (int w = pt_max_warps<DT>(); w >= 4; --w)
    if (project_tma_smem<DT>(w, X->d, kp) <= budget) return w;
  return 0;
}

template <int DT>
static CUtensorMap project_map(const ch_set* X) {
  CUtensorMap m;
  const cuuint64_t rb = static_cast<cuuint64_t>(X->d) * elem_size(DT);
  cuuint64_t dims[2] = {rb, static_cast<cuuint64_t>(X->n)};
  cuuint64_t strides[1] = {rb};
  cuuint32_t boxd[2] = {static_cast<cuuint32_t>(kPTBox), static_cast<cuuint32_t>(kPTRows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(X->data), dims, strides, boxd, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CHX_CHECK(r == CUDA_SUCCESS, CH_ECUDA, "cuTensorMapEncodeTiled failed (projection)");
  return m;
}

template <int DT>
static void project_dt(const ch_set* X, const float* G, int k, int kp, float* Y, uint32_t* box, float* norms,
                       cudaStream_t s) {
  const int rows_per_block = kp <= 16 ? 256 : 128;
  const int grid = static_cast<int>(ceil_div(X->n, rows_per_block));
  const bool aligned = (int64_t(X->d) * int64_t(elem_size(DT))) % 16 == 0 &&
                       (reinterpret_cast<uintptr_t>(X->data) & 15) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
  if (aligned) {
    const int grid_a = static_cast<int>(ceil_div(X->n, int64_t(kProjThreads) * (kp <= 16 ? 2 : 1)));
#define CHX_PROJA(KPV)                                                                                       \
  do {                                                                                                       \
    const size_t sm = project_async_smem<DT, KPV>();                                                         \
    CHX_CUDA(cudaFuncSetAttribute(k_project_async<DT, KPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                  static_cast<int>(project_async_smem<DT, KPV>())));                         \
    launch_k(k_project_async<DT, KPV>, grid_a, kProjThreads, sm, s, X->data, X->scales, X->n, X->d, G, k, Y, box, norms,      \
                                                   X->status);                                               \
  } while (0)
    if (kp == 8) CHX_PROJA(8);
    else if (kp == 16) CHX_PROJA(16);
    else if (kp == 32) CHX_PROJA(32);
    else CHX_PROJA(64);
#undef CHX_PROJA
    return;
  }
#define CHX_PROJ(KPV) \
  launch_k(k_project<DT, KPV>, grid, 128, 0, s, X->data, X->scales, X->n, X->d, G, k, Y, box, norms, X->status)
  if (kp == 8) CHX_PROJ(8);
  else if (kp == 16) CHX_PROJ(16);
  else if (kp == 32) CHX_PROJ(32);
  else CHX_PROJ(64);
#undef CHX_PROJ
}

template <int DT, int KP>
static int launch_project_tma(const ch_set* X, uint64_t seed, int k, float* Y, uint32_t* box, float* norms,
                              int warps, int sm_count, cudaStream_t s) {
  static const bool attr = [] {
    CHX_CUDA(cudaFuncSetAttribute(k_project_tma<DT, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
    return true;
  }();
  (void)attr;
  const CUtensorMap map = project_map<DT>(X);
  const int64_t ntiles = ceil_div(X->n, kPTRows);
  const int sms = std::min(sm_count, kMaxBoxParts);
  // as few warps per block as cover the tiles in the same number of rounds, so
  // that every SM gets a block
  const int64_t rounds = ceil_div(ntiles, int64_t(sms) * warps);
  warps = static_cast<int>(std::min<int64_t>(warps, ceil_div(ntiles, int64_t(sms) * rounds)));
  const int grid = static_cast<int>(std::min<int64_t>(sms, ntiles));
  launch_k(k_project_tma<DT, KP>, grid, warps * 32, project_tma_smem<DT>(warps, X->d, KP), s, 
      map, X->data, X->scales, X->n, X->d, seed, k, Y, box, norms, X->status);
  return grid;
}

template <int DT, int KP>
static int launch_project_small(const ch_set* X, uint64_t seed, int k, float* Y, uint32_t* box, float* norms,
                                int sm_count, cudaStream_t s) {
  const int grid = project_small_blocks(X->n, sm_count);
  switch (X->d) {
#define CHX_PS(DV)                                                                                              \
  case DV:                                                                                                      \
    launch_k(k_project_small<DT, KP, DV>, grid, 128, 0, s, X->data, X->scales, X->n, seed, k, Y, box, norms,  \
             X->status);                                                                                        \
    break;
    CHX_PS(1) CHX_PS(2) CHX_PS(3) CHX_PS(4) CHX_PS(5) CHX_PS(6) CHX_PS(7) CHX_PS(8)
#undef CHX_PS
    default: CHX_CHECK(false, CH_EINVAL, "small projection: d must be in 1..8");
  }
  return grid;
}

template <int DT>
static int project_any(const ch_set* X, uint64_t seed, int k, int kp, float* Y, uint32_t* box, float* norms,
                       int sm_count, cudaStream_t s) {
  if (X->d <= kProjSmallMaxD && kp <= 16) {
    if (kp == 8) return launch_project_small<DT, 8>(X, seed, k, Y, box, norms, sm_count, s);
    return launch_project_small<DT, 16>(X, seed, k, Y, box, norms, sm_count, s);
  }
  const int warps = project_tma_warps<DT>(X, kp);
  if (warps > 0) {
    if (kp == 8) return launch_project_tma<DT, 8>(X, seed, k, Y, box, norms, warps, sm_count, s);
    return launch_project_tma<DT, 16>(X, seed, k, Y, box, norms, warps, sm_count, s);
  }
  // the other kernels merge into one box with global atomics
  CHX_CUDA(cudaMemsetAsync(box, 0xFF, size_t(k) * 4, s));
  CHX_CUDA(cudaMemsetAsync(box + k, 0, size_t(k) * 4, s));
  // the Gaussian matrix lives in the tail of Y's allocation
  float* G = Y + ((X->n * k + 3) & ~int64_t(3));  // 16-byte aligned
  const int64_t gn = int64_t(kp) * X->d;
  launch_k(k_gauss, static_cast<int>(ceil_div(gn, 256)), 256, 0, s, seed, k, kp, X->d, G);
  launch_check("gauss");
  project_dt<DT>(X, G, k, kp, Y, box, norms, s);
  return 1;
}

int launch_project(const ch_set* X, uint64_t seed, int k, float* Y, uint32_t* box, uint32_t* status, int sm_count,
                   cudaStream_t s) {
  (void)status;
  const int kp = k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64;
  // the set's |x|^2 and finite check come for free with this pass
  ch_set* mut = const_cast<ch_set*>(X);
  float* norms = (X->ready & READY_NORMS) ? nullptr : X->norms;
  if (norms) mut->ready |= READY_NORMS;  // no write when ready (sets may be shared by host threads)
  if (X->n == 0) {  // an empty box
    CHX_CUDA(cudaMemsetAsync(box, 0xFF, size_t(k) * 4, s));
    CHX_CUDA(cudaMemsetAsync(box + k, 0, size_t(k) * 4, s));
    return 1;
  }
  int parts;
  switch (X->dtype) {
    case CH_F32: parts = project_any<CH_F32>(X, seed, k, kp, Y, box, norms, sm_count, s); break;
    case CH_BF16: parts = project_any<CH_BF16>(X, seed, k, kp, Y, box, norms, sm_count, s); break;
    default: parts = project_any<CH_FP8E4M3>(X, seed, k, kp, Y, box, norms, sm_count, s); break;
  }
  launch_check("project");
  return parts;
}

// ------------------------------------------------------------------ scales
// Delta = sum_j (max_j - min_j) over the joint box (binary64, coordinate order),
// e_top = ceil(log2 Delta) + 1 (0 if Delta = 0); scales 2^e, e = e_top-L+1..e_top.
// Shift z_{e,j} = (w0 >> 8) 2^(e-24), w0 = Philox(j, e, 1, 0).x; multiplier
// K_j = Philox(j, 0, 4, 0).(y:x) | 1; salt_e = mix64((uint32)e ^ seed).
// the scale tables of one pair, by one whole block
__device__ void scale_tables_block(const uint32_t* boxA, int partsA, const uint32_t* boxB, int partsB, int dd, int L,
                                   int top_exp_in, uint64_t seed, const ScaleTables& t, int32_t* e_top_out,
                                   uint32_t* status) {
  __shared__ int s_elo;
  __shared__ uint32_t s_box[2 * kMaxProj];  // merged partial boxes (partial boxes only come with dd <= kMaxProj)
  const bool merge = partsA > 1 || partsB > 1;
  if (merge && top_exp_in == CH_TOP_EXP_AUTO) {
    for (int c = threadIdx.x; c < 2 * dd; c += blockDim.x) s_box[c] = c < dd ? 0xFFFFFFFFu : 0u;
    __syncthreads();
    // thread (group g, entry c): a register min / max over parts g, g + ng, ...
    // (independent loads), then one shared atomic per thread
    const int w = 2 * dd, ng = blockDim.x / w;
    const int c = threadIdx.x % w, g = threadIdx.x / w;
    if (g < ng) {
      const bool is_lo = c < dd;
      uint32_t v = is_lo ? 0xFFFFFFFFu : 0u;
#pragma unroll 8
      for (int p = g; p < partsA; p += ng) {
        const uint32_t u = __ldg(&boxA[size_t(p) * w + c]);
        v = is_lo ? min(v, u) : max(v, u);
      }
#pragma unroll 8
      for (int p = g; p < partsB; p += ng) {
        const uint32_t u = __ldg(&boxB[size_t(p) * w + c]);
        v = is_lo ? min(v, u) : max(v, u);
      }
      if (is_lo) atomicMin(&s_box[c], v);
      else atomicMax(&s_box[c], v);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int e_top;
    if (top_exp_in != CH_TOP_EXP_AUTO) {
      e_top = top_exp_in;
    } else {
      double delta = 0.0;
      for (int j = 0; j < dd; ++j) {
        const uint32_t lo = merge ? s_box[j] : min(boxA[j], boxB[j]);
        const uint32_t hi = merge ? s_box[dd + j] : max(boxA[dd + j], boxB[dd + j]);
        delta += static_cast<double>(ord_dec(hi)) - static_cast<double>(ord_dec(lo));
      }
      if (delta == 0.0) {
        e_top = 0;
      } else {
        int E;
        const double m = frexp(delta, &E);
        e_top = (m == 0.5 ? E - 1 : E) + 1;
      }
    }
    int e_lo = e_top - L + 1;
    if (e_lo < -120 || e_top > 120) {
      atomicOr(status, ST_RANGE);
      e_lo = 0;  // keep the tables well defined; the call reports CH_EINVAL
    }
    s_elo = e_lo;
    t.e_lo[0] = e_lo;
    if (e_top_out) *e_top_out = e_lo + L - 1;
  }
  __syncthreads();
  const int e_lo = s_elo;
  const uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
  for (int idx = threadIdx.x; idx < dd * L; idx += blockDim.x) {
    const int j = idx / L, l = idx % L;
    const int e = e_lo + l;
    const P4 w = philox10(P4{uint32_t(j), uint32_t(e), 1u, 0u}, k0, k1);
    t.shift[idx] = __double2float_rn(ldexp(static_cast<double>(w.x >> 8), e - 24));
  }
  for (int j = threadIdx.x; j < dd; j += blockDim.x) {
    const P4 w = philox10(P4{uint32_t(j), 0u, 4u, 0u}, k0, k1);
    t.mult[j] = ((uint64_t(w.y) << 32) | w.x) | 1ull;
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const int e = e_lo + l;
    t.inv_r[l] = pow2f(-e);
    t.salt[l] = mix64(uint64_t(uint32_t(e)) ^ seed);
  }
}

__global__ void k_scale_tables(const uint32_t* boxA, int partsA, const uint32_t* boxB, int partsB, int dd, int L,
                               int top_exp_in, uint64_t seed, ScaleTables t, int32_t* e_top_out, uint32_t* status,
                               uint4* zero, int64_t zero16, unsigned long long* left, int64_t n_left,
                               int n_zero_words) {
  pdl_entry();
  if (left && blockIdx.x == 0 && threadIdx.x <= n_zero_words)
    left[threadIdx.x] = threadIdx.x == 0 ? static_cast<unsigned long long>(n_left) : 0ull;
  if (blockIdx.x > 0) {  // the other blocks clear the bucket tables meanwhile
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int64_t i = int64_t(blockIdx.x - 1) * blockDim.x + threadIdx.x; i < zero16;
         i += int64_t(gridDim.x - 1) * blockDim.x)
      zero[i] = z;
    return;
  }
  scale_tables_block(boxA, partsA, boxB, partsB, dd, L, top_exp_in, seed, t, e_top_out, status);
}

__global__ void k_scale_tables_batch(const CrudePair* P) {
  pdl_entry();
  const CrudePair& p = P[blockIdx.x];
  scale_tables_block(p.boxA, p.partsA, p.boxB, p.partsB, p.A.dd, p.L, p.top_exp, p.seed, p.t, nullptr, p.status);
}

void launch_scale_tables_batch(const CrudePair* P, int np, cudaStream_t s) {
  if (np == 0) return;
  launch_k(k_scale_tables_batch, np, 256, 0, s, P);
  launch_check("scale_tables_batch");
}

void launch_scale_tables(const uint32_t* boxA, int partsA, const uint32_t* boxB, int partsB, int dd, int L,
                         int top_exp_in, uint64_t seed, ScaleTables t, int32_t* e_top_out, uint32_t* status,
                         cudaStream_t s, void* zero, size_t zero_bytes, int sm_count, unsigned long long* left,
                         int64_t n_left, int n_zero_words) {
  CHX_CHECK(n_zero_words < 1024, CH_EINVAL, "too many scale groups");
  CHX_CHECK((partsA <= 1 && partsB <= 1) || dd <= kMaxProj, CH_EINVAL, "partial boxes need dd <= 64");
  // 1024 threads: the partial-box loads of all blocks are in flight at once
  const int64_t zero16 = zero ? static_cast<int64_t>(zero_bytes / 16) : 0;
  const int zblocks = zero16 ? static_cast<int>(std::min<int64_t>(ceil_div(zero16, 1024 * 4), 2 * sm_count)) : 0;
  launch_k(k_scale_tables, 1 + zblocks, 1024, 0, s, boxA, partsA, boxB, partsB, dd, L, top_exp_in, seed, t, e_top_out,
           status, static_cast<uint4*>(zero), zero16, left, n_left, n_zero_words);
  launch_check("scale_tables");
}


// ------------------------------------------------------------------ crude distance
// D_a = canonical d(a, B[b(a)]): G lanes per a (G = min(32, next pow2 of d)),
// lane q sums coordinates j = q, q+32, ... in increasing j; then p_q += p_{q+s}
// for s = G/2 .. 1 via shuffles (steps s >= G would add +0).  Grid-stride; with
// maxD set, each block also folds max_a D_a into *maxD (ordered-encoded) with a
// single atomic, which saves the sampler its own pass over D.
// D_a of one pair's points by the warps of a block run: lane group of G lanes
// per a, first = this block's first lane index, step = the run's lanes
template <int DTA, int DTB, int METRIC>
__device__ __forceinline__ void crude_dist_span(const void* A, const float* scA, int64_t nA, const void* B,
                                                const float* scB, int d, int G, const int64_t* bidx, float* D,
                                                int64_t first, int64_t step, uint32_t& mx) {
  const int gshift = __ffs(G) - 1;
  const int64_t total = nA * G;
  // every lane runs the same number of rounds (the shuffles need the whole warp)
  for (int64_t g0 = first; g0 < total; g0 += step) {
    const int64_t gt = g0 + threadIdx.x;
    const int64_t a = gt >> gshift;  // G is a power of two: no 64-bit division
    const int q = static_cast<int>(gt & (G - 1));
    const bool live = gt < total;
    float p = 0.0f;
    if (live) {
      const int64_t b = bidx[a];
      for (int j = q; j < d; j += 32) {
        const float t = __fsub_rn(load_elem<DTA>(A, a, d, j, scA), load_elem<DTB>(B, b, d, j, scB));
        if (METRIC == CH_L1)
          p = __fadd_rn(p, fabsf(t));
        else
          p = __fmaf_rn(t, t, p);
      }
    }
    for (int sh = G >> 1; sh >= 1; sh >>= 1) {
      const float o = __shfl_down_sync(0xFFFFFFFFu, p, sh, G);
      p = __fadd_rn(p, o);
    }
    if (live && q == 0) {
      const float v = (METRIC == CH_L1) ? p : __fsqrt_rn(p);
      D[a] = v;
      mx = max(mx, ord_enc(v));
    }
  }
}

template <int DTA, int DTB, int METRIC>
__global__ void __launch_bounds__(256) k_crude_dist(const void* A, const float* scA, int64_t nA, const void* B,
                                                    const float* scB, int d, int G, const int64_t* bidx,
                                                    float* D, uint32_t* maxD) {
  pdl_entry();
  __shared__ uint32_t s_max[8];
  uint32_t mx = 0;
  crude_dist_span<DTA, DTB, METRIC>(A, scA, nA, B, scB, d, G, bidx, D, int64_t(blockIdx.x) * blockDim.x,
                                    int64_t(gridDim.x) * blockDim.x, mx);
  if (!maxD) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) mx = max(mx, s_max[w]);
    if (mx) atomicMax(maxD, mx);
  }
}

int crude_dist_lanes(int d) {
  int G = 1;
  while (G < d && G < 32) G <<= 1;
  return G;
}

template <int DT, int METRIC>
__global__ void __launch_bounds__(256) k_crude_dist_batch(const CrudePair* P, const int* blk0, int np) {
  pdl_entry();
  const int pi = find_pair(blk0, np, blockIdx.x);
  const CrudePair& p = P[pi];
  int G = 1;
  while (G < p.d && G < 32) G <<= 1;
  uint32_t mx = 0;
  const int64_t local = blockIdx.x - blk0[pi];
  crude_dist_span<DT, DT, METRIC>(p.rawA, p.scA, p.A.n, p.rawB, p.scB, p.d, G, p.bidx, p.D, local * blockDim.x,
                                  int64_t(p.gx_dist) * blockDim.x, mx);
}

void launch_crude_dist_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int metric,
                             cudaStream_t s) {
  if (np == 0 || blocks == 0) return;
#define CHX_CDB(DTV)                                                                                         \
  do {                                                                                                       \
    if (metric == CH_L1)                                                                                     \
      launch_k(k_crude_dist_batch<DTV, CH_L1>, blocks, 256, 0, s, P, blk0, np);                              \
    else                                                                                                     \
      launch_k(k_crude_dist_batch<DTV, CH_L2>, blocks, 256, 0, s, P, blk0, np);                              \
  } while (0)
  switch (dtype) {
    case CH_F32: CHX_CDB(CH_F32); break;
    case CH_BF16: CHX_CDB(CH_BF16); break;
    default: CHX_CDB(CH_FP8E4M3); break;
  }
#undef CHX_CDB
  launch_check("crude_dist_batch");
}

// Vector form for rows of a multiple of 16 bytes on 16-byte aligned bases (A and B
// of one storage type): rows move in 16-byte chunks of C = 16 / ES coordinates.
// A row group of LPR = 32 / C lanes reads one a and its b(a); lane l of the group
// owns partials p_{lC} .. p_{lC + C - 1} and takes chunks m = l, l + LPR, ... in
// increasing m, so partial r still collects the coordinates j = r (mod 32) in
// increasing j.  The tree p_q += p_{q+s} for s = 16 .. 1 runs by shuffles inside
// the group for s >= C and in registers below: the same sums, in the same order,
// as the lane-per-partial form.
template <int DT>
__device__ __forceinline__ void chunk_vals(const uint4 raw, float sc, float (&v)[16 / (DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1)]) {
  if constexpr (DT == CH_F32) {
    v[0] = __uint_as_float(raw.x);
    v[1] = __uint_as_float(raw.y);
    v[2] = __uint_as_float(raw.z);
    v[3] = __uint_as_float(raw.w);
  } else if constexpr (DT == CH_BF16) {
    const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[2 * e] = __uint_as_float(w4[e] << 16);
      v[2 * e + 1] = __uint_as_float(w4[e] & 0xFFFF0000u);
    }
  } else {
    const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __fmul_rn(e4m3_to_f32(static_cast<uint8_t>(w4[e / 4] >> (8 * (e % 4)))), sc);
  }
}

// Resident blocks of the vector crude-distance kernel per SM.  Each lane keeps
// all its chunks of a and of b(a) in flight at once (d / 32 of each: 12 at d =
// 384), and the row group's b(a) is read one row group ahead, so a row costs
// one memory round trip instead of four (1M x 384 bf16, alone: 256 -> 169 us for
// 95 % of A).
constexpr int kCrudeDistBlocks = 2;
// chunks of a and of b(a) in flight per lane (fp8 decodes 16 codes a chunk: half as many)
template <int DT>
constexpr int kCrudeU = DT == CH_FP8E4M3 ? 6 : 12;

// D_a for the row group's a, whose b(a) is b (a < 0: none; every lane of the
// warp calls this); folds D_a into mx on the group's first lane
template <int DT, int METRIC>
__device__ __forceinline__ void crude_row(const void* A, const float* scA, const void* B, const float* scB, int d,
                                          float* D, int64_t a, int64_t b, uint32_t& mx) {
  constexpr int ES = DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1;
  constexpr int C = 16 / ES;    // coordinates per chunk
  constexpr int LPR = 32 / C;   // lanes per row
  constexpr int U = kCrudeU<DT>;
  const int sub = (threadIdx.x & 31) % LPR;
  const int chunks = d / C;
  const size_t rowq = size_t(d) / C;  // 16-byte words per row
  const bool live = a >= 0;
  float p[C];
#pragma unroll
  for (int i = 0; i < C; ++i) p[i] = 0.0f;
  if (live) {
    const uint4* ra = static_cast<const uint4*>(A) + size_t(a) * rowq;
    const uint4* rb = static_cast<const uint4*>(B) + size_t(b) * rowq;
    const float sa = DT == CH_FP8E4M3 ? scA[a] : 1.0f;
    const float sb = DT == CH_FP8E4M3 ? scB[b] : 1.0f;
    for (int m0 = sub; m0 < chunks; m0 += LPR * U) {
      uint4 qa[U], qb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = m0 + u * LPR;
        if (m < chunks) {
          qa[u] = __ldcs(ra + m);  // A is read once: evict first
          qb[u] = rb[m];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (m0 + u * LPR < chunks) {
          float va[C], vb[C];
          chunk_vals<DT>(qa[u], sa, va);
          chunk_vals<DT>(qb[u], sb, vb);
#pragma unroll
          for (int i = 0; i < C; ++i) {
            const float t = __fsub_rn(va[i], vb[i]);
            if (METRIC == CH_L1)
              p[i] = __fadd_rn(p[i], fabsf(t));
            else
              p[i] = __fmaf_rn(t, t, p[i]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int s = 16; s >= C; s >>= 1) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const float o = __shfl_down_sync(0xFFFFFFFFu, p[i], s / C, LPR);
      p[i] = __fadd_rn(p[i], o);
    }
  }
#pragma unroll
  for (int s = C / 2; s >= 1; s >>= 1)
#pragma unroll
    for (int i = 0; i < s; ++i) p[i] = __fadd_rn(p[i], p[i + s]);
  if (live && sub == 0) {
    const float v = (METRIC == CH_L1) ? p[0] : __fsqrt_rn(p[0]);
    D[a] = v;
    mx = max(mx, ord_enc(v));
  }
}

// Row groups of RPW points of A go round-robin over the warps; every lane runs
// the same number of rounds (the shuffles need the whole warp), and b(a) of the
// next row group is read before this one's rows.
template <int DT, int METRIC>
__global__ void __launch_bounds__(256, kCrudeDistBlocks) k_crude_dist_v(const void* A, const float* scA, int64_t nA,
                                                                           const void* B, const float* scB, int d,
                                                                           const int64_t* bidx, float* D, uint32_t* maxD) {
  pdl_entry();
  constexpr int ES = DT == CH_F32 ? 4 : DT == CH_BF16 ? 2 : 1;
  constexpr int LPR = 32 / (16 / ES);  // lanes per row
  constexpr int RPW = 32 / LPR;        // rows per warp
  __shared__ uint32_t s_max[8];
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPR;
  const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t wstep = (int64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t mx = 0;
  int64_t a = warp0 * RPW + grp;
  int64_t b = a < nA ? bidx[a] : 0;
  for (int64_t a0 = warp0 * RPW; a0 < nA; a0 += wstep * RPW) {
    const int64_t an = a + wstep * RPW;
    const int64_t bn = an < nA ? bidx[an] : 0;
    crude_row<DT, METRIC>(A, scA, B, scB, d, D, a < nA ? a : -1, b, mx);
    a = an;
    b = bn;
  }
  if (!maxD) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if (lane == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) mx = max(mx, s_max[w]);
    if (mx) atomicMax(maxD, mx);
  }
}

template <int DTA, int DTB>
static void crude_dist_2(const ch_set* A, const ch_set* B, int metric, const int64_t* bidx, float* D,
                         uint32_t* maxD, int G, int grid, cudaStream_t s) {
  if (metric == CH_L1)
    launch_k(k_crude_dist<DTA, DTB, CH_L1>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d, G, bidx, D,
                                                        maxD);
  else
    launch_k(k_crude_dist<DTA, DTB, CH_L2>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d, G, bidx, D,
                                                        maxD);
}

template <int DTA>
static void crude_dist_1(const ch_set* A, const ch_set* B, int metric, const int64_t* bidx, float* D, uint32_t* maxD,
                         int G, int grid, cudaStream_t s) {
  switch (B->dtype) {
    case CH_F32: crude_dist_2<DTA, CH_F32>(A, B, metric, bidx, D, maxD, G, grid, s); break;
    case CH_BF16: crude_dist_2<DTA, CH_BF16>(A, B, metric, bidx, D, maxD, G, grid, s); break;
    default: crude_dist_2<DTA, CH_FP8E4M3>(A, B, metric, bidx, D, maxD, G, grid, s); break;
  }
}

// the vector form applies: one storage type, rows of a multiple of 16 bytes on 16-byte aligned bases
static bool crude_dist_vector_ok(const ch_set* A, const ch_set* B) {
  const size_t es = elem_size(A->dtype);
  return A->dtype == B->dtype && (size_t(A->d) * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(A->data) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(B->data) & 15) == 0;
}

static void launch_crude_dist_vector(const ch_set* A, const ch_set* B, int metric, const int64_t* bidx, float* D,
                                     uint32_t* maxD, int sm_count, cudaStream_t s) {
  const size_t es = elem_size(A->dtype);
  // a row group of 32 / (16 / es) lanes per a: 16 / es rows per warp
  const int64_t rpw = int64_t(16 / es);
  const int grid = static_cast<int>(
      std::min<int64_t>(ceil_div(ceil_div(A->n, rpw) * 32, 256), int64_t(sm_count) * kCrudeDistBlocks));
#define CHX_CDV(DTV)                                                                                              \
  do {                                                                                                            \
    if (metric == CH_L1)                                                                                          \
      launch_k(k_crude_dist_v<DTV, CH_L1>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d,  \
               bidx, D, maxD);                                                                                    \
    else                                                                                                          \
      launch_k(k_crude_dist_v<DTV, CH_L2>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d,  \
               bidx, D, maxD);                                                                                    \
  } while (0)
  switch (A->dtype) {
    case CH_F32: CHX_CDV(CH_F32); break;
    case CH_BF16: CHX_CDV(CH_BF16); break;
    default: CHX_CDV(CH_FP8E4M3); break;
  }
#undef CHX_CDV
  launch_check("crude_dist");
}

void launch_crude_dist(const ch_set* A, const ch_set* B, int metric, const int64_t* bidx, float* D, uint32_t* maxD,
                       int sm_count, cudaStream_t s) {
  if (maxD) CHX_CUDA(cudaMemsetAsync(maxD, 0, sizeof(uint32_t), s));
  if (A->n == 0) return;
  if (crude_dist_vector_ok(A, B)) {
    launch_crude_dist_vector(A, B, metric, bidx, D, maxD, sm_count, s);
    return;
  }
  int G = 1;
  while (G < A->d && G < 32) G <<= 1;
  // 8 resident blocks of 256 per SM; each block merges its maximum once
  const int grid = static_cast<int>(std::min<int64_t>(ceil_div(A->n * G, 256), int64_t(sm_count) * 8));
  switch (A->dtype) {
    case CH_F32: crude_dist_1<CH_F32>(A, B, metric, bidx, D, maxD, G, grid, s); break;
    case CH_BF16: crude_dist_1<CH_BF16>(A, B, metric, bidx, D, maxD, G, grid, s); break;
    default: crude_dist_1<CH_FP8E4M3>(A, B, metric, bidx, D, maxD, G, grid, s); break;
  }
  launch_check("crude_dist");
}

// ------------------------------------------------------------------ k x W candidates
// One warp per a: the canonical distance to each candidate (lane r sums
// coordinates j = r mod 32, then the halving tree by shuffles), the minimum with
// the smallest index on ties; one atomic per warp folds max D into *maxD.
template <int DTA, int DTB, int METRIC>
__global__ void __launch_bounds__(256) k_cand_dist(const void* A, const float* scA, int64_t nA, const void* B,
                                                   const float* scB, int d, const int32_t* cand, int stride,
                                                   int64_t* bidx, float* D, uint32_t* maxD) {
  pdl_entry();
  const int64_t a = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= nA) return;
  float best = __int_as_float(0x7F800000);
  int64_t arg = INT64_MAX;
  for (int c = 0; c < stride; ++c) {
    const int32_t b = cand[a * stride + c];
    if (b < 0) continue;
    float p = 0.0f;
    for (int j = lane; j < d; j += 32) {
      const float t = __fsub_rn(load_elem<DTA>(A, a, d, j, scA), load_elem<DTB>(B, b, d, j, scB));
      p = (METRIC == CH_L1) ? __fadd_rn(p, fabsf(t)) : __fmaf_rn(t, t, p);
    }
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) p = __fadd_rn(p, __shfl_down_sync(0xFFFFFFFFu, p, sh));
    const float v = __shfl_sync(0xFFFFFFFFu, (METRIC == CH_L1) ? p : __fsqrt_rn(p), 0);
    if (v < best || (v == best && b < arg)) {
      best = v;
      arg = b;
    }
  }
  if (lane == 0) {
    D[a] = best;
    bidx[a] = arg;
    if (maxD) atomicMax(maxD, ord_enc(best));
  }
}

void launch_cand_dist(const ch_set* A, const ch_set* B, int metric, const int32_t* cand, int stride, int64_t* bidx,
                      float* D, uint32_t* maxD, cudaStream_t s) {
  if (maxD) CHX_CUDA(cudaMemsetAsync(maxD, 0, sizeof(uint32_t), s));
  if (A->n == 0) return;
  const int grid = static_cast<int>(ceil_div(A->n * 32, 256));
  auto go = [&](auto dta, auto dtb) {
    constexpr int DTA = decltype(dta)::value, DTB = decltype(dtb)::value;
    if (metric == CH_L1)
      launch_k(k_cand_dist<DTA, DTB, CH_L1>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d, cand,
                                                          stride, bidx, D, maxD);
    else
      launch_k(k_cand_dist<DTA, DTB, CH_L2>, grid, 256, 0, s, A->data, A->scales, A->n, B->data, B->scales, A->d, cand,
                                                          stride, bidx, D, maxD);
  };
  using F = std::integral_constant<int, CH_F32>;
  using H = std::integral_constant<int, CH_BF16>;
  using E = std::integral_constant<int, CH_FP8E4M3>;
  // both sets have one storage type (checked by the caller)
  switch (A->dtype) {
    case CH_F32: go(F{}, F{}); break;
    case CH_BF16: go(H{}, H{}); break;
    default: go(E{}, E{}); break;
  }
  launch_check("cand_dist");
}

}  // namespace chx
