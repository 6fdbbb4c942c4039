// k_scan.cu -- exact sampled nearest-neighbour scan (Fig. 1, step 3) and the
// exact brute force (Section 1) on CUDA cores.
//
// Every (q, b) pair is evaluated with the canonical binary32 distance: 32
// strided partials p_r = sum_{j = r mod 32} term_j in increasing j, combined
// by the halving tree p_r += p_{r+s}, s = 16, 8, 4, 2, 1.  A thread holds a
// PQ x PB block of pairs and walks the tree depth first (leaves in bit-reversed
// order), so each pair needs ~6 live registers instead of 32; subtrees whose
// leaves are all beyond d are +0 and skipped (adding +0 to a non-negative
// partial is exact).  The result is bit-identical to the definition, for both
// the minimum and the smallest-index argmin.
#include "common.cuh"

namespace chx {

// Resident blocks per SM of k_scan_exact: the register cap (80 per thread,
// no spills) lets three 256-thread blocks share an SM, so one block's tile
// copy overlaps the others' arithmetic.
constexpr int kScanBlocksPerSM = 3;

// NJ > 0: d lies in (32 (NJ - 1), 32 NJ], so every partial holds NJ - 1 or NJ
// terms and the loops unroll; NJ = 0: any d, runtime loops.
template <int METRIC, int PQ, int PB, int QS, int BS, int NJ>
struct Tree {
  // the term of coordinate j for every pair; FIRST starts the partial with it
  // (|t| or t*t alone, bit-identical to adding it to +0)
  template <bool FIRST>
  static __device__ __forceinline__ void term(float (&acc)[PQ][PB], const float* __restrict__ Qt,
                                              const float* __restrict__ Bt, int j) {
    float qv[PQ], bv[PB];
    if constexpr (PQ == 2) {
      const float2 t = *reinterpret_cast<const float2*>(Qt + j * QS);
      qv[0] = t.x;
      qv[1] = t.y;
    } else {
#pragma unroll
      for (int p = 0; p < PQ; ++p) qv[p] = Qt[j * QS + p];
    }
    if constexpr (PB == 4) {
      const float4 t = *reinterpret_cast<const float4*>(Bt + j * BS);
      bv[0] = t.x;
      bv[1] = t.y;
      bv[2] = t.z;
      bv[3] = t.w;
    } else if constexpr (PB == 2) {
      const float2 t = *reinterpret_cast<const float2*>(Bt + j * BS);
      bv[0] = t.x;
      bv[1] = t.y;
    } else {
#pragma unroll
      for (int b = 0; b < PB; ++b) bv[b] = Bt[j * BS + b];
    }
#pragma unroll
    for (int p = 0; p < PQ; ++p)
#pragma unroll
      for (int b = 0; b < PB; ++b) {
        const float t = __fsub_rn(qv[p], bv[b]);
        if constexpr (METRIC == CH_L1)
          acc[p][b] = FIRST ? fabsf(t) : __fadd_rn(acc[p][b], fabsf(t));
        else
          acc[p][b] = FIRST ? __fmul_rn(t, t) : __fmaf_rn(t, t, acc[p][b]);
      }
  }

  // leaf R (R < d): sum over j = R, R+32, ... of |q_j - b_j| or (q_j - b_j)^2
  template <int R>
  static __device__ __forceinline__ void leaf(float (&acc)[PQ][PB], const float* __restrict__ Qt,
                                              const float* __restrict__ Bt, int d) {
    term<true>(acc, Qt, Bt, R);
    if constexpr (NJ > 0) {
#pragma unroll
      for (int t = 1; t < NJ; ++t)
        if (t < NJ - 1 || R + 32 * t < d) term<false>(acc, Qt, Bt, R + 32 * t);
    } else {
      for (int j = R + 32; j < d; j += 32) term<false>(acc, Qt, Bt, j);
    }
  }

  // value of partial R after tree steps 16 .. S  (S = 32: the leaf itself)
  template <int R, int S>
  static __device__ __forceinline__ void node(float (&out)[PQ][PB], const float* __restrict__ Qt,
                                              const float* __restrict__ Bt, int d) {
    if constexpr (S == 32) {
      leaf<R>(out, Qt, Bt, d);
    } else {
      node<R, 2 * S>(out, Qt, Bt, d);
      if (NJ >= 2 || R + S < d) {  // d > 32: no partial is empty
        float tmp[PQ][PB];
        node<R + S, 2 * S>(tmp, Qt, Bt, d);
#pragma unroll
        for (int p = 0; p < PQ; ++p)
#pragma unroll
          for (int b = 0; b < PB; ++b) out[p][b] = __fadd_rn(out[p][b], tmp[p][b]);
      }
    }
  }
};

// Copies coordinates jl, jl + 8, ... of source row `row` (-1: zeros) into column
// r of a coordinate-major tile (Ts[j * S + r]).  Lane (rl, jl) = (lane & 3,
// lane >> 2) of a warp takes row 4g + rl of row group g: one warp instruction
// reads 8 consecutive coordinates of 4 rows and, with S = 4 mod 8, stores to
// 32 distinct banks.
template <int DT, int S, int NJ>
__device__ __forceinline__ void stage_row(float* __restrict__ Ts, int r, const void* __restrict__ base,
                                          const float* __restrict__ scales, int64_t row, int d, int jl) {
  static_assert(S % 8 == 4, "conflict-free staging needs S = 4 mod 8");
  if constexpr (NJ > 0) {
#pragma unroll
    for (int k = 0; k < 4 * NJ; ++k) {
      const int j = jl + 8 * k;
      if (k < 4 * (NJ - 1) || j < d) Ts[j * S + r] = row >= 0 ? load_elem<DT>(base, row, d, j, scales) : 0.0f;
    }
  } else {
    for (int j = jl; j < d; j += 8) Ts[j * S + r] = row >= 0 ? load_elem<DT>(base, row, d, j, scales) : 0.0f;
  }
}

// The binary32 form of stage_row as asynchronous 4-byte copies (cp.async, no
// register round trip): row < 0 fills zeros (source size 0).  The copies land
// after cp.async.wait_group.
template <int S, int NJ>
__device__ __forceinline__ void stage_row_async(float* __restrict__ Ts, int r, const float* __restrict__ base,
                                                int64_t row, int d, int jl) {
  static_assert(S % 8 == 4, "conflict-free staging needs S = 4 mod 8");
  const float* src = base + (row >= 0 ? row : 0) * int64_t(d);
  const uint32_t n = row >= 0 ? 4u : 0u;
  auto one = [&](int j) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(static_cast<uint32_t>(
                     __cvta_generic_to_shared(Ts + j * S + r))),
                 "l"(src + j), "r"(n)
                 : "memory");
  };
  if constexpr (NJ > 0) {
#pragma unroll
    for (int k = 0; k < 4 * NJ; ++k) {
      const int j = jl + 8 * k;
      if (k < 4 * (NJ - 1) || j < d) one(j);
    }
  } else {
    for (int j = jl; j < d; j += 8) one(j);
  }
}

// One block: QT samples against a chunk of B, staged SUB x BT rows at a time
// (one pair of barriers per stage); each thread owns PQ samples x PB rows of
// every BT-row sub-tile.
template <int DT, int METRIC, int QT, int BT, int PQ, int PB, int NJ, int SUB, bool DB>
__global__ void __launch_bounds__(256, kScanBlocksPerSM)
    k_scan_exact(const void* __restrict__ A, const float* __restrict__ scA, const int64_t* __restrict__ qidx, int64_t T,
                 int64_t nA, const void* __restrict__ B, const float* __restrict__ scB, int64_t nB, int d,
                 int64_t chunk_len, float* part_val, int64_t* part_idx) {
  pdl_entry();
  constexpr int NTQ = QT / PQ, NTB = BT / PB;
  static_assert(NTQ * NTB == 256, "256 threads");
  static_assert(NTB == 16, "16 thread rows (the occupancy estimate assumes it)");
  constexpr int ST = BT * SUB;  // rows per stage
  constexpr int QS = QT + 4, BS = ST + 4;
  extern __shared__ __align__(16) float smem[];
  float* Qs = smem;
  float* Bs = smem + size_t(d) * QS;  // DB: two stages, the next one in flight during this one's arithmetic
  __shared__ float r_val[NTB][QT];
  __shared__ int64_t r_idx[NTB][QT];

  const int tid = threadIdx.x;
  const int tq = tid % NTQ, tb = tid / NTQ;
  const int64_t q0 = int64_t(blockIdx.x) * QT;
  const int64_t b_begin = int64_t(blockIdx.y) * chunk_len;
  const int64_t b_end = min(nB, b_begin + chunk_len);

  // tiles are staged transposed (coordinate-major), four rows per warp instruction
  const int warp = tid >> 5, rl = (tid & 31) & 3, jl = (tid & 31) >> 2;
  for (int g = warp; g < QT / 4; g += 8) {
    const int q = 4 * g + rl;
    const int64_t l = q0 + q;
    int64_t a = l < T ? (qidx ? qidx[l] : l) : -1;
    if (a >= nA) a = -1;
    stage_row<DT, QS, NJ>(Qs, q, A, scA, a, d, jl);
  }

  float best_val[PQ], best_p0[PQ];
  int64_t best_idx[PQ];
#pragma unroll
  for (int p = 0; p < PQ; ++p) {
    best_val[p] = __int_as_float(0x7F800000);
    best_p0[p] = __int_as_float(0x7F800000);
    best_idx[p] = INT64_MAX;
  }
  const float* Qt = Qs + tq * PQ;
  // stage `st` (rows b0 .. b0 + ST - 1 of the chunk) into buffer `buf`
  auto stage_async = [&](int64_t b0, int buf) {
    const int64_t rows = min(static_cast<int64_t>(ST), b_end - b0);
    float* dst = Bs + size_t(buf) * d * BS;
    for (int g = warp; g < ST / 4; g += 8) {
      const int r = 4 * g + rl;
      stage_row_async<BS, NJ>(dst, r, static_cast<const float*>(B), r < rows ? b0 + r : int64_t(-1), d, jl);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if constexpr (DB) {
    if (b_begin < b_end) stage_async(b_begin, 0);
  }
  int buf = 0;
  for (int64_t b0 = b_begin; b0 < b_end; b0 += ST, buf ^= 1) {
    __syncthreads();
    const int64_t rows = min(static_cast<int64_t>(ST), b_end - b0);
    if constexpr (DB) {
      // the next stage goes into the other buffer (its last readers passed the
      // barrier above); then this stage's copies are waited for
      if (b0 + ST < b_end) {
        stage_async(b0 + ST, buf ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
    } else {
      for (int g = warp; g < ST / 4; g += 8) {
        const int r = 4 * g + rl;
        stage_row<DT, BS, NJ>(Bs, r, B, scB, r < rows ? b0 + r : int64_t(-1), d, jl);
      }
    }
    __syncthreads();
    const float* Bt = Bs + (DB ? size_t(buf) * d * BS : 0) + tb * PB;
    // distances of this thread's pairs in sub-tile `sub`, folded into its minima
    auto scan_sub = [&](int sub) {
      float out[PQ][PB];
      Tree<METRIC, PQ, PB, QS, BS, NJ>::template node<0, 1>(out, Qt, Bt + sub * BT, d);
#pragma unroll
      for (int p = 0; p < PQ; ++p)
#pragma unroll
        for (int b = 0; b < PB; ++b) {
          const int r = sub * BT + tb * PB + b;
          if (r < rows) {
            const float v = out[p][b];
            if constexpr (METRIC == CH_L1) {
              if (v < best_val[p]) {
                best_val[p] = v;
                best_idx[p] = b0 + r;
              }
            } else if (v < best_p0[p]) {
              best_p0[p] = v;
              const float sv = __fsqrt_rn(v);
              if (sv < best_val[p]) {
                best_val[p] = sv;
                best_idx[p] = b0 + r;
              }
            }
          }
        }
    };
    if constexpr (SUB == 1) {
      scan_sub(0);
    } else {
#pragma unroll 1
      for (int sub = 0; sub < SUB && sub * BT < rows; ++sub) scan_sub(sub);
    }
  }
#pragma unroll
  for (int p = 0; p < PQ; ++p) {
    r_val[tb][tq * PQ + p] = best_val[p];
    r_idx[tb][tq * PQ + p] = best_idx[p];
  }
  __syncthreads();
  if (tid < QT) {
    float bv = r_val[0][tid];
    int64_t bi = r_idx[0][tid];
    for (int k = 1; k < NTB; ++k) {
      const float v = r_val[k][tid];
      const int64_t i = r_idx[k][tid];
      if (v < bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
      }
    }
    const int64_t l = q0 + tid;
    if (l < T) {
      part_val[int64_t(blockIdx.y) * T + l] = bv;
      part_idx[int64_t(blockIdx.y) * T + l] = bi;
    }
  }
}

// Small dimensions (d <= 4, known at compile time): every partial p_r of the
// canonical distance holds the single term of coordinate r, so the halving tree
// reduces to a fixed expression, folded here at compile time.  A thread keeps
// kSmallPQ samples in registers and walks a shared-memory tile of B (broadcast
// reads); about 3d + 3 instructions per (sample, point) pair.
constexpr int kSmallMaxD = 4;
constexpr int kSmallPQ = 4;
constexpr int kSmallBT = 1024;
constexpr int kSmallQ = 256 * kSmallPQ;  // samples per block

// partial R after tree steps 16 .. S (S = 32: the leaf) for d = D <= 32 terms
template <int D, int R, int S>
__device__ __forceinline__ float small_node(const float (&leaf)[D]) {
  if constexpr (S == 32) {
    return leaf[R];
  } else if constexpr (R + S < D) {
    return __fadd_rn(small_node<D, R, 2 * S>(leaf), small_node<D, R + S, 2 * S>(leaf));
  } else {
    return small_node<D, R, 2 * S>(leaf);
  }
}

template <int DT, int METRIC, int D>
__global__ void __launch_bounds__(256) k_scan_small(const void* __restrict__ A, const float* __restrict__ scA,
                                                    const int64_t* __restrict__ qidx, int64_t T, int64_t nA,
                                                    const void* __restrict__ B, const float* __restrict__ scB,
                                                    int64_t nB, int64_t chunk_len, float* part_val,
                                                    int64_t* part_idx) {
  pdl_entry();
  __shared__ float Bs[kSmallBT * D];
  const int64_t l0 = int64_t(blockIdx.x) * kSmallQ + threadIdx.x;  // samples l0 + 256 p
  const int64_t b_begin = int64_t(blockIdx.y) * chunk_len;
  const int64_t b_end = min(nB, b_begin + chunk_len);
  float q[kSmallPQ][D];
  float best_val[kSmallPQ], best_p0[kSmallPQ];
  int64_t best_idx[kSmallPQ];
#pragma unroll
  for (int p = 0; p < kSmallPQ; ++p) {
    const int64_t l = l0 + 256 * p;
    int64_t a = -1;
    if (l < T) a = qidx ? qidx[l] : l;
#pragma unroll
    for (int j = 0; j < D; ++j) q[p][j] = (a >= 0 && a < nA) ? load_elem<DT>(A, a, D, j, scA) : 0.0f;
    best_val[p] = __int_as_float(0x7F800000);
    best_p0[p] = __int_as_float(0x7F800000);
    best_idx[p] = INT64_MAX;
  }
  for (int64_t b0 = b_begin; b0 < b_end; b0 += kSmallBT) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kSmallBT), b_end - b0));
    __syncthreads();
    for (int f = threadIdx.x; f < rows * D; f += 256) Bs[f] = load_elem<DT>(B, b0 + f / D, D, f % D, scB);
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      float bv[D];
#pragma unroll
      for (int j = 0; j < D; ++j) bv[j] = Bs[r * D + j];
#pragma unroll
      for (int p = 0; p < kSmallPQ; ++p) {
        float leaf[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float t = __fsub_rn(q[p][j], bv[j]);
          leaf[j] = (METRIC == CH_L1) ? fabsf(t) : __fmul_rn(t, t);
        }
        const float v = small_node<D, 0, 1>(leaf);
        if (METRIC == CH_L1) {
          if (v < best_val[p]) {
            best_val[p] = v;
            best_idx[p] = b0 + r;
          }
        } else if (v < best_p0[p]) {
          best_p0[p] = v;
          const float sv = __fsqrt_rn(v);
          if (sv < best_val[p]) {
            best_val[p] = sv;
            best_idx[p] = b0 + r;
          }
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kSmallPQ; ++p) {
    const int64_t l = l0 + 256 * p;
    if (l < T) {
      part_val[int64_t(blockIdx.y) * T + l] = best_val[p];
      part_idx[int64_t(blockIdx.y) * T + l] = best_idx[p];
    }
  }
}

// The batched form: one persistent launch over items (pair, sample block, chunk
// of B) of many pairs of one storage type, metric and dimension.  The estimate
// needs only each sample's minimum distance, not the point attaining it, so an
// item keeps the minimum of the canonical l1 sum or squared l2 sum per sample
// (one min per pair instead of a compare and two selects) and folds it, after
// one square root for l2 (sqrt is monotone, so sqrt(min) = min(sqrt)), into the
// pair's best[] as canonical distance bits << 32 by atomicMin.  kBatchPQ samples
// per thread amortise the broadcast reads of each B row.
constexpr int kBatchPQ = 8;
constexpr int kBatchQ = 256 * kBatchPQ;  // samples per item

template <int DT, int METRIC, int D>
__global__ void __launch_bounds__(256) k_scan_small_batch(const SmallScanPair* __restrict__ pairs,
                                                          const SmallScanItem* __restrict__ items, int64_t n_items,
                                                          int64_t chunk_len) {
  pdl_entry();
  __shared__ float Bs[kSmallBT * D];
  for (int64_t w = blockIdx.x; w < n_items; w += gridDim.x) {
    const SmallScanItem it = items[w];
    const SmallScanPair pr = pairs[it.pair];
    const int64_t l0 = int64_t(it.sblock) * kBatchQ + threadIdx.x;
    const int64_t b_begin = it.b0;
    const int64_t b_end = min(pr.nB, b_begin + chunk_len);
    float q[kBatchPQ][D];
    float best[kBatchPQ];
#pragma unroll
    for (int p = 0; p < kBatchPQ; ++p) {
      const int64_t l = l0 + 256 * p;
      int64_t a = -1;
      if (l < pr.T) a = pr.qidx[l];
#pragma unroll
      for (int j = 0; j < D; ++j) q[p][j] = (a >= 0 && a < pr.nA) ? load_elem<DT>(pr.A, a, D, j, pr.scA) : 0.0f;
      best[p] = __int_as_float(0x7F800000);
    }
    for (int64_t b0 = b_begin; b0 < b_end; b0 += kSmallBT) {
      const int rows = static_cast<int>(min(static_cast<int64_t>(kSmallBT), b_end - b0));
      __syncthreads();
      for (int f = threadIdx.x; f < rows * D; f += 256) Bs[f] = load_elem<DT>(pr.B, b0 + f / D, D, f % D, pr.scB);
      __syncthreads();
      for (int r = 0; r < rows; ++r) {
        float bv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) bv[j] = Bs[r * D + j];
#pragma unroll
        for (int p = 0; p < kBatchPQ; ++p) {
          float leaf[D];
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const float t = __fsub_rn(q[p][j], bv[j]);
            leaf[j] = (METRIC == CH_L1) ? fabsf(t) : __fmul_rn(t, t);
          }
          best[p] = fminf(best[p], small_node<D, 0, 1>(leaf));
        }
      }
    }
#pragma unroll
    for (int p = 0; p < kBatchPQ; ++p) {
      const int64_t l = l0 + 256 * p;
      if (l < pr.T) {
        const float m = (METRIC == CH_L1) ? best[p] : __fsqrt_rn(best[p]);
        atomicMin(&pr.best[l], static_cast<unsigned long long>(__float_as_uint(m)) << 32);
      }
    }
    __syncthreads();  // Bs is refilled by the next item
  }
}

__global__ void k_scan_merge(const float* part_val, const int64_t* part_idx, int chunks, int64_t T,
                             const int64_t* qidx, float* min_d, int64_t* argmin) {
  pdl_entry();
  const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= T) return;
  float bv = part_val[l];
  int64_t bi = part_idx[l];
  for (int c = 1; c < chunks; ++c) {
    const float v = part_val[int64_t(c) * T + l];
    const int64_t i = part_idx[int64_t(c) * T + l];
    if (v < bv || (v == bv && i < bi)) {
      bv = v;
      bi = i;
    }
  }
  const bool none = qidx && qidx[l] < 0;
  min_d[l] = none ? 0.0f : bv;
  if (argmin) argmin[l] = none ? -1 : bi;
}

struct TileShape {
  int QT, BT, SUB;  // samples, rows per sub-tile, sub-tiles per stage
};

// small d stages more rows per barrier pair, so the copy of a stage is not
// short next to its latency
static TileShape tile_for(int d) {
  if (d <= 32) return {32, 64, 4};
  if (d <= 192) return {32, 64, 1};
  if (d <= 768) return {32, 32, 1};
  return {16, 16, 1};
}

// Binary32 rows of d <= 64 stage B through two buffers with asynchronous copies,
// the next stage in flight during this one's arithmetic (100k x 100k, T = 4606:
// d = 8 l1 0.82 -> 0.74 ms, d = 16 l1 1.22 -> 1.06 ms, d = 64 l1 3.12 -> 2.90 ms,
// l2 3.35 -> 2.99 ms).  At d = 128 the second buffer leaves room for two blocks
// per SM instead of three, and the scan was slower (5.0 -> 5.5 ms).
static bool scan_double_buffered(int dtype, int d) { return dtype == CH_F32 && d <= 64; }

static size_t scan_smem(int d, bool db) {
  const TileShape t = tile_for(d);
  return size_t(d) * ((t.QT + 4) + (db ? 2 : 1) * (t.BT * t.SUB + 4)) * sizeof(float);
}

// Blocks of k_scan_exact one SM holds at once for dimension d: the dynamic
// tiles, the static per-row minima (16 thread rows x QT x (4 + 8) bytes) and
// the 1 KB reserved per block, out of 228 KB of shared memory per SM.
static int scan_blocks_per_sm(int d, bool db) {
  const TileShape t = tile_for(d);
  const size_t per_block = scan_smem(d, db) + size_t(16) * t.QT * 12 + 1024;
  return static_cast<int>(std::max<size_t>(1, std::min<size_t>(kScanBlocksPerSM, (228u * 1024u) / per_block)));
}

int scan_exact_chunks(int64_t T, int64_t nB, int d, int dtype, int sm_count) {
  if (d <= kSmallMaxD) {  // k_scan_small: about 4 blocks per SM, chunks of >= 256 points
    const int64_t qblocks = ceil_div(std::max<int64_t>(T, 1), kSmallQ);
    int64_t chunks = ceil_div(int64_t(sm_count) * 4, qblocks);
    chunks = std::min<int64_t>(chunks, ceil_div(nB, 256));
    return static_cast<int>(std::max<int64_t>(chunks, 1));
  }
  // B is cut into equal chunks, one block per (sample tile, chunk).  The count
  // minimises (waves of resident blocks) x (B tiles per block), the kernel's time
  // when every wave runs at the same rate; ties go to fewer chunks (less merging).
  const TileShape t = tile_for(d);
  const int64_t qtiles = ceil_div(std::max<int64_t>(T, 1), t.QT);
  const int64_t resident = int64_t(sm_count) * scan_blocks_per_sm(d, scan_double_buffered(dtype, d));
  const int64_t btiles = ceil_div(std::max<int64_t>(nB, 1), int64_t(t.BT) * t.SUB);  // stages
  const int64_t max_chunks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(btiles, 4), 4 * resident));
  int64_t best = 1, best_cost = INT64_MAX;
  for (int64_t c = 1; c <= max_chunks; ++c) {
    const int64_t cost = ceil_div(qtiles * c, resident) * ceil_div(btiles, c);
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
    if (qtiles * c >= 8 * resident) break;  // past eight waves the cost only flattens
  }
  return static_cast<int>(best);
}

template <int DT, int METRIC, int QT, int BT, int PQ, int PB, int NJ = 0, int SUB = 1>
static void scan_launch(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, ScanPart part,
                        cudaStream_t s) {
  constexpr bool kDB = DT == CH_F32 && NJ > 0 && NJ <= 2;  // the launches of scan_double_buffered(DT, d)
  auto kern = k_scan_exact<DT, METRIC, QT, BT, PQ, PB, NJ, SUB, kDB>;
  const bool db = kDB;
  CHX_CHECK(tile_for(A->d).BT == BT && tile_for(A->d).SUB == SUB, CH_ENOTSUP, "scan tile mismatch");
  const size_t smem = scan_smem(A->d, db);
  // a constant value, so concurrent callers on other threads never race on it
  CHX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
  const int64_t chunk_len = ceil_div(ceil_div(B->n, part.chunks), BT * SUB) * (BT * SUB);
  dim3 grid(static_cast<unsigned>(ceil_div(T, QT)), static_cast<unsigned>(part.chunks));
  launch_k(kern, grid, 256, smem, s, A->data, A->scales, qidx, T, A->n, B->data, B->scales, B->n, A->d, chunk_len,
                               part.val, part.idx);
}

template <int DT, int METRIC>
static void scan_shape(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, ScanPart part,
                       cudaStream_t s) {
  const TileShape t = tile_for(A->d);
  if (A->d <= 128) {  // terms per partial fixed at compile time
    switch ((A->d + 31) / 32) {
      case 1: scan_launch<DT, METRIC, 32, 64, 2, 4, 1, 4>(A, qidx, T, B, part, s); break;
      case 2: scan_launch<DT, METRIC, 32, 64, 2, 4, 2>(A, qidx, T, B, part, s); break;
      case 3: scan_launch<DT, METRIC, 32, 64, 2, 4, 3>(A, qidx, T, B, part, s); break;
      default: scan_launch<DT, METRIC, 32, 64, 2, 4, 4>(A, qidx, T, B, part, s); break;
    }
  } else if (t.BT == 64)
    scan_launch<DT, METRIC, 32, 64, 2, 4>(A, qidx, T, B, part, s);
  else if (t.BT == 32)
    scan_launch<DT, METRIC, 32, 32, 2, 2>(A, qidx, T, B, part, s);
  else
    scan_launch<DT, METRIC, 16, 16, 1, 1>(A, qidx, T, B, part, s);
}

template <int DT, int METRIC, int D>
static void scan_small_launch(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, ScanPart part,
                              cudaStream_t s) {
  const int64_t chunk_len = ceil_div(B->n, part.chunks);
  dim3 grid(static_cast<unsigned>(ceil_div(T, kSmallQ)), static_cast<unsigned>(part.chunks));
  launch_k(k_scan_small<DT, METRIC, D>, grid, 256, 0, s, A->data, A->scales, qidx, T, A->n, B->data, B->scales, B->n,
                                                   chunk_len, part.val, part.idx);
}

template <int DT, int METRIC>
static void scan_small(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, ScanPart part,
                       cudaStream_t s) {
  switch (A->d) {
    case 1: scan_small_launch<DT, METRIC, 1>(A, qidx, T, B, part, s); break;
    case 2: scan_small_launch<DT, METRIC, 2>(A, qidx, T, B, part, s); break;
    case 3: scan_small_launch<DT, METRIC, 3>(A, qidx, T, B, part, s); break;
    default: scan_small_launch<DT, METRIC, 4>(A, qidx, T, B, part, s); break;
  }
}

template <int DT>
static void scan_metric(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int metric, ScanPart part,
                        cudaStream_t s) {
  if (A->d <= kSmallMaxD) {
    if (metric == CH_L1)
      scan_small<DT, CH_L1>(A, qidx, T, B, part, s);
    else
      scan_small<DT, CH_L2>(A, qidx, T, B, part, s);
    return;
  }
  if (metric == CH_L1)
    scan_shape<DT, CH_L1>(A, qidx, T, B, part, s);
  else
    scan_shape<DT, CH_L2>(A, qidx, T, B, part, s);
}

void launch_scan_exact(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int metric, ScanPart part,
                       int sm_count, cudaStream_t s) {
  (void)sm_count;
  if (T == 0) return;
  CHX_CHECK(scan_smem(A->d, false) <= 220 * 1024, CH_ENOTSUP, "dimension too large for the exact scan");
  switch (A->dtype) {
    case CH_F32: scan_metric<CH_F32>(A, qidx, T, B, metric, part, s); break;
    case CH_BF16: scan_metric<CH_BF16>(A, qidx, T, B, metric, part, s); break;
    default: scan_metric<CH_FP8E4M3>(A, qidx, T, B, metric, part, s); break;
  }
  launch_check("scan_exact");
}

void launch_scan_merge(ScanPart part, int64_t T, const int64_t* qidx, float* min_d, int64_t* argmin, cudaStream_t s) {
  if (T == 0) return;
  launch_k(k_scan_merge, static_cast<int>(ceil_div(T, 256)), 256, 0, s, part.val, part.idx, part.chunks, T, qidx, min_d,
                                                                  argmin);
  launch_check("scan_merge");
}

int small_scan_samples_per_item() { return kBatchQ; }

template <int DT, int METRIC>
static void small_batch_d(const SmallScanPair* pairs, const SmallScanItem* items, int64_t n, int64_t chunk_len, int d,
                          int grid, cudaStream_t s) {
  switch (d) {
    case 1: launch_k(k_scan_small_batch<DT, METRIC, 1>, grid, 256, 0, s, pairs, items, n, chunk_len); break;
    case 2: launch_k(k_scan_small_batch<DT, METRIC, 2>, grid, 256, 0, s, pairs, items, n, chunk_len); break;
    case 3: launch_k(k_scan_small_batch<DT, METRIC, 3>, grid, 256, 0, s, pairs, items, n, chunk_len); break;
    default: launch_k(k_scan_small_batch<DT, METRIC, 4>, grid, 256, 0, s, pairs, items, n, chunk_len); break;
  }
}

template <int DT>
static void small_batch_m(const SmallScanPair* pairs, const SmallScanItem* items, int64_t n, int64_t chunk_len,
                          int metric, int d, int grid, cudaStream_t s) {
  if (metric == CH_L1)
    small_batch_d<DT, CH_L1>(pairs, items, n, chunk_len, d, grid, s);
  else
    small_batch_d<DT, CH_L2>(pairs, items, n, chunk_len, d, grid, s);
}

void launch_scan_small_batch(const SmallScanPair* pairs, const SmallScanItem* items, int64_t n_items,
                             int64_t chunk_len, int dtype, int metric, int d, int sm_count, cudaStream_t s) {
  if (n_items == 0) return;
  CHX_CHECK(d >= 1 && d <= kSmallMaxD, CH_EINVAL, "batched small scan: d must be in 1..4");
  // a persistent grid: about four resident blocks per SM
  const int grid = static_cast<int>(std::min<int64_t>(n_items, int64_t(sm_count) * 4));
  switch (dtype) {
    case CH_F32: small_batch_m<CH_F32>(pairs, items, n_items, chunk_len, metric, d, grid, s); break;
    case CH_BF16: small_batch_m<CH_BF16>(pairs, items, n_items, chunk_len, metric, d, grid, s); break;
    default: small_batch_m<CH_FP8E4M3>(pairs, items, n_items, chunk_len, metric, d, grid, s); break;
  }
  launch_check("scan_small_batch");
}

}  // namespace chx
