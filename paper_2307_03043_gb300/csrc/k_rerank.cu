// k_rerank.cu -- the canonical rerank after the tensor-core screen (Fig. 1,
// step 3): for each sample, the R best screened entries by screen score, the
// canonical binary32 distance of every column they stand for, and the minimum.
#include "common.cuh"

namespace chx {

namespace {

constexpr int kRerankWarps = 8;  // samples per block; each warp's candidate list in dynamic shared memory

// One warp per sample: the R best screened entries over all chunks (by s, then
// index), the canonical binary32 distance of each of an entry's occ columns
// (first column + o * stride, o < occ, columns < nB), and their minimum (ties:
// smaller index).
template <int DT, int METRIC>
__global__ void __launch_bounds__(32 * kRerankWarps) k_rerank(const void* A, const float* scA, int64_t nA, const void* B,
                                                const float* scB, int64_t nB, int d, const int64_t* idx, int64_t T,
                                                const float* part_s, const int32_t* part_i, int parts, int per,
                                                int occ, int stride, int R, float* min_d, int64_t* argmin) {
  pdl_entry();
  extern __shared__ float s_dyn[];  // [kRerankWarps][parts * per] scores, then as many indices
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = parts * per;
  float* s_s = s_dyn + wib * nc;
  int32_t* s_i = reinterpret_cast<int32_t*>(s_dyn + kRerankWarps * nc) + wib * nc;
  const int64_t l = int64_t(blockIdx.x) * kRerankWarps + wib;
  if (l >= T) return;
  const int64_t a = idx ? idx[l] : l;
  if (a < 0 || a >= nA) {
    if (lane == 0) {
      min_d[l] = 0.0f;
      if (argmin) argmin[l] = -1;
    }
    return;
  }
  for (int p = lane; p < nc; p += 32) {
    const int c = p / per, k = p % per;
    const size_t off = (size_t(c) * T + l) * per + k;
    s_s[p] = part_s[off];
    s_i[p] = part_i[off];
  }
  __syncwarp();
  float best = __int_as_float(0x7F800000);
  int64_t bidx = INT64_MAX;
  for (int round = 0; round < R; ++round) {
    float ms = __int_as_float(0x7F800000);
    int32_t mi = INT32_MAX;
    int mp = -1;
    for (int p = lane; p < nc; p += 32) {
      const float v = s_s[p];
      const int32_t i = s_i[p];
      if (i >= 0 && (v < ms || (v == ms && i < mi))) {
        ms = v;
        mi = i;
        mp = p;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xFFFFFFFFu, ms, o);
      const int32_t oi = __shfl_xor_sync(0xFFFFFFFFu, mi, o);
      const int op = __shfl_xor_sync(0xFFFFFFFFu, mp, o);
      if (os < ms || (os == ms && oi < mi)) {
        ms = os;
        mi = oi;
        mp = op;
      }
    }
    if (mi == INT32_MAX || mi < 0) break;  // fewer than R entries
    if (lane == (mp & 31)) s_i[mp] = -1;  // taken
    __syncwarp();
    // canonical distances to the entry's columns, all at once (lane r sums
    // coordinates j = r mod 32 of each; the reduction trees run side by side)
    int64_t bo[kRerankMaxOcc];
    bool vo[kRerankMaxOcc];
    float part[kRerankMaxOcc];
#pragma unroll
    for (int o = 0; o < kRerankMaxOcc; ++o) {
      bo[o] = int64_t(mi) + int64_t(o) * stride;
      vo[o] = o < occ && bo[o] < nB;
      part[o] = 0.0f;
    }
#pragma unroll 4
    for (int j = lane; j < d; j += 32) {
      const float x = load_elem<DT>(A, a, d, j, scA);
#pragma unroll
      for (int o = 0; o < kRerankMaxOcc; ++o) {
        if (vo[o]) {
          const float t = __fsub_rn(x, load_elem<DT>(B, bo[o], d, j, scB));
          part[o] = (METRIC == CH_L1) ? __fadd_rn(part[o], fabsf(t)) : __fmaf_rn(t, t, part[o]);
        }
      }
    }
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) {
#pragma unroll
      for (int o = 0; o < kRerankMaxOcc; ++o) part[o] = __fadd_rn(part[o], __shfl_down_sync(0xFFFFFFFFu, part[o], sh));
    }
#pragma unroll
    for (int o = 0; o < kRerankMaxOcc; ++o) {
      const float dist = __shfl_sync(0xFFFFFFFFu, (METRIC == CH_L1) ? part[o] : __fsqrt_rn(part[o]), 0);
      if (vo[o] && (dist < best || (dist == best && bo[o] < bidx))) {
        best = dist;
        bidx = bo[o];
      }
    }
  }
  if (lane == 0) {
    min_d[l] = best;
    if (argmin) argmin[l] = bidx;
  }
}

}  // namespace

void launch_rerank(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, const float* part_s,
                   const int32_t* part_i, int parts, int per, int occ, int stride, int R, float* min_d,
                   int64_t* argmin, cudaStream_t s) {
  CHX_CHECK(parts * per <= kRerankMaxCand && occ <= kRerankMaxOcc, CH_EINVAL, "rerank candidate list too long");
  const int blocks = static_cast<int>(ceil_div(T, kRerankWarps));
  const size_t smem = size_t(kRerankWarps) * parts * per * 8;
#define CHX_RERANK(DT)                                                                                        \
  do {                                                                                                        \
    CHX_CUDA(cudaFuncSetAttribute(k_rerank<DT, CH_L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                  static_cast<int>(size_t(kRerankWarps) * kRerankMaxCand * 8)));               \
    launch_k(k_rerank<DT, CH_L2>, blocks, 32 * kRerankWarps, smem, s, A->data, A->scales, A->n, B->data,        \
             B->scales, B->n, A->d, qidx, T, part_s, part_i, parts, per, occ, stride, R, min_d, argmin);       \
  } while (0)
  if (A->dtype == CH_F32) CHX_RERANK(CH_F32);
  else if (A->dtype == CH_BF16) CHX_RERANK(CH_BF16);
  else CHX_RERANK(CH_FP8E4M3);
#undef CHX_RERANK
  launch_check("rerank");
}

}  // namespace chx
