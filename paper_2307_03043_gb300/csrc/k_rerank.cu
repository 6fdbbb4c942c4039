// k_rerank.cu -- the canonical rerank after the tensor-core screen (Fig. 1,
// step 3): for each sample, the R best screened entries by screen score, the
// canonical binary32 distance of every column they stand for, and the minimum.
#include "common.cuh"

namespace chx {

namespace {

// One warp per sample.  First the R best screened entries over all chunks (by s,
// then index); an entry stands for occ columns (first + o * stride, o < occ,
// columns < nB).  Then their canonical binary32 distances, 32 columns at a time:
// lane r sums coordinates j = r mod 32 of all 32 columns (loads of every column
// in flight together), and a transposing butterfly finishes the 32 halving trees
// at once -- at step s lane pairs (q, q + s) add the same partials the tree adds,
// so lane q ends with column q's canonical sum.  Minimum, smallest index on ties.
template <int DT, int METRIC>
__global__ void __launch_bounds__(256) k_rerank(const void* A, const float* scA, int64_t nA, const void* B,
                                                const float* scB, int64_t nB, int d, const int64_t* idx, int64_t T,
                                                const float* part_s, const int32_t* part_i, int parts, int per,
                                                int occ, int stride, int R, float* min_d, int64_t* argmin) {
  __shared__ float s_s[8][kRerankMaxCand];
  __shared__ int32_t s_i[8][kRerankMaxCand];
  __shared__ int32_t s_sel[8][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t l = int64_t(blockIdx.x) * 8 + wib;
  if (l >= T) return;
  const int64_t a = idx ? idx[l] : l;
  if (a < 0 || a >= nA) {
    if (lane == 0) {
      min_d[l] = 0.0f;
      if (argmin) argmin[l] = -1;
    }
    return;
  }
  const int nc = parts * per;
  for (int p = lane; p < nc; p += 32) {
    const int c = p / per, k = p % per;
    const size_t off = (size_t(c) * T + l) * per + k;
    s_s[wib][p] = part_s[off];
    s_i[wib][p] = part_i[off];
  }
  __syncwarp();
  // the R best entries (selection only; no distance yet)
  int nsel = 0;
  for (int round = 0; round < R; ++round) {
    float ms = __int_as_float(0x7F800000);
    int32_t mi = INT32_MAX;
    int mp = -1;
    for (int p = lane; p < nc; p += 32) {
      const float v = s_s[wib][p];
      const int32_t i = s_i[wib][p];
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
    if (lane == (mp & 31)) s_i[wib][mp] = -1;  // taken
    if (lane == 0) s_sel[wib][round] = mi;
    ++nsel;
    __syncwarp();
  }
  __syncwarp();
  float best = __int_as_float(0x7F800000);
  int64_t bidx = INT64_MAX;
  const int ncol = nsel * occ;
  for (int c0 = 0; c0 < ncol; c0 += 32) {
    // column c0 + q: entry (c0 + q) / occ, occurrence (c0 + q) % occ
    int32_t col[32];  // B has fewer than 2^31 points (the screen's own limit)
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int c = c0 + q;
      col[q] = -1;
      if (c < ncol) {
        const int64_t b = int64_t(s_sel[wib][c / occ]) + int64_t(c % occ) * stride;
        if (b < nB) col[q] = static_cast<int32_t>(b);
      }
    }
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = 0.0f;
    for (int j = lane; j < d; j += 32) {
      const float x = load_elem<DT>(A, a, d, j, scA);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        if (col[q] >= 0) {
          const float t = __fsub_rn(x, load_elem<DT>(B, col[q], d, j, scB));
          v[q] = (METRIC == CH_L1) ? __fadd_rn(v[q], fabsf(t)) : __fmaf_rn(t, t, v[q]);
        }
      }
    }
    // transposing butterfly: at the step with xor distance w the lane keeps the
    // columns whose bit w agrees with its own lane bit w
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
      const bool up = (lane & w) != 0;
#pragma unroll
      for (int k = 0; k < w; ++k) {
        const float keep = up ? v[k + w] : v[k];
        const float send = up ? v[k] : v[k + w];
        v[k] = __fadd_rn(keep, __shfl_xor_sync(0xFFFFFFFFu, send, w));
      }
    }
    // lane q now holds column c0 + q
    int64_t mine = -1;
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q == lane) mine = col[q];  // -1 stays -1
    float dist = (METRIC == CH_L1) ? v[0] : __fsqrt_rn(v[0]);
    if (mine < 0) dist = __int_as_float(0x7F800000);
    int64_t bi = mine < 0 ? INT64_MAX : mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xFFFFFFFFu, dist, o);
      const int64_t oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
      if (od < dist || (od == dist && oi < bi)) {
        dist = od;
        bi = oi;
      }
    }
    if (dist < best || (dist == best && bi < bidx)) {
      best = dist;
      bidx = bi;
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
  const int blocks = static_cast<int>(ceil_div(T, 8));
#define CHX_RERANK(DT)                                                                                              \
  k_rerank<DT, CH_L2><<<blocks, 256, 0, s>>>(A->data, A->scales, A->n, B->data, B->scales, B->n, A->d, qidx, T,  \
                                             part_s, part_i, parts, per, occ, stride, R, min_d, argmin)
  if (A->dtype == CH_F32) CHX_RERANK(CH_F32);
  else if (A->dtype == CH_BF16) CHX_RERANK(CH_BF16);
  else CHX_RERANK(CH_FP8E4M3);
#undef CHX_RERANK
  launch_check("rerank");
}

}  // namespace chx
