// k_keys.cu -- bucket keys of the shifted grids at every scale and the
// per-scale bucket tables of CrudeNN (Fig. 2, steps 2-3).
//
// Key of a point with hashed coordinates y at scale 2^e:
//   c_j = ceil((y_j + z_{e,j}) * 2^-e) + 0          (the grid cell, exact)
//   h   = sum_j bits(c_j) * K_j  (mod 2^64)          (fingerprint of the cell)
//   key = mix64(h + salt_e), 0 replaced by 1         (0 marks an empty slot)
// Two points share a bucket at scale e iff their keys at e are equal.
//
// Bucket tables: one open-addressing table (linear probing, 16-byte slots
// {key, ~min b}) per scale; B inserts, then each a probes its scales in
// increasing order and stops at the first bucket that holds a b.
#include <type_traits>

#include "common.cuh"

namespace chx {

namespace {

// Rows of up to 32 hashed coordinates are held in registers and keyed one
// scale at a time; wider rows (l1 in high dimension) stream their coordinates
// once and accumulate up to 16 scales together.
constexpr int kRegRow = 32;

// row of width dd <= W into registers (float4 loads for aligned binary32 rows of width W)
template <int DT, int W>
__device__ inline void load_row(const HashSrc& src, int64_t r, float (&y)[W]) {
  if constexpr (DT == CH_F32) {
    if (src.dd == W && (reinterpret_cast<uintptr_t>(src.base) & 15) == 0) {
      const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(src.base) + r * W);
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const float4 v = p[q];
        y[4 * q] = v.x;
        y[4 * q + 1] = v.y;
        y[4 * q + 2] = v.z;
        y[4 * q + 3] = v.w;
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < W; ++j) y[j] = (j < src.dd) ? load_elem<DT>(src.base, r, src.dd, j, src.scales) : 0.0f;
}

__device__ inline void cell_acc(float y, float z, float inv_r, uint64_t K, uint64_t& h) {
  float c = ceilf(__fmul_rn(__fadd_rn(y, z), inv_r));
  c = __fadd_rn(c, 0.0f);
  const uint32_t bits = __float_as_uint(c);
  h += uint64_t(bits) * uint32_t(K) + (uint64_t(bits * uint32_t(K >> 32)) << 32);
}

__device__ inline uint64_t finish_key(uint64_t h, const ScaleTables& t, int lvl) {
  const uint64_t k = mix64(h + __ldg(reinterpret_cast<const unsigned long long*>(&t.salt[lvl])));
  return k == 0 ? 1 : k;
}

// key of a register-resident row at absolute scale index lvl
template <int W>
__device__ inline uint64_t reg_key(const float (&y)[W], int dd, int L, int lvl, const ScaleTables& t) {
  const float inv_r = __ldg(&t.inv_r[lvl]);
  uint64_t h = 0;
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (j < dd)
      cell_acc(y[j], __ldg(&t.shift[j * L + lvl]), inv_r,
               __ldg(reinterpret_cast<const unsigned long long*>(&t.mult[j])), h);
  return finish_key(h, t, lvl);
}

// keys of a streamed row at scales L0 .. L0+nl-1 (nl <= 16)
template <int DT>
__device__ inline void stream_keys(const HashSrc& src, int64_t r, int L, int L0, int nl, const ScaleTables& t,
                                   uint64_t (&key)[kLevelBlock]) {
  uint64_t h[kLevelBlock];
  float inv_r[kLevelBlock];
#pragma unroll
  for (int l = 0; l < kLevelBlock; ++l) {
    h[l] = 0;
    inv_r[l] = (l < nl) ? __ldg(&t.inv_r[L0 + l]) : 1.0f;
  }
  for (int j = 0; j < src.dd; ++j) {
    const float y = load_elem<DT>(src.base, r, src.dd, j, src.scales);
    const uint64_t K = __ldg(reinterpret_cast<const unsigned long long*>(&t.mult[j]));
    const float* zrow = t.shift + int64_t(j) * L + L0;
#pragma unroll
    for (int l = 0; l < kLevelBlock; ++l)
      if (l < nl) cell_acc(y, __ldg(&zrow[l]), inv_r[l], K, h[l]);
  }
#pragma unroll
  for (int l = 0; l < kLevelBlock; ++l)
    if (l < nl) key[l] = finish_key(h[l], t, L0 + l);
}

__device__ inline uint32_t slot_home(uint64_t key, uint32_t log_cap) {
  return log_cap == 0 ? 0u : static_cast<uint32_t>(key >> (64 - log_cap));
}

// Inserts (key -> min b).  Lanes of a warp holding the same key are merged
// first: only the lowest lane (the smallest b, since b grows with the lane)
// touches the table, which keeps the coarse scales -- where most points share
// a handful of buckets -- from serialising on one L2 line.
template <bool MERGE = true>
__device__ inline void table_insert(ulonglong2* tab, uint32_t log_cap, uint64_t key, int64_t b, uint32_t* status) {
  if (MERGE) {  // equal keys of a warp: only the lowest lane (the smallest b) inserts
    const unsigned peers = __match_any_sync(__activemask(), static_cast<unsigned long long>(key));
    if ((threadIdx.x & 31) != __ffs(peers) - 1) return;
  }
  const uint32_t cap = 1u << log_cap;
  const unsigned long long want = ~static_cast<unsigned long long>(b);
  uint32_t pos = slot_home(key, log_cap);
  for (uint32_t it = 0; it < cap; ++it) {
    // A read first: a slot's key only ever goes from 0 to its final value and
    // its y only grows, so a stale read is safe.  A present key costs no atomic
    // round trip (points of one cluster share buckets at the coarse scales,
    // and their CAS would queue on one address), and the min-update is skipped
    // when it cannot raise y.
    const ulonglong2 seen = __ldcg(&tab[pos]);
    if (seen.x == key) {
      if (seen.y < want) atomicMax(&tab[pos].y, want);
      return;
    }
    if (seen.x == 0ull) {
      // one round trip: claim the slot or learn its owner; the min-update is a
      // fire-and-forget reduction
      const unsigned long long cur = atomicCAS(&tab[pos].x, 0ull, static_cast<unsigned long long>(key));
      if (cur == 0ull || cur == key) {
        atomicMax(&tab[pos].y, want);
        return;
      }
    }
    pos = (pos + 1) & (cap - 1);
  }
  atomicOr(status, ST_TABLE_FULL);
}

// bucket of key at one scale: the smallest b, or -1 if empty
__device__ inline int64_t table_find(const ulonglong2* tab, uint32_t log_cap, uint64_t key) {
  const uint32_t cap = 1u << log_cap;
  uint32_t pos = slot_home(key, log_cap);
  for (uint32_t it = 0; it < cap; ++it) {
    const ulonglong2 sl = tab[pos];
    if (sl.x == key) return static_cast<int64_t>(~sl.y);
    if (sl.x == 0ull) return -1;
    pos = (pos + 1) & (cap - 1);
  }
  return -1;
}

// Narrow rows: one thread per (point, scale) (blockIdx.y = scale), so the
// scales' insert round trips overlap instead of forming one chain per point.
template <int DT, int W>
__global__ void __launch_bounds__(128) k_table_insert_ps(HashSrc src, int L, int L0, int nl, ScaleTables t,
                                                         HashTable h, uint32_t* status) {
  pdl_entry();
  const int l = blockIdx.y;  // scale; blocks run scale by scale, as the flat order t = l * n + r did
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= src.n) return;
  float y[W];
  load_row<DT, W>(src, r, y);
  const size_t cap = size_t(1) << h.log_cap;
  table_insert(h.slots + size_t(l) * cap, h.log_cap, reg_key(y, src.dd, L, L0 + l, t), r, status);
}

template <int DT>
__global__ void __launch_bounds__(128) k_table_insert(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                      uint32_t* status) {
  pdl_entry();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= src.n) return;
  const size_t cap = size_t(1) << h.log_cap;
  {
    for (int b0 = 0; b0 < nl; b0 += kLevelBlock) {
      uint64_t key[kLevelBlock];
      const int nb = min(kLevelBlock, nl - b0);
      stream_keys<DT>(src, r, L, L0 + b0, nb, t, key);
#pragma unroll
      for (int l = 0; l < kLevelBlock; ++l)
        if (l < nb) table_insert(h.slots + size_t(b0 + l) * cap, h.log_cap, key[l], r, status);
    }
  }
}

// Each unresolved a walks the scales of the group in increasing order and
// stops at the first bucket that holds a b (Fig. 2, step 3).
template <int DT, int W, bool WIDE>
__global__ void __launch_bounds__(128) k_table_probe(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                     int64_t* bidx, uint8_t* level) {
  pdl_entry();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= src.n) return;
  if (L0 > 0 && level[r] < L) return;  // resolved at a finer scale group
  if (L0 == 0) {
    // first group: start from "no scale collides" (b = 0, level = L)
    bidx[r] = 0;
    level[r] = static_cast<uint8_t>(L);
  }
  const size_t cap = size_t(1) << h.log_cap;
  if (!WIDE) {  // rows in registers (dd <= W); the wide form is compiled only where needed
    float y[W];
    load_row<DT, W>(src, r, y);
    for (int l = 0; l < nl; ++l) {
      const int64_t b = table_find(h.slots + size_t(l) * cap, h.log_cap, reg_key(y, src.dd, L, L0 + l, t));
      if (b >= 0) {
        bidx[r] = b;
        level[r] = static_cast<uint8_t>(L0 + l);
        return;
      }
    }
  } else {
    for (int b0 = 0; b0 < nl; b0 += kLevelBlock) {
      uint64_t key[kLevelBlock];
      const int nb = min(kLevelBlock, nl - b0);
      stream_keys<DT>(src, r, L, L0 + b0, nb, t, key);
#pragma unroll
      for (int l = 0; l < kLevelBlock; ++l) {
        if (l >= nb) continue;
        const int64_t b = table_find(h.slots + size_t(b0 + l) * cap, h.log_cap, key[l]);
        if (b >= 0) {
          bidx[r] = b;
          level[r] = static_cast<uint8_t>(L0 + b0 + l);
          return;
        }
      }
    }
  }
}

template <int DT, int W>
__global__ void __launch_bounds__(128) k_keys_write(HashSrc src, int L, ScaleTables t, uint64_t* keys) {
  pdl_entry();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= src.n) return;
  if (src.dd <= W) {
    float y[W];
    load_row<DT, W>(src, r, y);
    for (int l = 0; l < L; ++l) keys[size_t(l) * src.n + r] = reg_key(y, src.dd, L, l, t);
  } else {
    for (int b0 = 0; b0 < L; b0 += kLevelBlock) {
      uint64_t key[kLevelBlock];
      const int nb = min(kLevelBlock, L - b0);
      stream_keys<DT>(src, r, L, b0, nb, t, key);
#pragma unroll
      for (int l = 0; l < kLevelBlock; ++l)
        if (l < nb) keys[size_t(b0 + l) * src.n + r] = key[l];
    }
  }
}

// calls f(dtype constant, register row width constant) for a hashed source
template <class F>
void dispatch_dt_w(int dtype, int dd, F&& f) {
  auto with_w = [&](auto dtc) {
    if (dd <= 16)
      f(dtc, std::integral_constant<int, 16>{});
    else
      f(dtc, std::integral_constant<int, kRegRow>{});
  };
  switch (dtype) {
    case CH_F32: with_w(std::integral_constant<int, CH_F32>{}); break;
    case CH_BF16: with_w(std::integral_constant<int, CH_BF16>{}); break;
    default: with_w(std::integral_constant<int, CH_FP8E4M3>{}); break;
  }
}

}  // namespace

// SimHash keys (random hyperplanes at every scale): bit i of a point is 1 unless
// y_i < 0; level l keeps the first max(1, K >> l) bits; key = mix64(bits +
// mix64((l << 32) ^ seed)), 0 replaced by 1.  One thread per point, all levels.
__global__ void k_simhash_keys(const float* Y, int64_t n, int K, int L, uint64_t seed, uint64_t* keys) {
  pdl_entry();
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint64_t word = 0;
  for (int i = 0; i < K; ++i)
    if (!(Y[p * K + i] < 0.0f)) word |= 1ull << i;
  for (int l = 0; l < L; ++l) {
    const int t = max(1, K >> l);
    const uint64_t bits = t >= 64 ? word : (word & ((1ull << t) - 1));
    const uint64_t k = mix64(bits + mix64((static_cast<uint64_t>(static_cast<uint32_t>(l)) << 32) ^ seed));
    keys[int64_t(l) * n + p] = k == 0 ? 1 : k;
  }
}

void launch_simhash_keys(const float* Y, int64_t n, int K, int L, uint64_t seed, uint64_t* keys, cudaStream_t s) {
  if (n == 0) return;
  launch_k(k_simhash_keys, static_cast<int>(ceil_div(n, 128)), 128, 0, s, Y, n, K, L, seed, keys);
  launch_check("simhash_keys");
}

void launch_keys_write(HashSrc X, int L, ScaleTables t, uint64_t* keys, cudaStream_t s) {
  if (X.n == 0) return;
  const int grid = static_cast<int>(ceil_div(X.n, 128));
  dispatch_dt_w(X.dtype, X.dd, [&](auto dtc, auto wc) {
    launch_k(k_keys_write<decltype(dtc)::value, decltype(wc)::value>, grid, 128, 0, s, X, L, t, keys);
  });
  launch_check("keys_write");
}

void launch_group_insert(HashSrc B, int L, int L0, int nl, ScaleTables t, HashTable h, uint32_t* status,
                         cudaStream_t s) {
  if (B.n == 0) return;
  if (B.dd <= kRegRow) {
    const dim3 grid_ps(static_cast<unsigned>(ceil_div(B.n, 128)), static_cast<unsigned>(nl));
    dispatch_dt_w(B.dtype, B.dd, [&](auto dtc, auto wc) {
      launch_k(k_table_insert_ps<decltype(dtc)::value, decltype(wc)::value>, grid_ps, 128, 0, s, B, L, L0, nl, t, h,
                                                                                            status);
    });
    launch_check("table_insert");
    return;
  }
  const int grid = static_cast<int>(ceil_div(B.n, 128));
  switch (B.dtype) {
    case CH_F32: launch_k(k_table_insert<CH_F32>, grid, 128, 0, s, B, L, L0, nl, t, h, status); break;
    case CH_BF16: launch_k(k_table_insert<CH_BF16>, grid, 128, 0, s, B, L, L0, nl, t, h, status); break;
    default: launch_k(k_table_insert<CH_FP8E4M3>, grid, 128, 0, s, B, L, L0, nl, t, h, status); break;
  }
  launch_check("table_insert");
}

void launch_group_probe(HashSrc A, int L, int L0, int nl, ScaleTables t, HashTable h, int64_t* bidx, uint8_t* level,
                        cudaStream_t s) {
  if (A.n == 0) return;
  const int grid = static_cast<int>(ceil_div(A.n, 128));
  dispatch_dt_w(A.dtype, A.dd, [&](auto dtc, auto wc) {
    constexpr int DT = decltype(dtc)::value, W = decltype(wc)::value;
    if (A.dd <= W)  // the register form alone: 32-odd registers instead of 115, so 4x the resident warps
      launch_k(k_table_probe<DT, W, false>, grid, 128, 0, s, A, L, L0, nl, t, h, bidx, level);
    else
      launch_k(k_table_probe<DT, W, true>, grid, 128, 0, s, A, L, L0, nl, t, h, bidx, level);
  });
  launch_check("table_probe");
}

}  // namespace chx
