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
#include <cstddef>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "common.cuh"

namespace chx {

namespace {

// Rows of up to 64 hashed coordinates are held in registers and keyed one
// scale at a time (the reverse groups up to 32); wider rows (l1 in high
// dimension) stream their coordinates once and accumulate up to 16 scales
// together.
constexpr int kRegRow = 32;
// forward tables and key writes keep rows of up to 64 values in registers (l1 in
// d <= 64); the reverse groups stay at kRegRow
constexpr int kRegRowMax = 64;

// row of width dd <= W into registers (float4 loads for aligned binary32 rows of width W)
template <int DT, int W>
__device__ inline void load_row(const HashSrc& src, int64_t r, float (&y)[W]) {
  if constexpr (DT == CH_F32) {
    if (src.dd == W && (reinterpret_cast<uintptr_t>(src.base) & 15) == 0) {
      const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(src.base) + r * W);
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        // evict-first: the rows stream past the bucket tables, which are to stay in L2
        const float4 v = __ldcs(p + q);
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

// The scale constants of a group, staged in shared memory once per block
// (the table kernels are grid-stride, so a block keys many points): the shifts
// of each scale contiguous in the coordinate, so a key reads them and the
// multipliers as 16-byte words instead of one scalar global load per term.
// 16-byte aligned: group_key reads the shifts and the multipliers as 16-byte words
template <int W>
struct __align__(16) GroupConsts {
  float z[kMaxLevels][W];  // z_{e,j} of scale L0 + l, l < nl <= kMaxLevels
  uint64_t K[W];           // multipliers
  float inv_r[kMaxLevels];
  uint64_t salt[kMaxLevels];
};
static_assert(alignof(GroupConsts<4>) == 16 && alignof(GroupConsts<16>) == 16 && alignof(GroupConsts<32>) == 16,
              "vector reads of the staged constants need 16-byte alignment");
static_assert(offsetof(GroupConsts<16>, K) % 16 == 0 && offsetof(GroupConsts<32>, K) % 16 == 0 &&
                  offsetof(GroupConsts<4>, K) % 16 == 0,
              "the multipliers start on a 16-byte boundary");

// fills c for the scales L0 .. L0 + nl - 1 (nl <= kMaxLevels, the bound every
// caller's hash parameters were checked against); every thread of the block calls it
template <int W>
__device__ void load_group_consts(GroupConsts<W>& c, const ScaleTables& t, int dd, int L, int L0, int nl) {
  for (int i = threadIdx.x; i < kMaxLevels * W; i += blockDim.x) {
    const int l = i / W, j = i % W;
    c.z[l][j] = (l < nl && j < dd) ? __ldg(&t.shift[j * L + L0 + l]) : 0.0f;
  }
  for (int j = threadIdx.x; j < W; j += blockDim.x)
    c.K[j] = j < dd ? __ldg(reinterpret_cast<const unsigned long long*>(&t.mult[j])) : 0ull;
  for (int l = threadIdx.x; l < kMaxLevels; l += blockDim.x) {
    c.inv_r[l] = l < nl ? __ldg(&t.inv_r[L0 + l]) : 1.0f;
    c.salt[l] = l < nl ? __ldg(reinterpret_cast<const unsigned long long*>(&t.salt[L0 + l])) : 0ull;
  }
  __syncthreads();
}

// key of a register-resident row at the group's scale l (the same key as reg_key at L0 + l)
template <int W>
__device__ inline uint64_t group_key(const float (&y)[W], int dd, int l, const GroupConsts<W>& c) {
  const float inv_r = c.inv_r[l];
  uint64_t h = 0;
#pragma unroll
  for (int j4 = 0; j4 < W / 4; ++j4) {
    const float4 z4 = *reinterpret_cast<const float4*>(&c.z[l][4 * j4]);
    const ulonglong2 k01 = *reinterpret_cast<const ulonglong2*>(&c.K[4 * j4]);
    const ulonglong2 k23 = *reinterpret_cast<const ulonglong2*>(&c.K[4 * j4 + 2]);
    const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
    const uint64_t kk[4] = {k01.x, k01.y, k23.x, k23.y};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * j4 + q < dd) cell_acc(y[4 * j4 + q], zz[q], inv_r, kk[q], h);
  }
  const uint64_t k = mix64(h + c.salt[l]);
  return k == 0 ? 1 : k;
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

// ------------------------------------------------------------------ scale groups
// The scales run in groups whose tables stay L2-resident.  The first kernel a
// group launches reads *h.left (the points of A no finer scale resolved; it does
// not change while that kernel runs, so all its blocks agree) and records the
// group's mode for the group's later kernels:
//   GM_SKIP  nothing left: every launch of the group returns at once;
//   GM_FWD   B's points go into tables sized for B, the unresolved a probe them;
//   GM_REV   few points left (*left <= h.rev_max): the unresolved a's buckets go
//            into small tables, B streams past them once, marking each bucket
//            with its smallest b, and the a read their buckets back.
// Both forward and reverse give, for each a, the first scale of the group at
// which some b shares its bucket and the smallest such b (Fig. 2, step 3).
enum : int32_t { GM_SKIP = 0, GM_FWD = 1, GM_REV = 2 };

__device__ __forceinline__ int group_mode(const HashTable& h) {
  if (!h.left) return GM_FWD;
  if (h.first) {
    const unsigned long long v = *h.left;
    const int m = v == 0 ? GM_SKIP : (v <= h.rev_max ? GM_REV : GM_FWD);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) h.mode[h.group] = m;
    return m;
  }
  return h.mode[h.group];
}

// takes n resolved points off *h.left: one atomic per block (every thread of the
// block calls this)
__device__ __forceinline__ void take_off_left(const HashTable& h, unsigned n) {
  __shared__ unsigned s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const unsigned w = __reduce_add_sync(0xFFFFFFFFu, n);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_n, w);
  __syncthreads();
  if (threadIdx.x == 0 && s_n) atomicAdd(h.left, 0ull - static_cast<unsigned long long>(s_n));
}

__global__ void k_table_clear(HashTable h, int64_t n16) {
  pdl_entry();
  if (group_mode(h) != GM_FWD) return;
  uint4* z = reinterpret_cast<uint4*>(h.slots);
  const uint4 zero = make_uint4(0, 0, 0, 0);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += int64_t(gridDim.x) * blockDim.x)
    z[i] = zero;
}

// Narrow rows: one thread per (point, scale) (blockIdx.y = scale), so the
// scales' insert round trips overlap instead of forming one chain per point;
// grid-stride over the points, so that a skipped group costs a short launch.
template <int DT, int W>
__global__ void __launch_bounds__(128) k_table_insert_ps(HashSrc src, int L, int L0, int nl, ScaleTables t,
                                                         HashTable h, uint32_t* status) {
  pdl_entry();
  if (group_mode(h) != GM_FWD) return;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, t, src.dd, L, L0, nl);
  const int l = blockIdx.y;
  const size_t cap = size_t(1) << h.log_cap;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
    float y[W];
    load_row<DT, W>(src, r, y);
    table_insert(h.slots + size_t(l) * cap, h.log_cap, group_key(y, src.dd, l, gc), r, status);
  }
}

template <int DT>
__global__ void __launch_bounds__(128) k_table_insert(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                      uint32_t* status) {
  pdl_entry();
  if (group_mode(h) != GM_FWD) return;
  const size_t cap = size_t(1) << h.log_cap;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
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

// Reverse group, step 1: the unresolved a's (level = L) buckets at the group's
// scales go into the small tables (one per scale), with no b yet (y = 0).
template <int DT, int W>
__global__ void __launch_bounds__(128) k_rev_insert(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                    const uint8_t* level, uint32_t* status) {
  pdl_entry();
  if (group_mode(h) != GM_REV) return;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, t, src.dd, L, L0, nl);
  const uint32_t rcap = 1u << h.rev_log_cap;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
    if (level[r] < L) continue;
    float y[W];
    load_row<DT, W>(src, r, y);
    for (int l = 0; l < nl; ++l) {
      ulonglong2* tab = h.rev + size_t(l) * rcap;
      const uint64_t key = group_key(y, src.dd, l, gc);
      uint32_t pos = slot_home(key, h.rev_log_cap);
      uint32_t it = 0;
      for (; it < rcap; ++it) {
        const unsigned long long cur = atomicCAS(&tab[pos].x, 0ull, static_cast<unsigned long long>(key));
        if (cur == 0ull || cur == key) break;
        pos = (pos + 1) & (rcap - 1);
      }
      if (it == rcap) atomicOr(status, ST_TABLE_FULL);
    }
  }
}

// Reverse group, step 2: every b looks its buckets up in the small tables and
// marks the ones present with its index (smallest b wins); one thread per
// (b, scale), as for the forward insert.
template <int DT, int W>
__global__ void __launch_bounds__(128) k_rev_stream(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h) {
  pdl_entry();
  if (group_mode(h) != GM_REV) return;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, t, src.dd, L, L0, nl);
  const uint32_t rcap = 1u << h.rev_log_cap;
  const int l = blockIdx.y;
  ulonglong2* tab = h.rev + size_t(l) * rcap;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
    float y[W];
    load_row<DT, W>(src, r, y);
    const uint64_t key = group_key(y, src.dd, l, gc);
    const unsigned long long want = ~static_cast<unsigned long long>(r);
    uint32_t pos = slot_home(key, h.rev_log_cap);
    for (uint32_t it = 0; it < rcap; ++it) {
      const ulonglong2 sl = tab[pos];
      if (sl.x == key) {
        if (sl.y < want) atomicMax(&tab[pos].y, want);
        break;
      }
      if (sl.x == 0ull) break;
      pos = (pos + 1) & (rcap - 1);
    }
  }
}

// Reverse group, step 3: each unresolved a takes the first of its buckets (in
// scale order) that some b marked; the points resolved come off *h.left.
template <int DT, int W>
__global__ void __launch_bounds__(128) k_rev_resolve(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                     int64_t* bidx, uint8_t* level) {
  pdl_entry();
  if (group_mode(h) != GM_REV) return;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, t, src.dd, L, L0, nl);
  const uint32_t rcap = 1u << h.rev_log_cap;
  unsigned resolved = 0;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
    if (level[r] < L) continue;
    float y[W];
    load_row<DT, W>(src, r, y);
    for (int l = 0; l < nl; ++l) {
      const ulonglong2* tab = h.rev + size_t(l) * rcap;
      const uint64_t key = group_key(y, src.dd, l, gc);
      uint32_t pos = slot_home(key, h.rev_log_cap);
      unsigned long long yb = 0;
      for (uint32_t it = 0; it < rcap; ++it) {
        const ulonglong2 sl = tab[pos];
        if (sl.x == key) {
          yb = sl.y;
          break;
        }
        if (sl.x == 0ull) break;
        pos = (pos + 1) & (rcap - 1);
      }
      if (yb) {
        bidx[r] = static_cast<int64_t>(~yb);
        level[r] = static_cast<uint8_t>(L0 + l);
        ++resolved;
        break;
      }
    }
  }
  take_off_left(h, resolved);
}

// Each unresolved a walks the scales of the group in increasing order and
// stops at the first bucket that holds a b (Fig. 2, step 3); the points this
// group resolves come off *h.left.
template <int DT, int W, bool WIDE>
__global__ void __launch_bounds__(128) k_table_probe(HashSrc src, int L, int L0, int nl, ScaleTables t, HashTable h,
                                                     int64_t* bidx, uint8_t* level) {
  pdl_entry();
  if (group_mode(h) != GM_FWD) return;
  __shared__ GroupConsts<WIDE ? 4 : W> gc;
  if constexpr (!WIDE) load_group_consts(gc, t, src.dd, L, L0, nl);
  const size_t cap = size_t(1) << h.log_cap;
  unsigned resolved = 0;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gridDim.x) * blockDim.x) {
    if (L0 > 0 && level[r] < L) continue;  // resolved at a finer scale group
    if (L0 == 0) {
      // first group: start from "no scale collides" (b = 0, level = L)
      bidx[r] = 0;
      level[r] = static_cast<uint8_t>(L);
    }
    bool found = false;
    if constexpr (!WIDE) {  // rows in registers (dd <= W); the wide form is compiled only where needed
      float y[W];
      load_row<DT, W>(src, r, y);
      for (int l = 0; l < nl && !found; ++l) {
        const int64_t b = table_find(h.slots + size_t(l) * cap, h.log_cap, group_key(y, src.dd, l, gc));
        if (b >= 0) {
          bidx[r] = b;
          level[r] = static_cast<uint8_t>(L0 + l);
          found = true;
        }
      }
    } else {
      for (int b0 = 0; b0 < nl && !found; b0 += kLevelBlock) {
        uint64_t key[kLevelBlock];
        const int nb = min(kLevelBlock, nl - b0);
        stream_keys<DT>(src, r, L, L0 + b0, nb, t, key);
#pragma unroll
        for (int l = 0; l < kLevelBlock; ++l) {
          if (l >= nb || found) continue;
          const int64_t b = table_find(h.slots + size_t(b0 + l) * cap, h.log_cap, key[l]);
          if (b >= 0) {
            bidx[r] = b;
            level[r] = static_cast<uint8_t>(L0 + b0 + l);
            found = true;
          }
        }
      }
    }
    resolved += found;
  }
  if (h.left) take_off_left(h, resolved);
}

// Batched forms (one launch for many pairs, each pair's scales in one group):
// block run of pair p, local block i = (scale l, x) with x < gx_insert inserts
// B's rows x, x + gx_insert * 128, ... at scale l, as k_table_insert_ps does.
template <int DT, int W>
__global__ void __launch_bounds__(128) k_table_insert_batch(const CrudePair* P, const int* blk0, int np) {
  pdl_entry();
  const int pi = find_pair(blk0, np, blockIdx.x);
  const CrudePair& p = P[pi];
  const int local = blockIdx.x - __ldg(&blk0[pi]);
  const int gx = p.gx_insert;
  const int l = local / gx;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, p.t, p.B.dd, p.L, 0, p.L);
  const HashSrc src = p.B;
  const size_t cap = size_t(1) << p.log_cap;
  for (int64_t r = int64_t(local % gx) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gx) * blockDim.x) {
    float y[W];
    load_row<DT, W>(src, r, y);
    table_insert(p.slots + size_t(l) * cap, p.log_cap, group_key(y, src.dd, l, gc), r, p.status);
  }
}

// block run of pair p: each a walks the pair's scales in increasing order and
// stops at the first bucket that holds a b, as k_table_probe does for a single group
template <int DT, int W>
__global__ void __launch_bounds__(128) k_table_probe_batch(const CrudePair* P, const int* blk0, int np) {
  pdl_entry();
  const int pi = find_pair(blk0, np, blockIdx.x);
  const CrudePair& p = P[pi];
  const int local = blockIdx.x - __ldg(&blk0[pi]);
  const int gx = p.gx_probe;
  __shared__ GroupConsts<W> gc;
  load_group_consts(gc, p.t, p.A.dd, p.L, 0, p.L);
  const HashSrc src = p.A;
  const int L = p.L;
  const size_t cap = size_t(1) << p.log_cap;
  for (int64_t r = int64_t(local) * blockDim.x + threadIdx.x; r < src.n; r += int64_t(gx) * blockDim.x) {
    int64_t bb = 0;
    int lv = L;
    float y[W];
    load_row<DT, W>(src, r, y);
    for (int l = 0; l < L; ++l) {
      const int64_t b = table_find(p.slots + size_t(l) * cap, p.log_cap, group_key(y, src.dd, l, gc));
      if (b >= 0) {
        bb = b;
        lv = l;
        break;
      }
    }
    p.bidx[r] = bb;
    p.level[r] = static_cast<uint8_t>(lv);
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
    else if (dd <= kRegRow)
      f(dtc, std::integral_constant<int, kRegRow>{});
    else
      f(dtc, std::integral_constant<int, kRegRowMax>{});
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

// Grids of the table kernels: grid-stride over the points, two waves of the
// blocks that fit on the SMs at once (a skipped group then costs a short launch;
// 1M x 384 CrudeNN: 1.070 ms at one wave, 1.039 ms at two, 1.111 ms with a block
// per 128 points).
template <class K>
static int table_grid(K kernel, int64_t n, int sm_count) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> per_sm_of;  // resident 128-thread blocks per SM, per kernel
  int per_sm;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = per_sm_of.find(reinterpret_cast<const void*>(kernel));
    if (it == per_sm_of.end()) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 128, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 4;
      }
      it = per_sm_of.emplace(reinterpret_cast<const void*>(kernel), b).first;
    }
    per_sm = it->second;
  }
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 128), int64_t(sm_count) * per_sm * 2)));
}

void launch_table_clear(HashTable h, int nl, int sm_count, cudaStream_t s) {
  const int64_t n16 = int64_t(nl) << h.log_cap;  // 16-byte slots
  const int grid = static_cast<int>(std::min<int64_t>(ceil_div(n16, 1024), int64_t(sm_count) * 2));
  launch_k(k_table_clear, grid, 1024, 0, s, h, n16);
  launch_check("table_clear");
}

void launch_group_insert(HashSrc B, int L, int L0, int nl, ScaleTables t, HashTable h, uint32_t* status, int sm_count,
                         cudaStream_t s) {
  if (B.n == 0) return;
  if (B.dd <= kRegRowMax) {
    dispatch_dt_w(B.dtype, B.dd, [&](auto dtc, auto wc) {
      auto kern = k_table_insert_ps<decltype(dtc)::value, decltype(wc)::value>;
      // the nl block rows (one per scale) share the grid's two waves: sized for a
      // row count of n * nl, so a group of many scales keeps every row in its own
      // thread where the waves allow (100k x 128, 10 scales: CrudeNN 0.163 -> 0.110 ms; 4096 d = 3
      // pairs: l2 149.3 -> 139.9 ms per batch)
      const int gx = std::max(1, table_grid(kern, B.n * nl, sm_count) / nl);
      launch_k(kern, dim3(static_cast<unsigned>(gx), static_cast<unsigned>(nl)), 128, 0, s, B, L, L0, nl, t, h,
               status);
    });
    launch_check("table_insert");
    return;
  }
  switch (B.dtype) {
    case CH_F32:
      launch_k(k_table_insert<CH_F32>, table_grid(k_table_insert<CH_F32>, B.n, sm_count), 128, 0, s, B, L, L0, nl, t,
               h, status);
      break;
    case CH_BF16:
      launch_k(k_table_insert<CH_BF16>, table_grid(k_table_insert<CH_BF16>, B.n, sm_count), 128, 0, s, B, L, L0, nl,
               t, h, status);
      break;
    default:
      launch_k(k_table_insert<CH_FP8E4M3>, table_grid(k_table_insert<CH_FP8E4M3>, B.n, sm_count), 128, 0, s, B, L,
               L0, nl, t, h, status);
      break;
  }
  launch_check("table_insert");
}

void launch_group_probe(HashSrc A, int L, int L0, int nl, ScaleTables t, HashTable h, int64_t* bidx, uint8_t* level,
                        int sm_count, cudaStream_t s) {
  if (A.n == 0) return;

  dispatch_dt_w(A.dtype, A.dd, [&](auto dtc, auto wc) {
    constexpr int DT = decltype(dtc)::value, W = decltype(wc)::value;
    if (A.dd <= W)  // the register form alone: 48 registers instead of 127, so 2.5x the resident warps
      launch_k(k_table_probe<DT, W, false>, table_grid(k_table_probe<DT, W, false>, A.n, sm_count), 128, 0, s, A, L,
               L0, nl, t, h, bidx, level);
    else
      launch_k(k_table_probe<DT, W, true>, table_grid(k_table_probe<DT, W, true>, A.n, sm_count), 128, 0, s, A, L,
               L0, nl, t, h, bidx, level);
  });
  launch_check("table_probe");
}

void launch_insert_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int dd, cudaStream_t s) {
  if (np == 0 || blocks == 0) return;
  CHX_CHECK(dd <= kRegRowMax, CH_EINVAL, "batched insert: hashed rows of <= 64 values");
  dispatch_dt_w(dtype, dd, [&](auto dtc, auto wc) {
    launch_k(k_table_insert_batch<decltype(dtc)::value, decltype(wc)::value>, blocks, 128, 0, s, P, blk0, np);
  });
  launch_check("table_insert_batch");
}

void launch_probe_batch(const CrudePair* P, const int* blk0, int np, int blocks, int dtype, int dd, cudaStream_t s) {
  if (np == 0 || blocks == 0) return;
  CHX_CHECK(dd <= kRegRowMax, CH_EINVAL, "batched probe: hashed rows of <= 64 values");
  dispatch_dt_w(dtype, dd, [&](auto dtc, auto wc) {
    launch_k(k_table_probe_batch<decltype(dtc)::value, decltype(wc)::value>, blocks, 128, 0, s, P, blk0, np);
  });
  launch_check("table_probe_batch");
}

void launch_group_reverse(HashSrc A, HashSrc B, int L, int L0, int nl, ScaleTables t, HashTable h, int64_t* bidx,
                          uint8_t* level, uint32_t* status, int sm_count, cudaStream_t s) {
  CHX_CHECK(A.dd <= kRegRow && B.dd <= kRegRow, CH_EINVAL, "reverse scale groups need hashed rows of <= 32 values");
  dispatch_dt_w(A.dtype, A.dd, [&](auto dtc, auto wc) {
    auto kern = k_rev_insert<decltype(dtc)::value, decltype(wc)::value>;
    launch_k(kern, table_grid(kern, A.n, sm_count), 128, 0, s, A, L, L0, nl, t, h, level, status);
  });
  launch_check("rev_insert");
  HashTable later = h;
  later.first = 0;
  dispatch_dt_w(B.dtype, B.dd, [&](auto dtc, auto wc) {
    auto kern = k_rev_stream<decltype(dtc)::value, decltype(wc)::value>;
    const int gx = std::max(1, table_grid(kern, B.n * nl, sm_count) / nl);
    launch_k(kern, dim3(static_cast<unsigned>(gx), static_cast<unsigned>(nl)), 128, 0, s, B, L, L0, nl, t, later);
  });
  launch_check("rev_stream");
  dispatch_dt_w(A.dtype, A.dd, [&](auto dtc, auto wc) {
    auto kern = k_rev_resolve<decltype(dtc)::value, decltype(wc)::value>;
    launch_k(kern, table_grid(kern, A.n, sm_count), 128, 0, s, A, L, L0, nl, t, later, bidx, level);
  });
  launch_check("rev_resolve");
}

}  // namespace chx
