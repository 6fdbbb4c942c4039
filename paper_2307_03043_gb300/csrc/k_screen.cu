// k_screen.cu -- tensor-core screen for the sampled l2 scan (Fig. 1, step 3).
//
// For each sample q and every b: s(q, b) = |b|^2 - 2 q.b ranks b exactly like
// |q - b|^2 (|q|^2 is constant per sample).  The dot products are a dense
// contraction S = Q B^T run on the 5th-generation tensor cores:
//   * TMA (cp.async.bulk.tensor, 128-byte swizzle) stages Q (128 samples x d,
//     resident per work item below 768-byte rows, else streamed beside B) and B
//     tiles (256 points x one 128-byte K block) through a ring of shared-memory
//     stages;
//   * one elected thread issues tcgen05.mma (kind::tf32 for binary32 data,
//     kind::f16 with bf16 operands, kind::f8f6f4 with e4m3 operands) into a
//     double-buffered 128 x 256 binary32 accumulator in tensor memory;
//   * eight epilogue warps read the accumulator with tcgen05.ld (one row and a
//     128-column slice per thread), form s and keep, per residue class of
//     columns, the running minimum and the tile it came from.
// Work items are (128-sample tile, chunk of B) pairs spread over a persistent
// grid (up to 16 chunks, so that the items fill the SMs); a rerank kernel then
// takes each sample's R best screened entries over all chunks and evaluates the
// canonical binary32 distance on the columns each stands for, so the reported
// minimum is exact whenever the true nearest point survives the screen.
//
// Every mbarrier wait is bounded (about 2 s of SM clock, or the context's own
// budget); on expiry the CTA raises ST_TIMEOUT and stops issuing work.  Before
// its tensor memory is freed and it returns, the producer waits (with the full
// 2 s bound) for every copy it issued to land, and the MMA thread commits once
// more and waits for that commit, so no copy or MMA is still in flight.
#include "tma.cuh"

namespace chx {

namespace {

constexpr int kBM = 128;          // samples per tile (TMEM lanes)
constexpr int kBN = 256;          // B points per tile (accumulator columns)
constexpr int kKB = 128;          // bytes of K per stage (one 128B swizzle row)
constexpr int kEpiWarps = 8;      // epilogue warps: 2 per TMEM lane quadrant
constexpr int kSlices = kEpiWarps / 4;     // column slices of an accumulator tile
constexpr int kSliceCols = kBN / kSlices;  // 128 columns per epilogue thread and tile
constexpr int kThreads = 64 + 32 * kEpiWarps;  // warp 0 TMA, warp 1 MMA, warps 2.. epilogue
constexpr int kMaxChunks = 16;  // kSlices x 16 x kClasses = the rerank's 1024 candidates
// Each epilogue thread keeps one running minimum per residue class (column mod
// kClasses) of its slice; a class has kOcc columns in a tile slice, and the
// thread first takes their minimum (kOcc - 1 min operations), then updates the
// class's running (value, tile) pair once per tile.  A candidate is therefore a
// (tile, class) entry standing for kOcc columns, all of which the rerank
// evaluates exactly.
constexpr int kOcc = 4;
constexpr int kClasses = kSliceCols / kOcc;  // 32

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                  // leading byte offset (unused for SW128 K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                  // SWIZZLE_128B
  return d;
}

// instruction descriptor: D f32, A/B K-major, M = 128, N = 256
template <int SCREEN>
__host__ __device__ constexpr uint32_t idesc() {
  // operand format: tf32 = 2 (kind::tf32), bf16 = 1 (kind::f16), e4m3 = 0 (kind::f8f6f4)
  constexpr uint32_t fmt = SCREEN == CH_SCREEN_TF32 ? 2u : SCREEN == CH_SCREEN_BF16 ? 1u : 0u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(kBN >> 3) << 17) |
         (static_cast<uint32_t>(kBM >> 4) << 24);
}

template <int SCREEN>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t id = idesc<SCREEN>();
  if constexpr (SCREEN == CH_SCREEN_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
  } else if constexpr (SCREEN == CH_SCREEN_BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
  }
}

// 32 columns of this warp's 32 TMEM lanes; the registers are valid only after
// tmem_wait_ld()
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// the wait, with the 16 registers of a tmem_ld16_async tied to it so that no read
// of them is scheduled before it
__device__ __forceinline__ void tmem_wait_ld16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// 16 columns; valid after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct ScreenArgs {
  int64_t T;          // samples (rows of Q)
  int64_t nB;
  int kblocks;        // ceil(d * elem / 128)
  int row_tiles;
  int chunks;
  int64_t chunk_len;  // B points per chunk (multiple of kBN)
  int stages;
  int stream_q;       // 1: the sample tile's K blocks stream through the stages with B's (rows too wide to keep)
  const float* normB;   // |b|^2 [nB]
  const float* scaleB;  // FP8 row scales [nB] or null
  const float* scaleQ;  // FP8 sample scales [T] or null
  float* part_s;        // [chunks][T][R]
  int32_t* part_i;
  uint32_t* status;
  long long wait_cycles;  // budget of each pipeline wait (SM cycles)
};

// arrive on this CTA's mbarrier at shared address addr; relaxed: what it
// publishes (the tensor-memory reads) is ordered by the tcgen05 fences around it
__device__ __forceinline__ void mbar_arrive_relaxed(uint32_t addr) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// The epilogue (eight warps: warps 2 .. 9 of the block): one sample row per
// thread.  Warp w reads TMEM lane quadrant w % 4 (the only one it may access) and
// one 128-column slice of each accumulator tile, forms the scores and keeps, per
// residue class of columns, the running minimum and the tile it came from.  Work
// item `item` covers sample tile tile_of(item) and chunk item / items_per_chunk.
// After reading an accumulator each warp arrives once on acc_empty[acc] (given by
// its shared address).
template <int SCREEN, class TileOf>
__device__ __forceinline__ void screen_epilogue(const ScreenArgs& args, int first_item, int item_stride, int n_items,
                                              int items_per_chunk, TileOf tile_of, uint32_t tmem_base,
                                              float* nb_s, float* sb_s, uint64_t* acc_full,
                                              const uint32_t (&acc_empty_c)[2], volatile int* abort_flag,
                                              long long budget) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ew = warp & 3;
  const int qs = (warp - 2) >> 2;  // column slice
  const int row = ew * 32 + lane;
  uint32_t acc = 0, accphase = 0;
  for (int item = first_item; item < n_items && !*abort_flag; item += item_stride) {
    const int mt = tile_of(item), ck = item / items_per_chunk;
    const int64_t b_begin = int64_t(ck) * args.chunk_len;
    const int64_t b_end = min(args.nB, b_begin + args.chunk_len);
    const int64_t grow = int64_t(mt) * kBM + row;
    float sq = 1.0f;
    if constexpr (SCREEN == CH_SCREEN_FP8) sq = (grow < args.T) ? args.scaleQ[grow] : 1.0f;
    const uint64_t sq2 = f2_pack(sq, sq);
    const uint64_t neg2 = f2_pack(-2.0f, -2.0f);
    // running minima per residue class of this warp's slice; best_c holds the
    // tile (within the chunk) of each minimum
    float best_s[kClasses];
    int32_t best_c[kClasses];
#pragma unroll
    for (int i = 0; i < kClasses; ++i) {
      best_s[i] = __int_as_float(0x7F800000);
      best_c[i] = -1;
    }
    int32_t tile = 0;  // tile index within the chunk
    // |b|^2 (and -2 x FP8 scale) of this lane's columns of a tile slice,
    // fetched one tile ahead so the load latency hides behind a tile of work;
    // +inf past the end of the chunk
    constexpr int kPer = kSliceCols / 32;
    float pn[kPer], ps[kPer];
    auto prefetch_norms = [&](int64_t t0) {
      const int64_t base = t0 + qs * kSliceCols;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int64_t b = base + lane + 32 * k;
        pn[k] = (b < b_end) ? __ldg(&args.normB[b]) : __int_as_float(0x7F800000);
        ps[k] = 0.0f;
        if constexpr (SCREEN == CH_SCREEN_FP8) ps[k] = (b < b_end) ? -2.0f * __ldg(&args.scaleB[b]) : 0.0f;
      }
    };
    prefetch_norms(b_begin);
    bool ok = true;
    for (int64_t b0 = b_begin; b0 < b_end; b0 += kBN) {
      // stage |b|^2 (and -2 x FP8 scale) of this tile in this warp's own buffer;
      // +inf past the end of B.  Only __syncwarp is used inside the epilogue, so
      // a warp that gives up on a wait can never strand another one.
      float* nb = nb_s + ((warp - 2) * 2 + acc) * kSliceCols;
      float* sb = sb_s + ((warp - 2) * 2 + acc) * kSliceCols;
      // this tile's norms were fetched into registers during the previous tile
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        nb[lane + 32 * k] = pn[k];
        if constexpr (SCREEN == CH_SCREEN_FP8) sb[lane + 32 * k] = ps[k];
      }
      __syncwarp();
      prefetch_norms(b0 + kBN);  // next tile's, consumed one tile from now
      const bool got = mbar_wait(&acc_full[acc], accphase, abort_flag, budget);
      if (!__all_sync(0xFFFFFFFFu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(ew * 32) << 16) + acc * kBN + qs * kSliceCols;
      // scores s = |b|^2 - 2 q.b (FP8: |b|^2 - 2 s_q s_b q8.b8) of the 16 columns
      // ch*16 .. ch*16+15 of the slice, two columns per packed instruction (each
      // half rounded as fmaf and __fmul_rn round)
      auto scores = [&](const uint32_t(&r)[16], int ch, float(&o)[16]) {
        const float4* nb4 = reinterpret_cast<const float4*>(nb + ch * 16);
        const float4* sb4 = reinterpret_cast<const float4*>(sb + ch * 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 n = nb4[q];
          uint64_t m01 = neg2, m23 = neg2;
          if constexpr (SCREEN == CH_SCREEN_FP8) {
            const float4 m = sb4[q];  // -2 x column scale, times this row's sample scale
            m01 = f2_mul(f2_pack(m.x, m.y), sq2);
            m23 = f2_mul(f2_pack(m.z, m.w), sq2);
          }
          uint64_t s01 = f2_pack(n.x, n.y), s23 = f2_pack(n.z, n.w);
          f2_fma(s01, m01, f2_pack(__uint_as_float(r[4 * q + 0]), __uint_as_float(r[4 * q + 1])));
          f2_fma(s23, m23, f2_pack(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3])));
          const float2 a = f2_unpack(s01), b = f2_unpack(s23);
          o[4 * q + 0] = a.x;
          o[4 * q + 1] = a.y;
          o[4 * q + 2] = b.x;
          o[4 * q + 3] = b.y;
        }
      };
      // Chunk ch holds classes (ch*16) mod kClasses + i (occurrence ch*16 / kClasses),
      // so chunks 0, 2, 4, 6 cover classes 0..15 and 1, 3, 5, 7 classes 16..31.  The
      // chunks are read in that order, two 16-column register buffers deep (the next
      // chunk loads while this one is scored); per half, the tile minimum of a class
      // is min(min(s0, s2), s4, s6), then the class's running (value, tile) pair
      // takes one update.
      static_assert(kSliceCols == 128 && kClasses == 32 && kOcc == 4, "chunk order below assumes 8 x 16 columns");
      constexpr int kOrder[8] = {0, 2, 4, 6, 1, 3, 5, 7};
      uint32_t ra[16], rb[16];
      float tm[16], pend[16], sc[16];
      // one running-minimum update per class and tile (classes h .. h+15)
      auto update = [&](int h) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const bool lt = tm[i] < best_s[h + i];
          best_s[h + i] = lt ? tm[i] : best_s[h + i];
          best_c[h + i] = lt ? tile : best_c[h + i];
        }
      };
      tmem_ld16_async(taddr + kOrder[0] * 16, ra);
      tmem_wait_ld16(ra);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint32_t(&cur)[16] = (k & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (k & 1) ? ra : rb;
        if (k + 1 < 8) tmem_ld16_async(taddr + kOrder[k + 1] * 16, nxt);
        const int occ = k & 3;
        if (occ == 0) {
          scores(cur, kOrder[k], tm);
        } else if (occ == 1) {
          scores(cur, kOrder[k], sc);
#pragma unroll
          for (int i = 0; i < 16; ++i) tm[i] = fminf(tm[i], sc[i]);
        } else if (occ == 2) {
          scores(cur, kOrder[k], pend);
        } else {
          scores(cur, kOrder[k], sc);
#pragma unroll
          for (int i = 0; i < 16; ++i) tm[i] = fmin3(tm[i], pend[i], sc[i]);
          if (k == 3) update(0);  // the second half's update follows the arrival below
        }
        if (k + 1 < 8) tmem_wait_ld16(nxt);
      }
      // the warp's tensor-memory reads are complete (tcgen05.wait::ld is warp-wide):
      // one arrival per warp frees the accumulator
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_relaxed(acc_empty_c[acc]);
      update(16);
      ++tile;
      acc ^= 1;
      if (acc == 0) accphase ^= 1;
      __syncwarp();  // this warp's staging buffer is rewritten two tiles later
    }
    if (!ok) break;
    if (grow < args.T) {
      // entry (tile t, class i) stands for columns
      // b_begin + t*256 + slice*kSliceCols + o*kClasses + i, o = 0 .. kOcc-1
      const size_t base = (size_t(ck * kSlices + qs) * args.T + grow) * kClasses;
#pragma unroll
      for (int i = 0; i < kClasses; ++i) {
        const int32_t t = best_c[i];
        args.part_s[base + i] = best_s[i];
        args.part_i[base + i] =
            t < 0 ? -1 : static_cast<int32_t>(b_begin + int64_t(t) * kBN + qs * kSliceCols + i);
      }
    }
  }
  }

template <int SCREEN, bool STREAMQ>
__global__ void __launch_bounds__(kThreads, 1)
    k_screen(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmB, ScreenArgs args) {
  pdl_entry();
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned by an offset from the shared array itself, so that the
  // compiler keeps every access below in the shared state space
  uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int KB = args.kblocks;
  const int S = args.stages;
  constexpr bool streamq = STREAMQ;  // the sample tile streams with B (rows of 768 bytes or more)
  uint8_t* q_smem = smem;  // KB x (128 rows x 128 B) resident, or S x (128 rows x 128 B) streamed
  uint8_t* b_smem = q_smem + size_t(streamq ? S : KB) * kBM * kKB;  // S x (256 rows x 128 B)
  float* nb_s = reinterpret_cast<float*>(b_smem + size_t(S) * kBN * kKB);  // [warps][2][64] |b|^2
  float* sb_s = nb_s + 2 * kEpiWarps * kSliceCols;                         // [warps][2][64] -2 x FP8 scale
  uint64_t* bars = reinterpret_cast<uint64_t*>(sb_s + 2 * kEpiWarps * kSliceCols);
  uint64_t* full = bars;            // [S]
  uint64_t* empty = bars + S;       // [S]
  uint64_t* q_full = bars + 2 * S;  // [1]
  uint64_t* q_empty = q_full + 1;   // [1]
  uint64_t* acc_full = q_empty + 1; // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* drain = acc_empty + 2;     // [1] the MMA thread's last commit
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(q_full, 1);
    mbar_init(q_empty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kEpiWarps);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(2 * kBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int n_items = args.row_tiles * args.chunks;
  const long long budget = args.wait_cycles;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, qphase = 0;
      // the stages (bit s) and the sample tile (q_issued) this thread has loaded,
      // and the barrier phase of each one's last copy
      uint32_t issued = 0, last_par = 0;
      bool q_issued = false;
      uint32_t q_par = 0;
      for (int item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
        const int mt = item % args.row_tiles, ck = item / args.row_tiles;
        const int64_t b_begin = int64_t(ck) * args.chunk_len;
        const int64_t b_end = min(args.nB, b_begin + args.chunk_len);
        constexpr int kEs = SCREEN == CH_SCREEN_TF32 ? 4 : SCREEN == CH_SCREEN_BF16 ? 2 : 1;
        if (!streamq) {
          if (!mbar_wait(q_empty, qphase ^ 1, abort_flag, budget)) break;
          mbar_expect_tx(q_full, uint32_t(KB) * kBM * kKB);
          for (int kb = 0; kb < KB; ++kb)
            tma_load_2d(q_smem + size_t(kb) * kBM * kKB, &tmQ, kb * kKB / kEs, mt * kBM, q_full);
          q_issued = true;
          q_par = qphase;
          qphase ^= 1;
        }
        bool ok = true;
        for (int64_t b0 = b_begin; b0 < b_end && ok; b0 += kBN) {
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, budget)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&full[stage], uint32_t(kBN) * kKB + (streamq ? uint32_t(kBM) * kKB : 0u));
            if (streamq)  // this K block of the sample tile rides along with B's
              tma_load_2d(q_smem + size_t(stage) * kBM * kKB, &tmQ, kb * kKB / kEs, mt * kBM, &full[stage]);
            tma_load_2d(b_smem + size_t(stage) * kBN * kKB, &tmB, kb * kKB / kEs, static_cast<int>(b0),
                        &full[stage]);
            issued |= 1u << stage;
            last_par = (last_par & ~(1u << stage)) | (phase << stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // drain: every copy issued has landed before the CTA's memory is released
      // (at once after a normal run, whose copies the MMAs have consumed)
      for (int st = 0; st < S; ++st)
        if (issued >> st & 1u) mbar_wait_bounded(&full[st], last_par >> st & 1u);
      if (q_issued) mbar_wait_bounded(q_full, q_par);
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, qphase = 0;
      uint32_t acc = 0, accphase = 0;
      for (int item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
        const int ck = item / args.row_tiles;
        const int64_t b_begin = int64_t(ck) * args.chunk_len;
        const int64_t b_end = min(args.nB, b_begin + args.chunk_len);
        if (!streamq) {
          if (!mbar_wait(q_full, qphase, abort_flag, budget)) break;
          qphase ^= 1;
          tc_fence_after();
        }
        bool ok = true;
        for (int64_t b0 = b_begin; b0 < b_end && ok; b0 += kBN) {
          if (!mbar_wait(&acc_empty[acc], accphase ^ 1, abort_flag, budget)) break;
          tc_fence_after();
          const uint32_t dtmem = tmem_base + acc * kBN;
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait(&full[stage], phase, abort_flag, budget)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t qa = su32(q_smem + size_t(streamq ? stage : kb) * kBM * kKB);
            const uint32_t ba = su32(b_smem + size_t(stage) * kBN * kKB);
#pragma unroll
            for (int k = 0; k < kKB / 32; ++k)  // 32 bytes of K per instruction
              tc_mma<SCREEN>(dtmem, sdesc(qa + k * 32), sdesc(ba + k * 32), (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[stage]);
            if (++stage == S) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          tc_commit(&acc_full[acc]);
          acc ^= 1;
          if (acc == 0) accphase ^= 1;
        }
        if (!streamq) tc_commit(q_empty);
        if (!ok) break;
      }
      // drain: this commit arrives once every MMA this thread issued has completed
      tc_commit(drain);
      mbar_wait_bounded(drain, 0);
    }
  } else {
    uint32_t acc_empty_c[2] = {su32(&acc_empty[0]), su32(&acc_empty[1])};
    screen_epilogue<SCREEN>(args, blockIdx.x, gridDim.x, n_items, args.row_tiles,
                            [&](int item) { return item % args.row_tiles; }, tmem_base, nb_s, sb_s, acc_full,
                            acc_empty_c, abort_flag, budget);
  }

  // ------------------------------------------------ teardown
  // (the producer and the MMA thread have drained their copies and MMAs above)
  __syncwarp();
  if (*abort_flag && threadIdx.x == 0) atomicOr(args.status, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * kBN) : "memory");
  }
}

// Gathers the sampled rows A[idx] into a dense [T][d] operand (raw storage type)
// and, for FP8, their scales; idx < 0 gives a zero row.
__global__ void k_gather_rows(const uint8_t* A, const float* scA, int64_t nA, int row_bytes, const int64_t* idx,
                              int64_t T, uint8_t* Q, float* sQ) {
  pdl_entry();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int words = row_bytes / 16;
  const int64_t row = t / words;
  const int w = static_cast<int>(t % words);
  if (row >= T) return;
  const int64_t a = idx ? idx[row] : row;
  uint4 v = make_uint4(0, 0, 0, 0);
  if (a >= 0 && a < nA) v = reinterpret_cast<const uint4*>(A + a * row_bytes)[w];
  reinterpret_cast<uint4*>(Q + row * row_bytes)[w] = v;
  if (sQ && w == 0) sQ[row] = (a >= 0 && a < nA) ? scA[a] : 1.0f;
}

CUtensorMap make_map(const void* base, int dtype, int64_t rows, int d, int box_rows) {
  CUtensorMap m;
  const int es = static_cast<int>(elem_size(dtype));
  const CUtensorMapDataType t = dtype == CH_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : dtype == CH_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(d), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(d) * es};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kKB / es), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, t, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CHX_CHECK(r == CUDA_SUCCESS, CH_ECUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

struct Plan {
  int kblocks, row_tiles, chunks, stages, R;
  bool stream_q;
  int64_t chunk_len, T;
  size_t smem;
  int grid;
};

int screen_dtype(int screen) { return screen == CH_SCREEN_TF32 ? CH_F32 : screen == CH_SCREEN_BF16 ? CH_BF16 : CH_FP8E4M3; }

Plan make_plan(int64_t T, int64_t nB, int d, int R, int sm_count, int chunk_sms, int screen) {
  Plan p;
  const int es = static_cast<int>(elem_size(screen_dtype(screen)));
  p.T = T;
  p.R = std::max(1, std::min(R, 32));  // candidates the rerank evaluates exactly
  p.kblocks = static_cast<int>(ceil_div(int64_t(d) * es, kKB));
  p.row_tiles = static_cast<int>(ceil_div(std::max<int64_t>(T, 1), kBM));
  // the sample tile stays resident below 96 KB (d * elem < 768 bytes); wider rows
  // stream, which leaves room for four or more B stages (at 768-byte rows a
  // resident tile leaves three, and the bf16 d = 384 screen ran 3.01 ms resident
  // against 2.81 ms streamed on 1M x 1M)
  p.stream_q = int64_t(p.kblocks) * kBM * kKB >= 96 * 1024;
  const size_t limit = 227 * 1024;
  const size_t fixed = 1024 + (p.stream_q ? 0 : size_t(p.kblocks) * kBM * kKB) + 16 * kBN * sizeof(float) + 256;
  const size_t per_stage = size_t(kBN) * kKB + (p.stream_q ? size_t(kBM) * kKB : 0);
  p.stages = static_cast<int>(std::min<size_t>(6, (limit - std::min(limit, fixed)) / per_stage));
  p.smem = fixed + size_t(p.stages) * per_stage;
  // chunks: smallest count whose items fill chunk_sms SMs to >= 90 % (at most
  // kMaxChunks); more chunks also mean more rerank candidates per sample
  const int fill = chunk_sms > 0 ? std::min(chunk_sms, sm_count) : sm_count;
  const int64_t btiles = ceil_div(nB, kBN);
  int best_c = 1;
  double best_eff = 0.0;
  for (int c = 1; c <= kMaxChunks && c <= btiles; ++c) {
    if (kSlices * c * kClasses > kRerankMaxCand) break;  // kSlices column slices per chunk
    const int64_t items = int64_t(p.row_tiles) * c;
    const int64_t rounds = ceil_div(items, fill);
    const double eff = double(items) / double(rounds * fill);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best_c = c;
    }
    if (eff >= 0.9) break;
  }
  p.chunks = best_c;
  p.chunk_len = ceil_div(ceil_div(nB, p.chunks), kBN) * kBN;
  p.chunks = static_cast<int>(ceil_div(nB, p.chunk_len));
  p.grid = static_cast<int>(std::min<int64_t>(int64_t(p.row_tiles) * p.chunks, sm_count));
  return p;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // a function-local static is initialised once, thread-safely
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CHX_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    CHX_CHECK(p && q == cudaDriverEntryPointSuccess, CH_ENOTSUP, "cuTensorMapEncodeTiled unavailable");
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

bool screen_supported(int screen, const ch_set* A, const ch_set* B) {
  if (screen != CH_SCREEN_TF32 && screen != CH_SCREEN_BF16 && screen != CH_SCREEN_FP8) return false;
  if (A->dtype != screen_dtype(screen) || B->dtype != screen_dtype(screen)) return false;
  const int es = static_cast<int>(elem_size(A->dtype));
  if ((int64_t(A->d) * es) % 16 != 0) return false;     // TMA row stride
  if (int64_t(A->d) * es < kKB) return false;            // at least one full 128-byte swizzle row
  if (int64_t(A->d) * es > 16384) return false;          // rows up to 16 KB (768 B or more stream)
  if (B->n >= (int64_t(1) << 31)) return false;
  return true;
}

size_t screen_workspace(int64_t T, int64_t nB, int d, int R, int sm_count, int chunk_sms, int screen) {
  const Plan p = make_plan(T, nB, d, R, sm_count, chunk_sms, screen);
  const int es = static_cast<int>(elem_size(screen_dtype(screen)));
  const size_t q = ((size_t(T) * d * es + 255) & ~size_t(255)) + ((size_t(T) * 4 + 255) & ~size_t(255));
  const size_t parts = size_t(kSlices * p.chunks) * T * kClasses * 8 + 512;
  return q + parts + 1024;
}

void launch_screen_l2(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int screen, int R, void* work,
                      float* min_d, int64_t* argmin, uint32_t* status, int sm_count, int chunk_sms,
                      cudaStream_t s, const KernelTimer& timer, long long wait_cycles) {
  if (T == 0) return;
  const Plan p = make_plan(T, B->n, A->d, R, sm_count, chunk_sms, screen);
  const int es = static_cast<int>(elem_size(A->dtype));
  const int row_bytes = A->d * es;
  uint8_t* w = static_cast<uint8_t*>(work);
  uint8_t* Q = w;
  w += (size_t(T) * row_bytes + 255) & ~size_t(255);
  float* sQ = reinterpret_cast<float*>(w);
  w += (size_t(T) * 4 + 255) & ~size_t(255);
  float* part_s = reinterpret_cast<float*>(w);
  w += (size_t(kSlices * p.chunks) * T * kClasses * 4 + 255) & ~size_t(255);
  int32_t* part_i = reinterpret_cast<int32_t*>(w);

  const int64_t words = T * (row_bytes / 16);
  launch_k(k_gather_rows, static_cast<int>(ceil_div(words, 256)), 256, 0, s, 
      static_cast<const uint8_t*>(A->data), A->scales, A->n, row_bytes, qidx, T, Q,
      screen == CH_SCREEN_FP8 ? sQ : nullptr);
  launch_check("gather_rows");

  const CUtensorMap tmQ = make_map(Q, A->dtype, T, A->d, kBM);
  const CUtensorMap tmB = make_map(B->data, B->dtype, B->n, B->d, kBN);
  ScreenArgs a;
  a.T = T;
  a.nB = B->n;
  a.kblocks = p.kblocks;
  a.row_tiles = p.row_tiles;
  a.chunks = p.chunks;
  a.chunk_len = p.chunk_len;
  a.stages = p.stages;
  a.stream_q = p.stream_q ? 1 : 0;
  a.normB = B->norms;
  a.scaleB = B->scales;
  a.scaleQ = sQ;
  a.part_s = part_s;
  a.part_i = part_i;
  a.status = status;
  a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTimeoutCycles;

#define CHX_SCREEN_LAUNCH(SCR)                                                                              \
  do {                                                                                                      \
    auto kern = p.stream_q ? k_screen<SCR, true> : k_screen<SCR, false>;                                    \
    CHX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)); /* constant */ \
    timer.start(s);                                                                                         \
    launch_k(kern, p.grid, kThreads, p.smem, s, tmQ, tmB, a);                                               \
    timer.stop(s);                                                                                          \
  } while (0)
  if (screen == CH_SCREEN_TF32) CHX_SCREEN_LAUNCH(CH_SCREEN_TF32);
  else if (screen == CH_SCREEN_BF16) CHX_SCREEN_LAUNCH(CH_SCREEN_BF16);
  else CHX_SCREEN_LAUNCH(CH_SCREEN_FP8);
#undef CHX_SCREEN_LAUNCH
  launch_check("screen");

  launch_rerank(A, qidx, T, B, part_s, part_i, kSlices * p.chunks, kClasses, kOcc, kClasses, p.R, min_d, argmin, s);
}

}  // namespace chx
