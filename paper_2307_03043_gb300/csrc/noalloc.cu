// noalloc.cu -- ch_sample_static: the sampling step (ch_sample) for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins whose host application
// owns every device allocation, or processes working under a device-memory
// budget fixed before they start, where an allocation in the middle of a run
// could fail or is forbidden.  ch_sample_static does the same work as ch_sample
// without allocating anything: its scratch (the running maximum, the weight
// shift, the total, per-block sums and the inclusive prefix of the weights)
// lives in one file-scope __device__ array of fixed size, which every GPU that
// loads this library holds until the process exits.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace {

// largest nA the static scratch serves
constexpr int64_t kStaticMaxA = int64_t(1) << 20;
constexpr size_t kStaticBlocks = static_cast<size_t>(chx::sample_blocks_c(kStaticMaxA));  // weight-scan blocks

// layout inside the array (each part 256-byte aligned)
constexpr size_t kOffMax = 0;                                   // uint32 running max (ordered encoding)
constexpr size_t kOffS = 256;                                   // int32 weight shift S
constexpr size_t kOffW = 512;                                   // uint64 total weight W
constexpr size_t kOffBlocks = 768;                              // uint64 [kStaticBlocks]
constexpr size_t kOffPrefix = kOffBlocks + ((kStaticBlocks * 8 + 255) & ~size_t(255));  // uint64 [kStaticMaxA]
constexpr size_t kStaticBytes = kOffPrefix + size_t(kStaticMaxA) * 8;                    // ~8.4 MB

static __device__ __align__(256) unsigned char g_sample_scratch[kStaticBytes];
static_assert(kOffPrefix >= kOffBlocks + kStaticBlocks * sizeof(uint64_t),
              "the block-sum region holds one entry per weight-scan block of the largest nA");

// Host code may not use g_sample_scratch's name as a device address: its
// device address is looked up with the device current, once per CUDA context.
// The cache is keyed on the context's unique id, so after cudaDeviceReset (a new
// primary context, the module loaded again) the address is looked up afresh.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  unsigned long long ctx_id;
  void* addr;
};
Cached g_addr[kMaxDevices] = {};

// driver calls through the runtime's entry-point table, so that the library
// loads (and its CPU-side checks run) on machines without the driver
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <class F>
F driver_fn(const char* name, int version) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return reinterpret_cast<F>(p);
}

bool current_ctx_id(unsigned long long* id) {
  static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  return get_current(&c) == CUDA_SUCCESS && c && get_id(c, id) == CUDA_SUCCESS;
}

ch_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CH_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  const bool have_ctx = current_ctx_id(&id);
  if (!have_ctx || !g_addr[dev].addr || g_addr[dev].ctx_id != id) {
    void* p = nullptr;  // the look-up also makes the device's primary context current
    if (cudaGetSymbolAddress(&p, g_sample_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CH_ECUDA;
    }
    if (!current_ctx_id(&id)) return CH_ECUDA;
    g_addr[dev] = Cached{id, p};
  }
  *out = static_cast<unsigned char*>(g_addr[dev].addr);
  return CH_OK;
}

}  // namespace

extern "C" ch_status ch_sample_static(const float* D, int64_t nA, int64_t T, uint64_t seed, int64_t* idx, uint64_t* w,
                                      uint64_t* W_total, void* stream) {
  if (nA < 0 || T < 0) return CH_EINVAL;
  if (nA > kStaticMaxA) return CH_EINVAL;  // beyond the fixed scratch
  if ((nA > 0 && (!D || !w)) || (T > 0 && !idx)) return CH_EINVAL;
  unsigned char* base = nullptr;
  const ch_status st = scratch_for_current_device(&base);
  if (st != CH_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    chx::SampleWork sw;
    sw.maxD = reinterpret_cast<uint32_t*>(base + kOffMax);
    sw.S = reinterpret_cast<int32_t*>(base + kOffS);
    sw.W = reinterpret_cast<uint64_t*>(base + kOffW);
    sw.blocksum = reinterpret_cast<uint64_t*>(base + kOffBlocks);
    uint64_t* prefix = reinterpret_cast<uint64_t*>(base + kOffPrefix);
    // the weight pass clears the running maximum itself before using it
    chx::launch_weights(D, nA, w, prefix, sw, s);
    if (nA == 0) {
      if (T > 0) CHX_CUDA(cudaMemsetAsync(idx, 0xFF, size_t(T) * sizeof(int64_t), s));
    } else {
      chx::launch_draws(prefix, nA, sw.W, T, seed, idx, s);
    }
    if (W_total) CHX_CUDA(cudaMemcpyAsync(W_total, sw.W, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  } catch (const chx::Err& e) {
    return e.st;
  }
  return CH_OK;
}
