// k_screen.cu -- tensor-core screen of the sampled l2 scan (placeholder until
// the tcgen05 kernel lands: reports no support, so callers use the exact scan).
#include "common.cuh"

namespace chx {

bool screen_supported(int screen, const ch_set* A, const ch_set* B) {
  (void)screen; (void)A; (void)B;
  return false;
}

size_t screen_workspace(int64_t T, int64_t nB, int d, int R, int sm_count, int screen) {
  (void)T; (void)nB; (void)d; (void)R; (void)sm_count; (void)screen;
  return 256;
}

void launch_screen_l2(const ch_set* A, const int64_t* qidx, int64_t T, const ch_set* B, int screen, int R,
                      void* work, float* min_d, int64_t* argmin, uint32_t* status, int sm_count, cudaStream_t s) {
  (void)A; (void)qidx; (void)T; (void)B; (void)screen; (void)R; (void)work; (void)min_d; (void)argmin;
  (void)status; (void)sm_count; (void)s;
  throw Err{CH_ENOTSUP, "tensor-core screen not built"};
}

}  // namespace chx
