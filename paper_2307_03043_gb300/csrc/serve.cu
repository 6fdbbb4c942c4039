// serve.cu -- request loop (placeholder: every call reports CH_ENOTSUP).
#include "common.cuh"

extern "C" {
ch_status ch_serve_create(ch_ctx*, const ch_serve_config*, ch_server**) { return CH_ENOTSUP; }
ch_status ch_serve_register(ch_server*, const void*, int, int64_t, int32_t, int32_t, const float*, uint64_t*) {
  return CH_ENOTSUP;
}
ch_status ch_serve_submit(ch_server*, uint64_t, uint64_t, const ch_est_params*, uint64_t*) { return CH_ENOTSUP; }
ch_status ch_serve_poll(ch_server*, uint64_t, double*, int32_t*) { return CH_ENOTSUP; }
ch_status ch_serve_wait(ch_server*, uint64_t, uint32_t, double*, int32_t*) { return CH_ENOTSUP; }
ch_status ch_serve_stats_get(ch_server*, ch_serve_stats*) { return CH_ENOTSUP; }
void ch_serve_destroy(ch_server*) {}
}
