// sssp_serve.cu -- serving loop (continuous batching).  Placeholder entry
// points until the persistent serving kernel lands; every call reports
// SSSP_E_INVAL so callers fail loudly.
#include "../../include/sssp.h"

extern "C" int sssp_serve_create(size_t, int32_t, int32_t, sssp_server** out) {
    if (out) *out = nullptr;
    return SSSP_E_INVAL;
}
extern "C" int sssp_serve_submit(sssp_server*, sssp_graph*, int32_t, void*, int32_t*, uint64_t*) {
    return SSSP_E_INVAL;
}
extern "C" int sssp_serve_poll(sssp_server*, uint64_t, int32_t*, int32_t*) { return SSSP_E_INVAL; }
extern "C" int sssp_serve_wait(sssp_server*, uint64_t, int32_t, int32_t*, int32_t*) { return SSSP_E_INVAL; }
extern "C" int sssp_serve_latency_us(sssp_server*, uint64_t, double*) { return SSSP_E_INVAL; }
extern "C" int sssp_serve_destroy(sssp_server*) { return SSSP_OK; }
