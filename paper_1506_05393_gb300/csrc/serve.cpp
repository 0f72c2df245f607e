// Serving loop (placeholder until continuous batching lands).
#include "mrf_internal.h"

extern "C" int mrf_serve_start(mrf_ctx *ctx, const mrf_serve_config *cfg) { (void)ctx; (void)cfg; return set_error(MRF_E_UNSUPPORTED, "serving not built yet"); }
extern "C" int mrf_serve_submit(mrf_ctx *ctx, const mrf_request *req, uint64_t *t) { (void)ctx; (void)req; (void)t; return set_error(MRF_E_UNSUPPORTED, "serving not built yet"); }
extern "C" int mrf_serve_poll(mrf_ctx *ctx, uint64_t t, int32_t ms, mrf_result *o) { (void)ctx; (void)t; (void)ms; (void)o; return set_error(MRF_E_UNSUPPORTED, "serving not built yet"); }
extern "C" int mrf_serve_cancel(mrf_ctx *ctx, uint64_t t) { (void)ctx; (void)t; return set_error(MRF_E_UNSUPPORTED, "serving not built yet"); }
extern "C" int mrf_serve_get_stats(mrf_ctx *ctx, mrf_serve_stats *s) { (void)ctx; (void)s; return set_error(MRF_E_UNSUPPORTED, "serving not built yet"); }
extern "C" int mrf_serve_stop(mrf_ctx *ctx) { (void)ctx; return MRF_OK; }
