// MRF-ZOOM kernel (placeholder until the persistent search kernel lands).
#include "mrf_internal.h"

int run_zoom(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, const mrf_zoom_opts *opts,
             const void *fp, int64_t V, mrf_result *out, cudaStream_t stream)
{
    (void)ctx; (void)seq; (void)grid; (void)opts; (void)fp; (void)V; (void)out; (void)stream;
    return set_error(MRF_E_UNSUPPORTED, "MRF-ZOOM kernel not built yet");
}
