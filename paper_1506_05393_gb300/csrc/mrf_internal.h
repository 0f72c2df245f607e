// Internal declarations shared by the library's translation units.
// Not part of the public ABI (include/mrf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mrf.h"

// ---------------------------------------------------------------------------
// Device-side views (plain structs passed by value to kernels)

// Sequence on the device. RF coefficients are in "deficit" form: the state is
// (Mx, My, W) with W = 1 - Mz (equilibrium M0 = 1), so that the longitudinal
// relaxation of Eq. A1 becomes W <- E1 W, a product with no cancellation.
struct SeqDev {
    int n;
    int xonly;          // every RF phase is a multiple of pi: R_RF is a rotation about x
    int symmetric;      // TE_j == TR_j - TE_j for every j (one evolution factor per step)
    int inversion;
    float inv_delay;    // ms
    const float4 *rfx;  // xonly: (c, s, 1 - c, TE_j) of the x-rotation by beta_j
    const float *rfg;   // general: 12 floats per j: R00..R22 row-major, 1 - R22, 0, 0
    const float2 *tau;  // (TE_j, TR_j - TE_j) in ms
    int finite;         // some RF pulse has a finite duration: R_RF depends on df (xonly is 0 then)
    const float4 *rff;  // finite: (-alpha cos phi, -alpha sin phi, alpha^2, 2 pi tau) per j
};

struct GridDev {
    int n_t1, n_t2, n_df;
    const float *t1;        // n_t1 values, ms
    const float *t2;        // n_t2 values, ms
    const float *df;        // n_df values, Hz
    const int64_t *a_off;   // n_t1 + 1: linear index of the first entry with T1 index a
    const int32_t *nb;      // n_t1: number of valid T2 indices for T1 index a
    int64_t count;
    int a_full;             // from this T1 index on every T2 index is valid (nb[a] == n_t2)
};

// ---------------------------------------------------------------------------
// Host-side objects behind the opaque ABI handles

struct mrf_seq {
    int32_t n = 0;
    int xonly = 0, symmetric = 0, inversion = 0;
    double inv_delay = 0.0;
    double min_tr = 0.0;
    int finite = 0;
    float4 *rfx = nullptr;      // rfx, rfg, tau and rff live in one block from the stream-ordered pool
    float *rfg = nullptr;
    float2 *tau = nullptr;
    float4 *rff = nullptr;
    void *block = nullptr;
    size_t bytes = 0;
    SeqDev dev() const {
        SeqDev s;
        s.n = n; s.xonly = xonly; s.symmetric = symmetric; s.inversion = inversion;
        s.inv_delay = (float)inv_delay; s.rfx = rfx; s.rfg = rfg; s.tau = tau;
        s.finite = finite; s.rff = rff;
        return s;
    }
};

// Device copy of a grid's axis values and index offsets.
struct GridBuf {
    mrf_grid_desc desc{};
    float *t1 = nullptr, *t2 = nullptr, *df = nullptr;
    int64_t *a_off = nullptr;
    int32_t *nb = nullptr;
    int64_t count = 0;
    int a_full = 1 << 30;       // set by grid_upload; the default never skips the table
    void *block = nullptr;      // t1, t2, df, a_off, nb in one block from the stream-ordered pool
    size_t bytes = 0;
    GridDev dev() const {
        GridDev g;
        g.n_t1 = desc.n_t1; g.n_t2 = desc.n_t2; g.n_df = desc.n_df;
        g.t1 = t1; g.t2 = t2; g.df = df; g.a_off = a_off; g.nb = nb; g.count = count; g.a_full = a_full;
        return g;
    }
};

struct mrf_dict {
    mrf_seq *seq = nullptr;     // private copy of the generating sequence
    GridBuf grid;
    int32_t dtype = 0;
    int64_t entries = 0;
    int32_t n = 0, ld = 0;
    void *hi = nullptr;
    void *lo = nullptr;
    float *norm = nullptr;
    float *scale = nullptr;
    void *block = nullptr;       // one stream-ordered pool allocation holding hi, lo, norm, scale
    size_t block_bytes = 0;
    size_t bytes = 0;
    // temporal smoothing applied to the stored entries (mrf_dict_smooth): half-width and
    // the weights w[k] = exp(-k^2 / (2 sigma^2)); the re-score smooths alike
    int smooth_h = 0;
    float smooth_w[3] = {1.f, 0.f, 0.f};
    int32_t smooth_width = 1;
    double smooth_sigma = 1.0;
};

struct ServeState;   // serve.cpp

enum ProfKind { kProfDictGen = 0, kProfMatcher = 1, kProfZoom = 2, kProfZoomLine = 3, kProfKinds = 4 };

struct ProfEvent {
    int kind;
    cudaEvent_t start, stop;
};

struct mrf_ctx {
    int device = 0;
    cudaStream_t aux = nullptr;  // the library's own non-blocking stream for small uploads
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    int *err_flag = nullptr;     // device int: set by kernels whose bounded waits run out
    unsigned long long *dev_stats = nullptr;   // device work counters (same allocation as err_flag)
    std::mutex mu;
    ServeState *serve = nullptr;
    // kernel accounting
    std::atomic<uint64_t> launches{0};
    std::atomic<uint64_t> kind_launches[kProfKinds];
    std::atomic<bool> profiling{false};
    std::mutex prof_mu;
    std::vector<ProfEvent> prof_pending;
    double prof_ms[kProfKinds] = {0, 0, 0, 0};
    uint64_t prof_timed[kProfKinds] = {0, 0, 0, 0};
    mrf_ctx() { for (auto &k : kind_launches) k = 0; }
};

// Profiling hooks around a main kernel launch (no-ops unless enabled).
struct ProfScope {
    mrf_ctx *ctx;
    int kind;
    cudaStream_t stream;
    cudaEvent_t start = nullptr;
    ProfScope(mrf_ctx *c, int k, cudaStream_t s);
    ~ProfScope();
};
inline void count_launch(mrf_ctx *ctx, int n = 1) { ctx->launches.fetch_add((uint64_t)n); }

// ---------------------------------------------------------------------------
// Helpers implemented in api.cu

int set_error(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
int budget_charge(mrf_ctx *ctx, size_t bytes);
void budget_release(mrf_ctx *ctx, size_t bytes);
// Small host-to-device uploads: one block from the stream-ordered pool, copied
// on the context's own non-blocking stream; the host waits for that copy only,
// never for work queued on the caller's streams.
int upload_block(mrf_ctx *ctx, const void *host, size_t bytes, void **dev, const char *what);
// Release a block: after every enqueued use (device-wide synchronisation) when
// `stream` is null and `sync` set, else in the order of `stream`.
void release_block(mrf_ctx *ctx, void *p, size_t bytes, cudaStream_t stream, bool sync);
int grid_validate(const mrf_grid_desc *g);
int grid_upload(mrf_ctx *ctx, const mrf_grid_desc *g, GridBuf *out);
void grid_release(mrf_ctx *ctx, GridBuf *g, cudaStream_t stream, bool sync);
// stream-ordered upload into one pool block; free with cudaFreeAsync + budget_release
int grid_upload_async(mrf_ctx *ctx, const mrf_grid_desc *g, cudaStream_t stream, GridDev *out, void **block,
                      size_t *bytes);
int seq_clone(mrf_ctx *ctx, const mrf_seq *src, mrf_seq **out);
void seq_release(mrf_ctx *ctx, mrf_seq *s, cudaStream_t stream, bool sync);
int check_device_error(mrf_ctx *ctx, cudaStream_t stream);   // synchronises; reads err_flag

// ---------------------------------------------------------------------------
// Launchers implemented in the kernel translation units

// bloch.cu
int launch_dict_generate(mrf_ctx *ctx, mrf_dict *d, cudaStream_t stream);
int launch_simulate(mrf_ctx *ctx, const mrf_seq *seq, int64_t count, const float *t1, const float *t2,
                    const float *df, void *out, cudaStream_t stream);

// match.cu
int run_match(mrf_ctx *ctx, const mrf_dict *d, const void *fp, int64_t V, int32_t precision, int32_t top_k,
              int rescore, mrf_result *out, int64_t *idx_out, float *cc2_out, cudaStream_t stream,
              bool fused = false);
// Chunked brute force: fold one range's results (part; nullptr = the first
// range, already in best) into best, with the range's first linear index
// `base` and first T1 index a0; second holds each voxel's runner-up CC.
int launch_chunk_merge(mrf_result *best, float *second, const mrf_result *part, int64_t V, int64_t base, int a0,
                       cudaStream_t stream);

// zoom.cu
int run_zoom(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, const mrf_zoom_opts *opts,
             const void *fp, int64_t V, mrf_result *out, cudaStream_t stream);

constexpr int kDeviceErrTimeout = 1;
constexpr int kDeviceErrBounds = 2;

#ifdef __CUDACC__
// Bounds-checked builds (compiled with -DMRF_CHECK): an index check that fails
// records kDeviceErrBounds in the context's error flag (mrf_stream_sync reports
// it) and the access it guards is skipped. Without MRF_CHECK every check is
// the constant true and compiles away.
__device__ __forceinline__ bool mrf_in_bounds(bool ok, int *err)
{
#ifdef MRF_CHECK
    if (!ok && err) atomicExch(err, kDeviceErrBounds);
    return ok;
#else
    (void)ok;
    (void)err;
    return true;
#endif
}
#endif
