// C-ABI entry points: context, budget, sequence, grid, dictionary, simulation,
// matching and ZOOM dispatch. Kernels live in bloch.cu, match.cu and zoom.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mrf_internal.h"

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return set_error(MRF_E_NOMEM, m);
    return set_error(MRF_E_CUDA, m);
}

extern "C" const char *mrf_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *mrf_version(void) { return "mrf-gb300 1.0 sm_103a"; }

// ---------------------------------------------------------------------------
// budget

int budget_charge(mrf_ctx *ctx, size_t bytes)
{
    size_t cur = ctx->used.load();
    for (;;) {
        if (cur + bytes > ctx->budget)
            return set_error(MRF_E_BUDGET, "HBM budget exceeded: need " + std::to_string(bytes) + " B, " +
                                                std::to_string(ctx->budget - cur) + " B left of " +
                                                std::to_string(ctx->budget));
        if (ctx->used.compare_exchange_weak(cur, cur + bytes)) return MRF_OK;
    }
}

void budget_release(mrf_ctx *ctx, size_t bytes) { ctx->used.fetch_sub(bytes); }

int upload_block(mrf_ctx *ctx, const void *host, size_t bytes, void **dev, const char *what)
{
    *dev = nullptr;
    if (bytes == 0) return MRF_OK;
    int rc = budget_charge(ctx, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMallocAsync(dev, bytes, ctx->aux);
    if (e == cudaSuccess && host) e = cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, ctx->aux);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux);
    if (e != cudaSuccess) {
        if (*dev) cudaFreeAsync(*dev, ctx->aux);
        *dev = nullptr;
        budget_release(ctx, bytes);
        return cuda_fail(e, what);
    }
    return MRF_OK;
}

void release_block(mrf_ctx *ctx, void *p, size_t bytes, cudaStream_t stream, bool sync)
{
    if (!p) return;
    if (sync) {
        cudaDeviceSynchronize();
        cudaFreeAsync(p, ctx->aux);
    } else {
        cudaFreeAsync(p, stream);
    }
    budget_release(ctx, bytes);
}

int check_device_error(mrf_ctx *ctx, cudaStream_t stream)
{
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read device error flag");
    if (flag) {
        cudaMemset(ctx->err_flag, 0, sizeof(int));
        if (flag == kDeviceErrTimeout)
            return set_error(MRF_E_TIMEOUT, "a device-side bounded wait ran out (kernel returned early)");
        return set_error(MRF_E_CUDA, "device-side check failed (code " + std::to_string(flag) + ")");
    }
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// context

extern "C" int mrf_ctx_create(int device, size_t hbm_budget_bytes, mrf_ctx **out)
{
    if (!out) return set_error(MRF_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return set_error(MRF_E_INVALID, "no such CUDA device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3))
        return set_error(MRF_E_INVALID, std::string("the library is compiled for sm_103a only; device is sm_") +
                                            std::to_string(prop.major) + std::to_string(prop.minor));
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    mrf_ctx *c = new mrf_ctx();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : free_b;
    // device words: the error flag, then the work counters of the profile
    e = cudaMalloc(&c->err_flag, 64);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(err flag)"); }
    c->dev_stats = (unsigned long long *)((char *)c->err_flag + 8);
    e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaFree(c->err_flag); delete c; return cuda_fail(e, "cudaStreamCreate"); }
    cudaMemset(c->err_flag, 0, 64);
    // keep stream-ordered scratch in the pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return MRF_OK;
}

extern "C" int mrf_serve_stop(mrf_ctx *ctx);

extern "C" void mrf_ctx_destroy(mrf_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->serve) mrf_serve_stop(ctx);
    cudaDeviceSynchronize();
    cudaFree(ctx->err_flag);
    cudaStreamDestroy(ctx->aux);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    delete ctx;
}

extern "C" int mrf_ctx_memory(const mrf_ctx *ctx, size_t *used_bytes, size_t *budget_bytes)
{
    if (!ctx) return set_error(MRF_E_INVALID, "ctx is NULL");
    if (used_bytes) *used_bytes = ctx->used.load();
    if (budget_bytes) *budget_bytes = ctx->budget;
    return MRF_OK;
}

extern "C" int mrf_stream_sync(mrf_ctx *ctx, void *stream)
{
    if (!ctx) return set_error(MRF_E_INVALID, "ctx is NULL");
    cudaSetDevice(ctx->device);
    return check_device_error(ctx, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// FP32 FMA rate: eight independent chains per thread, 64 warps per SM

namespace {
constexpr int kFmaIters = 8192;
constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) fma_rate_kernel(float *out, float a, float b)
{
    float x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = (float)(threadIdx.x + k) * 1.0e-3f;
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}
}  // namespace

extern "C" int mrf_fp32_fma_rate(mrf_ctx *ctx, double *tflops)
{
    if (!ctx || !tflops) return set_error(MRF_E_INVALID, "NULL argument");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int blocks = ctx->sm_count * 8, threads = 256;
    float *out = nullptr;
    e = cudaMalloc(&out, sizeof(float) * blocks * threads);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fma rate)");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0, ctx->aux);
        fma_rate_kernel<<<blocks, threads, 0, ctx->aux>>>(out, 0.9999999f, 1.0e-7f);
        cudaEventRecord(t1, ctx->aux);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms > 0.f &&
            (best == 0.f || ms < best))
            best = ms;   // the first launch only warms up
        count_launch(ctx);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "fma rate kernel");
    const double fmas = (double)blocks * threads * kFmaIters * kFmaChains;
    *tflops = best > 0.f ? 2.0 * fmas / (best * 1e-3) / 1e12 : 0.0;
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// kernel accounting

ProfScope::ProfScope(mrf_ctx *c, int k, cudaStream_t s) : ctx(c), kind(k), stream(s)
{
    ctx->kind_launches[kind].fetch_add(1);
    ctx->launches.fetch_add(1);
    if (ctx->profiling.load()) {
        if (cudaEventCreate(&start) == cudaSuccess) cudaEventRecord(start, stream);
        else start = nullptr;
    }
}

ProfScope::~ProfScope()
{
    if (!start) return;
    cudaEvent_t stop;
    if (cudaEventCreate(&stop) != cudaSuccess) { cudaEventDestroy(start); return; }
    cudaEventRecord(stop, stream);
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    ctx->prof_pending.push_back(ProfEvent{kind, start, stop});
}

extern "C" int mrf_profile_enable(mrf_ctx *ctx, int on)
{
    if (!ctx) return set_error(MRF_E_INVALID, "ctx is NULL");
    ctx->profiling.store(on != 0);
    return MRF_OK;
}

extern "C" int mrf_profile_read(mrf_ctx *ctx, mrf_profile *out, int reset)
{
    if (!ctx || !out) return set_error(MRF_E_INVALID, "NULL argument");
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    for (auto &ev : ctx->prof_pending) {
        cudaEventSynchronize(ev.stop);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.start, ev.stop) == cudaSuccess) {
            ctx->prof_ms[ev.kind] += ms;
            ctx->prof_timed[ev.kind] += 1;
        }
        cudaEventDestroy(ev.start);
        cudaEventDestroy(ev.stop);
    }
    ctx->prof_pending.clear();
    out->launches = ctx->launches.load();
    out->dictgen_launches = ctx->kind_launches[kProfDictGen].load();
    out->matcher_launches = ctx->kind_launches[kProfMatcher].load();
    out->zoom_launches = ctx->kind_launches[kProfZoom].load();
    out->dictgen_ms = ctx->prof_ms[kProfDictGen];
    out->matcher_ms = ctx->prof_ms[kProfMatcher];
    out->zoom_ms = ctx->prof_ms[kProfZoom];
    out->dictgen_timed = ctx->prof_timed[kProfDictGen];
    out->matcher_timed = ctx->prof_timed[kProfMatcher];
    out->zoom_timed = ctx->prof_timed[kProfZoom];
    out->zoomline_launches = ctx->kind_launches[kProfZoomLine].load();
    out->zoomline_ms = ctx->prof_ms[kProfZoomLine];
    out->zoomline_timed = ctx->prof_timed[kProfZoomLine];
    unsigned long long st[5] = {0, 0, 0, 0, 0};
    cudaDeviceSynchronize();
    if (cudaMemcpy(st, ctx->dev_stats, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess) {
        out->zoomline_pairs = st[0];
        out->zoomline_entries = st[1];
        out->zoom_rounds = st[2];
        out->zoom_candidates = st[3];
        out->zoom_max_voxel_rounds = st[4];
    }
    if (reset) {
        cudaMemset(ctx->dev_stats, 0, sizeof(st));
        ctx->launches = 0;
        for (int k = 0; k < kProfKinds; ++k) {
            ctx->kind_launches[k] = 0;
            ctx->prof_ms[k] = 0;
            ctx->prof_timed[k] = 0;
        }
    }
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// sequence

static bool is_fin(double v) { return isfinite(v) != 0; }

extern "C" int mrf_sequence_load(mrf_ctx *ctx, const mrf_sequence_desc *d, mrf_seq **out)
{
    if (!ctx || !d || !out) return set_error(MRF_E_INVALID, "NULL argument");
    *out = nullptr;
    const int n = d->n;
    if (n < 1 || !d->flip_rad || !d->tr_ms || !d->te_ms) return set_error(MRF_E_INVALID, "sequence: n < 1 or NULL array");
    if (d->inversion != 0 && d->inversion != 1) return set_error(MRF_E_INVALID, "sequence: inversion must be 0 or 1");
    if (!is_fin(d->inv_delay_ms) || d->inv_delay_ms < 0) return set_error(MRF_E_INVALID, "sequence: bad inversion delay");
    bool xonly = true, symmetric = true, finite = false;
    double min_tr = INFINITY;
    for (int j = 0; j < n; ++j) {
        double a = d->flip_rad[j], tr = d->tr_ms[j], te = d->te_ms[j];
        double ph = d->rf_phase_rad ? d->rf_phase_rad[j] : 0.0;
        double tp = d->pulse_ms ? d->pulse_ms[j] : 0.0;
        if (!is_fin(a) || !is_fin(tr) || !is_fin(te) || !is_fin(ph) || !is_fin(tp))
            return set_error(MRF_E_INVALID, "sequence: non-finite value at j=" + std::to_string(j));
        if (tp < 0) return set_error(MRF_E_INVALID, "sequence: negative pulse duration at j=" + std::to_string(j));
        if (tp > 0) finite = true;
        if (!(tr > 0) || te < 0 || te > tr)
            return set_error(MRF_E_INVALID, "sequence: need TR > 0 and 0 <= TE <= TR at j=" + std::to_string(j));
        if (fabs(sin(ph)) > 1e-12) xonly = false;
        if (fabs(te - (tr - te)) > 1e-12 * tr) symmetric = false;
        if (tr < min_tr) min_tr = tr;
    }
    if (finite) xonly = false;   // the effective field of a finite pulse is tilted out of the x-y plane
    std::vector<float4> rfx(n);
    std::vector<float> rfg(12 * (size_t)n, 0.f);
    std::vector<float2> tau(n);
    std::vector<float4> rff(n);
    for (int j = 0; j < n; ++j) {
        double a = d->flip_rad[j], ph = d->rf_phase_rad ? d->rf_phase_rad[j] : 0.0;
        // finite pulse (Appendix): rotation about (-alpha cos phi, -alpha sin phi, tau dw) by its length
        const double tp = d->pulse_ms ? d->pulse_ms[j] : 0.0;
        rff[j] = make_float4((float)(-a * cos(ph)), (float)(-a * sin(ph)), (float)(a * a), (float)(2.0 * M_PI * tp));
        // Hard pulse R_z(phi) R_x(-alpha) R_z(-phi) (Appendix). For phi = k pi it is
        // a rotation about x by beta = -alpha (k even) or +alpha (k odd).
        double beta = cos(ph) > 0 ? -a : a;
        double c = cos(beta), s = sin(beta), sh = sin(0.5 * beta);
        rfx[j] = make_float4((float)c, (float)s, (float)(2.0 * sh * sh), (float)d->te_ms[j]);
        // general matrix: rotation by -alpha about (cos phi, sin phi, 0) (Rodrigues)
        double kx = cos(ph), ky = sin(ph), th = -a;
        double ct = cos(th), st = sin(th), vt = 2.0 * sin(0.5 * th) * sin(0.5 * th);
        double R[9] = {ct + kx * kx * vt, kx * ky * vt, ky * st,
                       ky * kx * vt, ct + ky * ky * vt, -kx * st,
                       -ky * st, kx * st, ct};
        double omr22 = vt;   // 1 - R22 = 1 - cos(th)
        for (int q = 0; q < 9; ++q) rfg[12 * (size_t)j + q] = (float)R[q];
        rfg[12 * (size_t)j + 9] = (float)omr22;
        tau[j] = make_float2((float)d->te_ms[j], (float)(d->tr_ms[j] - d->te_ms[j]));
    }
    cudaSetDevice(ctx->device);
    mrf_seq *s = new mrf_seq();
    s->n = n; s->xonly = xonly; s->symmetric = symmetric; s->inversion = d->inversion;
    s->inv_delay = d->inv_delay_ms; s->min_tr = min_tr; s->finite = finite;
    // rfx | rfg | tau | rff in one block, 256-byte aligned pieces
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b1 = sizeof(float4) * n, b2 = sizeof(float) * 12 * (size_t)n, b3 = sizeof(float2) * n;
    const size_t b4 = sizeof(float4) * n;
    const size_t o2 = al(b1), o3 = o2 + al(b2), o4 = o3 + al(b3), total = o4 + al(b4);
    std::vector<uint8_t> h(total, 0);
    memcpy(h.data(), rfx.data(), b1);
    memcpy(h.data() + o2, rfg.data(), b2);
    memcpy(h.data() + o3, tau.data(), b3);
    memcpy(h.data() + o4, rff.data(), b4);
    int rc = upload_block(ctx, h.data(), total, &s->block, "sequence upload");
    if (rc) { delete s; return rc; }
    s->bytes = total;
    s->rfx = (float4 *)s->block;
    s->rfg = (float *)((uint8_t *)s->block + o2);
    s->tau = (float2 *)((uint8_t *)s->block + o3);
    s->rff = (float4 *)((uint8_t *)s->block + o4);
    *out = s;
    return MRF_OK;
}

void seq_release(mrf_ctx *ctx, mrf_seq *s, cudaStream_t stream, bool sync)
{
    if (!s) return;
    release_block(ctx, s->block, s->bytes, stream, sync);
    delete s;
}

int seq_clone(mrf_ctx *ctx, const mrf_seq *src, mrf_seq **out)
{
    mrf_seq *s = new mrf_seq(*src);
    s->block = nullptr;
    int rc = upload_block(ctx, nullptr, src->bytes, &s->block, "sequence copy");
    if (rc) { delete s; return rc; }
    cudaError_t e = cudaMemcpyAsync(s->block, src->block, src->bytes, cudaMemcpyDeviceToDevice, ctx->aux);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux);
    if (e != cudaSuccess) { seq_release(ctx, s, ctx->aux, false); return cuda_fail(e, "sequence copy"); }
    const ptrdiff_t d = (uint8_t *)s->block - (uint8_t *)src->block;
    s->rfx = (float4 *)((uint8_t *)src->rfx + d);
    s->rfg = (float *)((uint8_t *)src->rfg + d);
    s->tau = (float2 *)((uint8_t *)src->tau + d);
    s->rff = (float4 *)((uint8_t *)src->rff + d);
    *out = s;
    return MRF_OK;
}

extern "C" int mrf_sequence_free(mrf_ctx *ctx, mrf_seq *seq)
{
    if (!ctx || !seq) return set_error(MRF_E_INVALID, "NULL argument");
    cudaSetDevice(ctx->device);
    seq_release(ctx, seq, nullptr, true);
    return MRF_OK;
}

extern "C" int mrf_sequence_free_async(mrf_ctx *ctx, mrf_seq *seq, void *stream)
{
    if (!ctx || !seq) return set_error(MRF_E_INVALID, "NULL argument");
    cudaSetDevice(ctx->device);
    seq_release(ctx, seq, (cudaStream_t)stream, false);
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// grid

int grid_validate(const mrf_grid_desc *g)
{
    if (!g) return set_error(MRF_E_INVALID, "grid is NULL");
    if (g->n_t1 < 1 || g->n_t2 < 1 || g->n_df < 1) return set_error(MRF_E_INVALID, "grid: counts must be >= 1");
    if (!(g->t1_step > 0) || !(g->t2_step > 0) || !(g->df_step > 0))
        return set_error(MRF_E_INVALID, "grid: steps must be > 0");
    if (!is_fin(g->t1_min) || !is_fin(g->t2_min) || !is_fin(g->df_min) || !is_fin(g->t1_step) ||
        !is_fin(g->t2_step) || !is_fin(g->df_step))
        return set_error(MRF_E_INVALID, "grid: non-finite value");
    if (!(g->t1_min > 0) || !(g->t2_min > 0)) return set_error(MRF_E_INVALID, "grid: T1 and T2 must be > 0");
    if (g->require_t2_lt_t1 != 0 && g->require_t2_lt_t1 != 1)
        return set_error(MRF_E_INVALID, "grid: require_t2_lt_t1 must be 0 or 1");
    return MRF_OK;
}

static double t1v(const mrf_grid_desc *g, int a) { return g->t1_min + (double)a * g->t1_step; }
static double t2v(const mrf_grid_desc *g, int b) { return g->t2_min + (double)b * g->t2_step; }

static int32_t nb_valid(const mrf_grid_desc *g, int a)
{
    if (!g->require_t2_lt_t1) return g->n_t2;
    int32_t k = 0;
    for (int b = 0; b < g->n_t2; ++b) if (t2v(g, b) < t1v(g, a)) k = b + 1;
    return k;
}

extern "C" int64_t mrf_grid_count(const mrf_grid_desc *g)
{
    int rc = grid_validate(g);
    if (rc) return rc;
    int64_t total = 0;
    for (int a = 0; a < g->n_t1; ++a) total += (int64_t)nb_valid(g, a) * g->n_df;
    return total;
}

extern "C" int mrf_grid_unravel(const mrf_grid_desc *g, int64_t index, int32_t *a, int32_t *b, int32_t *c)
{
    int rc = grid_validate(g);
    if (rc) return rc;
    if (index < 0) return set_error(MRF_E_INVALID, "index < 0");
    int64_t off = 0;
    for (int aa = 0; aa < g->n_t1; ++aa) {
        int64_t cnt = (int64_t)nb_valid(g, aa) * g->n_df;
        if (index < off + cnt) {
            int64_t rem = index - off;
            if (a) *a = aa;
            if (b) *b = (int32_t)(rem / g->n_df);
            if (c) *c = (int32_t)(rem % g->n_df);
            return MRF_OK;
        }
        off += cnt;
    }
    return set_error(MRF_E_INVALID, "index beyond the grid");
}

// Host tables of a grid (axis values, T1-block offsets, valid-T2 counts) in
// one 256-byte aligned layout.
struct GridHost {
    std::vector<uint8_t> h;
    size_t o_t2, o_df, o_ao, o_nb, total;
    int64_t count;
    int a_full;
};

static void grid_tables(const mrf_grid_desc *g, GridHost &G)
{
    const size_t nt1 = g->n_t1, nt2 = g->n_t2, ndf = g->n_df;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    G.o_t2 = al(4 * nt1);
    G.o_df = G.o_t2 + al(4 * nt2);
    G.o_ao = G.o_df + al(4 * ndf);
    G.o_nb = G.o_ao + al(8 * (nt1 + 1));
    G.total = G.o_nb + al(4 * nt1);
    G.h.assign(G.total, 0);
    float *t1 = (float *)G.h.data(), *t2 = (float *)(G.h.data() + G.o_t2), *df = (float *)(G.h.data() + G.o_df);
    int64_t *ao = (int64_t *)(G.h.data() + G.o_ao);
    int32_t *nb = (int32_t *)(G.h.data() + G.o_nb);
    for (int a = 0; a < g->n_t1; ++a) t1[a] = (float)t1v(g, a);
    for (int b = 0; b < g->n_t2; ++b) t2[b] = (float)t2v(g, b);
    for (int c = 0; c < g->n_df; ++c) df[c] = (float)(g->df_min + (double)c * g->df_step);
    ao[0] = 0;
    for (int a = 0; a < g->n_t1; ++a) {
        nb[a] = nb_valid(g, a);
        ao[a + 1] = ao[a] + (int64_t)nb[a] * g->n_df;
    }
    G.count = ao[g->n_t1];
    G.a_full = g->n_t1;
    while (G.a_full > 0 && nb[G.a_full - 1] == g->n_t2) --G.a_full;
}

int grid_upload(mrf_ctx *ctx, const mrf_grid_desc *g, GridBuf *out)
{
    int rc = grid_validate(g);
    if (rc) return rc;
    GridHost G;
    grid_tables(g, G);
    GridBuf gb;
    gb.desc = *g;
    rc = upload_block(ctx, G.h.data(), G.total, &gb.block, "grid upload");
    if (rc) return rc;
    uint8_t *d = (uint8_t *)gb.block;
    gb.t1 = (float *)d;
    gb.t2 = (float *)(d + G.o_t2);
    gb.df = (float *)(d + G.o_df);
    gb.a_off = (int64_t *)(d + G.o_ao);
    gb.nb = (int32_t *)(d + G.o_nb);
    gb.count = G.count;
    gb.a_full = G.a_full;
    gb.bytes = G.total;
    *out = gb;
    return MRF_OK;
}

// The T1 rows [a0, a1) of grid g as a grid of their own: the same axis values
// (taken from g's tables, so validity and values match the whole grid bit for
// bit) and entry offsets counted from the range's first entry.
static int grid_upload_rows(mrf_ctx *ctx, const mrf_grid_desc *g, const GridHost &G, int a0, int a1, GridBuf *out)
{
    mrf_grid_desc sub = *g;
    sub.n_t1 = a1 - a0;
    sub.t1_min = t1v(g, a0);
    GridHost S;
    grid_tables(&sub, S);   // layout for the range; the contents are replaced below
    const float *t1 = (const float *)G.h.data();
    const int64_t *ao = (const int64_t *)(G.h.data() + G.o_ao);
    const int32_t *nb = (const int32_t *)(G.h.data() + G.o_nb);
    float *st1 = (float *)S.h.data();
    int64_t *sao = (int64_t *)(S.h.data() + S.o_ao);
    int32_t *snb = (int32_t *)(S.h.data() + S.o_nb);
    for (int a = a0; a < a1; ++a) {
        st1[a - a0] = t1[a];
        snb[a - a0] = nb[a];
        sao[a - a0] = ao[a] - ao[a0];
    }
    sao[a1 - a0] = ao[a1] - ao[a0];
    memcpy(S.h.data() + S.o_t2, G.h.data() + G.o_t2, 4 * (size_t)g->n_t2);
    memcpy(S.h.data() + S.o_df, G.h.data() + G.o_df, 4 * (size_t)g->n_df);
    S.count = ao[a1] - ao[a0];
    S.a_full = std::min(std::max(G.a_full - a0, 0), a1 - a0);
    GridBuf gb;
    gb.desc = sub;
    int rc = upload_block(ctx, S.h.data(), S.total, &gb.block, "grid upload");
    if (rc) return rc;
    uint8_t *d = (uint8_t *)gb.block;
    gb.t1 = (float *)d;
    gb.t2 = (float *)(d + S.o_t2);
    gb.df = (float *)(d + S.o_df);
    gb.a_off = (int64_t *)(d + S.o_ao);
    gb.nb = (int32_t *)(d + S.o_nb);
    gb.count = S.count;
    gb.a_full = S.a_full;
    gb.bytes = S.total;
    *out = gb;
    return MRF_OK;
}

int grid_upload_async(mrf_ctx *ctx, const mrf_grid_desc *g, cudaStream_t stream, GridDev *out, void **block,
                      size_t *bytes)
{
    (void)stream;   // uploaded on the library's own stream; the caller frees it in stream order
    int rc = grid_validate(g);
    if (rc) return rc;
    GridHost G;
    grid_tables(g, G);
    void *dv = nullptr;
    rc = upload_block(ctx, G.h.data(), G.total, &dv, "grid upload");
    if (rc) return rc;
    uint8_t *d = (uint8_t *)dv;
    out->n_t1 = g->n_t1; out->n_t2 = g->n_t2; out->n_df = g->n_df;
    out->t1 = (const float *)d;
    out->t2 = (const float *)(d + G.o_t2);
    out->df = (const float *)(d + G.o_df);
    out->a_off = (const int64_t *)(d + G.o_ao);
    out->nb = (const int32_t *)(d + G.o_nb);
    out->count = G.count;
    out->a_full = G.a_full;
    *block = d;
    *bytes = G.total;
    return MRF_OK;
}

void grid_release(mrf_ctx *ctx, GridBuf *g, cudaStream_t stream, bool sync)
{
    release_block(ctx, g->block, g->bytes, stream, sync);
    *g = GridBuf();
}

// ---------------------------------------------------------------------------
// simulation and dictionary

extern "C" int mrf_simulate(mrf_ctx *ctx, const mrf_seq *seq, int64_t count, const float *t1, const float *t2,
                            const float *df, void *out, void *stream)
{
    if (!ctx || !seq) return set_error(MRF_E_INVALID, "NULL argument");
    if (count < 0) return set_error(MRF_E_INVALID, "count < 0");
    if (count == 0) return MRF_OK;
    if (!t1 || !t2 || !df || !out) return set_error(MRF_E_INVALID, "NULL device array");
    cudaSetDevice(ctx->device);
    return launch_simulate(ctx, seq, count, t1, t2, df, out, (cudaStream_t)stream);
}

// Row length in elements: 2n rounded up to 128, plus 128 bytes so that rows do
// not sit on a power-of-two stride (which crowds them into few L2 sets).
// Row stride in elements: 2n rounded up to 128, plus padding that keeps rows
// off a power-of-two stride and every 1-byte plane's rows on 128-byte lines
// (FP8 rows; the e4m3 planes of MRF_F32): 128 elements, 64 for BF16.
static int dict_ld(int n, int dtype) { return ((2 * n + 127) / 128) * 128 + (dtype == MRF_BF16 ? 64 : 128); }

extern "C" int mrf_dict_free(mrf_ctx *ctx, mrf_dict *d)
{
    if (!ctx || !d) return set_error(MRF_E_INVALID, "NULL argument");
    cudaSetDevice(ctx->device);
    // work on any stream may still read the dictionary: wait for the device,
    // then hand the blocks back to the pool (no unmapping)
    if (d->block) release_block(ctx, d->block, d->block_bytes, nullptr, true);
    grid_release(ctx, &d->grid, ctx->aux, false);
    seq_release(ctx, d->seq, ctx->aux, false);
    delete d;
    return MRF_OK;
}

// Allocates d's rows (hi | lo | norm | scale in one block from the stream-
// ordered pool, so that generating and freeing dictionaries repeatedly maps no
// new memory) and queues their generation; d's sequence, grid, dtype, entries,
// n and ld are set. On failure the caller frees d.
static int dict_fill(mrf_ctx *ctx, mrf_dict *d, cudaStream_t stream)
{
    const size_t ebytes = d->dtype == MRF_FP8E4M3 ? 1 : 2;
    const size_t rows = (size_t)d->entries * d->ld * ebytes;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    const size_t b_lo = d->dtype == MRF_F32 ? al(rows) : 0, b_sc = al(4 * (size_t)d->entries);
    const size_t total = al(rows) + b_lo + al(4 * (size_t)d->entries) + b_sc;
    int rc = budget_charge(ctx, total);
    if (rc) return rc;
    cudaError_t e = cudaMallocAsync(&d->block, total, stream);
    if (e != cudaSuccess) {
        budget_release(ctx, total);
        d->block = nullptr;
        return cuda_fail(e, "dictionary");
    }
    d->block_bytes = total;
    uint8_t *blk = (uint8_t *)d->block;
    d->hi = blk;
    d->lo = d->dtype == MRF_F32 ? blk + al(rows) : nullptr;
    d->norm = (float *)(blk + al(rows) + b_lo);
    d->scale = (float *)(blk + al(rows) + b_lo + al(4 * (size_t)d->entries));
    d->bytes = total + d->grid.bytes + d->seq->bytes;
    return launch_dict_generate(ctx, d, stream);
}

extern "C" int mrf_dict_free_async(mrf_ctx *ctx, mrf_dict *d, void *stream_v)
{
    if (!ctx || !d) return set_error(MRF_E_INVALID, "NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_v;
    if (d->block) release_block(ctx, d->block, d->block_bytes, stream, false);
    grid_release(ctx, &d->grid, stream, false);
    seq_release(ctx, d->seq, stream, false);
    delete d;
    return MRF_OK;
}

extern "C" int mrf_dict_generate(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, mrf_dtype dtype,
                                 void *stream, mrf_dict **out)
{
    if (!ctx || !seq || !grid || !out) return set_error(MRF_E_INVALID, "NULL argument");
    *out = nullptr;
    if (dtype != MRF_F32 && dtype != MRF_BF16 && dtype != MRF_FP8E4M3)
        return set_error(MRF_E_INVALID, "unknown dtype");
    int64_t count = mrf_grid_count(grid);
    if (count < 0) return (int)count;
    if (count == 0) return set_error(MRF_E_INVALID, "grid has no valid entry");
    if (count > (int64_t)INT32_MAX) return set_error(MRF_E_UNSUPPORTED, "dictionaries above 2^31 entries");
    cudaSetDevice(ctx->device);
    mrf_dict *d = new mrf_dict();
    d->dtype = dtype;
    d->entries = count;
    d->n = seq->n;
    d->ld = dict_ld(seq->n, dtype);
    int rc = seq_clone(ctx, seq, &d->seq);
    if (rc) { delete d; return rc; }
    rc = grid_upload(ctx, grid, &d->grid);
    if (!rc) rc = dict_fill(ctx, d, (cudaStream_t)stream);
    if (rc) { mrf_dict_free(ctx, d); return rc; }
    *out = d;
    return MRF_OK;
}

extern "C" int mrf_dict_query(const mrf_dict *d, mrf_dict_info *info)
{
    if (!d || !info) return set_error(MRF_E_INVALID, "NULL argument");
    info->entries = d->entries;
    info->n = d->n;
    info->ld = d->ld;
    info->dtype = d->dtype;
    info->hi_dev = d->hi;
    info->lo_dev = d->lo;
    info->norm_dev = d->norm;
    info->scale_dev = d->scale;
    info->bytes = d->bytes;
    info->smooth_width = d->smooth_width;
    info->smooth_sigma = d->smooth_sigma;
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// matching and ZOOM

static bool valid_topk(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32; }

extern "C" int mrf_match_bruteforce(mrf_ctx *ctx, const mrf_dict *d, const void *fp, int64_t V,
                                    const mrf_match_opts *o, mrf_result *out, void *stream)
{
    if (!ctx || !d || !o) return set_error(MRF_E_INVALID, "NULL argument");
    if (V < 0) return set_error(MRF_E_INVALID, "V < 0");
    if (o->precision != d->dtype) return set_error(MRF_E_INVALID, "precision differs from the dictionary dtype");
    if (!valid_topk(o->top_k)) return set_error(MRF_E_INVALID, "top_k must be 1, 2, 4, 8, 16 or 32");
    if (o->rescore != 0 && o->rescore != 1) return set_error(MRF_E_INVALID, "rescore must be 0 or 1");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaSetDevice(ctx->device);
    return run_match(ctx, d, fp, V, o->precision, o->top_k, o->rescore, out, nullptr, nullptr,
                     (cudaStream_t)stream);
}

extern "C" int mrf_match_bruteforce_grid(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                                         const mrf_match_opts *o, int64_t chunk_entries, const void *fp, int64_t V,
                                         mrf_result *out, void *stream_v)
{
    if (!ctx || !seq || !grid || !o) return set_error(MRF_E_INVALID, "NULL argument");
    if (V < 0) return set_error(MRF_E_INVALID, "V < 0");
    if (o->precision != MRF_F32 && o->precision != MRF_BF16 && o->precision != MRF_FP8E4M3)
        return set_error(MRF_E_INVALID, "unknown precision");
    if (!valid_topk(o->top_k)) return set_error(MRF_E_INVALID, "top_k must be 1, 2, 4, 8, 16 or 32");
    if (o->rescore != 0 && o->rescore != 1) return set_error(MRF_E_INVALID, "rescore must be 0 or 1");
    if (chunk_entries < 0) return set_error(MRF_E_INVALID, "chunk_entries < 0");
    int rc = grid_validate(grid);
    if (rc) return rc;
    GridHost G;
    grid_tables(grid, G);
    if (G.count == 0) return set_error(MRF_E_INVALID, "grid has no valid entry");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    const int64_t cap = std::min<int64_t>(chunk_entries > 0 ? chunk_entries : (int64_t)1 << 23, INT32_MAX);
    const int32_t *nb = (const int32_t *)(G.h.data() + G.o_nb);
    const int64_t *ao = (const int64_t *)(G.h.data() + G.o_ao);
    for (int a = 0; a < grid->n_t1; ++a)
        if ((int64_t)nb[a] * grid->n_df > cap) return set_error(MRF_E_INVALID, "chunk_entries below a T1 row's entries");
    cudaSetDevice(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_v;
    // runner-up CC per voxel and one range's results, from the pool
    const size_t sb = (sizeof(float) * (size_t)V + 255) & ~(size_t)255;
    const size_t scratch = sb + sizeof(mrf_result) * (size_t)V;
    rc = budget_charge(ctx, scratch);
    if (rc) return rc;
    void *blk = nullptr;
    cudaError_t e = cudaMallocAsync(&blk, scratch, stream);
    if (e != cudaSuccess) { budget_release(ctx, scratch); return cuda_fail(e, "chunked match scratch"); }
    float *second = (float *)blk;
    mrf_result *part = (mrf_result *)((uint8_t *)blk + sb);
    bool first = true;
    for (int a0 = 0; a0 < grid->n_t1 && !rc;) {
        int a1 = a0;
        while (a1 < grid->n_t1 && ao[a1 + 1] - ao[a0] <= cap) ++a1;
        const int64_t cnt = ao[a1] - ao[a0];
        if (cnt > 0) {
            mrf_dict *d = new mrf_dict();
            d->seq = const_cast<mrf_seq *>(seq);   // borrowed: the range's dictionary dies in this call
            d->dtype = o->precision;
            d->entries = cnt;
            d->n = seq->n;
            d->ld = dict_ld(seq->n, o->precision);
            rc = grid_upload_rows(ctx, grid, G, a0, a1, &d->grid);
            if (!rc) rc = dict_fill(ctx, d, stream);
            if (!rc)
                rc = run_match(ctx, d, fp, V, o->precision, o->top_k, o->rescore, first ? out : part, nullptr,
                               nullptr, stream);
            if (!rc) rc = launch_chunk_merge(out, second, first ? nullptr : part, V, ao[a0], a0, stream);
            first = false;
            if (d->block) release_block(ctx, d->block, d->block_bytes, stream, false);
            grid_release(ctx, &d->grid, stream, false);
            delete d;
        }
        a0 = a1;
    }
    cudaFreeAsync(blk, stream);
    budget_release(ctx, scratch);
    return rc;
}

extern "C" int mrf_match_bruteforce_fused(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                                          const mrf_match_opts *o, const void *fp, int64_t V, mrf_result *out,
                                          void *stream_v)
{
    if (!ctx || !seq || !grid || !o) return set_error(MRF_E_INVALID, "NULL argument");
    if (V < 0) return set_error(MRF_E_INVALID, "V < 0");
    if (o->precision != MRF_F32 && o->precision != MRF_BF16)
        return set_error(MRF_E_INVALID, "fused brute force: precision must be MRF_F32 or MRF_BF16");
    if (!valid_topk(o->top_k)) return set_error(MRF_E_INVALID, "top_k must be 1, 2, 4, 8, 16 or 32");
    if (o->rescore != 0 && o->rescore != 1) return set_error(MRF_E_INVALID, "rescore must be 0 or 1");
    int rc = grid_validate(grid);
    if (rc) return rc;
    const int64_t D = mrf_grid_count(grid);
    if (D == 0) return set_error(MRF_E_INVALID, "grid has no valid entry");
    if (D > INT32_MAX) return set_error(MRF_E_INVALID, "fused brute force: more than 2^31 - 1 entries");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaSetDevice(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_v;
    // a dictionary with nothing stored: its entries are generated inside the matcher
    mrf_dict d;
    d.seq = const_cast<mrf_seq *>(seq);   // borrowed for the call
    d.dtype = o->precision;
    d.entries = D;
    d.n = seq->n;
    d.ld = dict_ld(seq->n, o->precision);
    rc = grid_upload(ctx, grid, &d.grid);
    if (rc) return rc;
    rc = run_match(ctx, &d, fp, V, o->precision, o->top_k, o->rescore, out, nullptr, nullptr, stream, true);
    grid_release(ctx, &d.grid, stream, false);
    return rc;
}

extern "C" int mrf_match_topk(mrf_ctx *ctx, const mrf_dict *d, const void *fp, int64_t V, int32_t precision,
                              int32_t top_k, int64_t *idx, float *cc2, void *stream)
{
    if (!ctx || !d) return set_error(MRF_E_INVALID, "NULL argument");
    if (V < 0) return set_error(MRF_E_INVALID, "V < 0");
    if (precision != d->dtype) return set_error(MRF_E_INVALID, "precision differs from the dictionary dtype");
    if (!valid_topk(top_k)) return set_error(MRF_E_INVALID, "top_k must be 1, 2, 4, 8, 16 or 32");
    if (V == 0) return MRF_OK;
    if (!fp || !idx || !cc2) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaSetDevice(ctx->device);
    return run_match(ctx, d, fp, V, precision, top_k, 0, nullptr, idx, cc2, (cudaStream_t)stream);
}

extern "C" void mrf_zoom_opts_default(mrf_zoom_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->omega_hz = 0.0;
    o->t1_init_ms = 1000.0;
    o->t2_init_ms = 100.0;
    o->s1a_step_frac = 6.0 / 7.0;
    o->s1b_half_frac = 1.0;
    o->s1b_step_frac = 1.0 / 20.0;
    o->s3_half_frac = 0.5;
    o->n_s2 = 2;
    o->s2_t1_ms[0] = 200.0; o->s2_t2_ms[0] = 200.0;
    o->s2_t1_ms[1] = 100.0; o->s2_t2_ms[1] = 100.0;
    const int p[8] = {0, 1, 0, 0, 0, 1, 1, 1};
    const double h[8] = {100.0, 100.0, 50.0, 20.0, 10.0, 50.0, 20.0, 10.0};
    o->n_s4 = 8;
    for (int i = 0; i < 8; ++i) { o->s4_param[i] = p[i]; o->s4_ms[i] = h[i]; }
    o->prior_chain = 0;
    o->prior_start = 1;
    o->prior_t1_ms = 3000.0;
    o->prior_t2_ms = 800.0;
    o->prior_df_hz = 150.0;
}

extern "C" int mrf_zoom_search(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                               const mrf_zoom_opts *opts, const void *fp, int64_t V, mrf_result *out,
                               void *stream)
{
    if (!ctx || !seq || !grid) return set_error(MRF_E_INVALID, "NULL argument");
    int rc = grid_validate(grid);
    if (rc) return rc;
    if (V < 0 || V > INT32_MAX) return set_error(MRF_E_INVALID, "zoom: V must be in [0, 2^31 - 1]");
    mrf_zoom_opts def;
    if (!opts) { mrf_zoom_opts_default(&def); opts = &def; }
    if (opts->n_s2 < 0 || opts->n_s2 > MRF_ZOOM_MAX_LEVELS || opts->n_s4 < 0 || opts->n_s4 > MRF_ZOOM_MAX_LEVELS)
        return set_error(MRF_E_INVALID, "zoom: level counts out of range");
    for (int i = 0; i < opts->n_s4; ++i)
        if (opts->s4_param[i] != 0 && opts->s4_param[i] != 1) return set_error(MRF_E_INVALID, "zoom: s4_param must be 0/1");
    if (!(opts->s1a_step_frac > 0) || !(opts->s1b_step_frac > 0) || opts->s1b_half_frac < 0 || opts->s3_half_frac < 0)
        return set_error(MRF_E_INVALID, "zoom: bad df search fractions");
    if (opts->prior_chain < 0 || (opts->prior_chain > 0 && opts->prior_start != 0 && opts->prior_start != 1) ||
        (opts->prior_chain > 0 && !(opts->prior_t1_ms >= 0 && opts->prior_t2_ms >= 0 && opts->prior_df_hz >= 0 &&
                                    std::isfinite(opts->prior_t1_ms) && std::isfinite(opts->prior_t2_ms) &&
                                    std::isfinite(opts->prior_df_hz))))
        return set_error(MRF_E_INVALID, "zoom: prior_chain >= 0; with a prior, prior_start 0 or 1 and finite "
                                        "non-negative half-widths");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaSetDevice(ctx->device);
    return run_zoom(ctx, seq, grid, opts, fp, V, out, (cudaStream_t)stream);
}
