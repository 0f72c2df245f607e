// Temporal smoothing (Methods, Experiment 4: 3- and 5-point moving Gaussian
// smoothing of the fingerprints and of the dictionary). A sample becomes the
// weighted mean of the samples within h = (width - 1) / 2 of it, weights
// exp(-k^2 / (2 sigma^2)) renormalised over the samples that exist at the
// ends of the timecourse; Re and Im alike.
//
// mrf_smooth: fingerprints, one thread per output sample.
// mrf_dict_smooth: a generated MRF_F32 or BF16 dictionary in place,
// one thread per entry re-simulating it from the dictionary's own sequence
// and grid (FP32 recurrence, accurate factors) twice: the norm of the
// smoothed entry, then the write in the dictionary's convention, rounded to
// storage once. The
// dictionary remembers the smoothing so that its top-k re-score smooths the
// re-simulated candidates alike.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "bloch.cuh"
#include "mrf_internal.h"
#include "split.cuh"

namespace {

struct SmoothW {
    int h;
    float w[3];   // w[k] = exp(-k^2 / (2 sigma^2)), k = 0..h
};

int make_weights(int width, double sigma, SmoothW &sw)
{
    if (width != 1 && width != 3 && width != 5) return set_error(MRF_E_INVALID, "smoothing width must be 1, 3 or 5");
    if (!(sigma > 0.0) || !isfinite(sigma)) return set_error(MRF_E_INVALID, "smoothing sigma must be > 0");
    sw.h = (width - 1) / 2;
    for (int k = 0; k < 3; ++k) sw.w[k] = k <= sw.h ? (float)exp(-(double)(k * k) / (2.0 * sigma * sigma)) : 0.f;
    return MRF_OK;
}

__global__ void smooth_kernel(const float2 *in, float2 *out, int64_t V, int n, SmoothW sw)
{
    const int64_t total = V * (int64_t)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / n;
        const int j = (int)(i - v * n);
        const float2 *row = in + v * n;
        float sr = 0.f, si = 0.f, ws = 0.f;
        for (int k = -sw.h; k <= sw.h; ++k) {
            const int t = j + k;
            if (t < 0 || t >= n) continue;
            const float w = sw.w[k < 0 ? -k : k];
            const float2 z = __ldg(&row[t]);
            sr = fmaf(w, z.x, sr);
            si = fmaf(w, z.y, si);
            ws += w;
        }
        out[i] = make_float2(sr / ws, si / ws);
    }
}

// Smoothed sample t from a window of raw samples win[k + 2] = s_{t+k}.
__device__ __forceinline__ float2 smoothed(const float2 (&win)[5], int t, int n, const SmoothW &sw)
{
    float sr = 0.f, si = 0.f, ws = 0.f;
#pragma unroll
    for (int k = -2; k <= 2; ++k) {
        if (k < -sw.h || k > sw.h || t + k < 0 || t + k >= n) continue;
        const float w = sw.w[k < 0 ? -k : k];
        sr = fmaf(w, win[k + 2].x, sr);
        si = fmaf(w, win[k + 2].y, si);
        ws += w;
    }
    return make_float2(sr / ws, si / ws);
}

// Raw samples of one entry, two ahead of the sample being smoothed: the
// window holds s_{t-2} .. s_{t+2} (zeros outside the timecourse).
template <bool XONLY>
struct RawStream {
    Bloch st;
    Relax r;
    int next;              // index of the next raw sample to simulate
    float2 win[5];
    __device__ __forceinline__ void start(const SeqDev &s, const Relax &rr)
    {
        r = rr;
        bloch_start(st, s, r);
        next = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) win[k] = make_float2(0.f, 0.f);
        for (int k = 0; k < 3; ++k) win[2 + k] = pull(s);
    }
    __device__ __forceinline__ float2 pull(const SeqDev &s)
    {
        if (next >= s.n) return make_float2(0.f, 0.f);
        float sr, si;
        bloch_step_otf<XONLY>(st, s, r, next, sr, si);
        ++next;
        return make_float2(sr, si);
    }
    __device__ __forceinline__ void advance(const SeqDev &s)
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) win[k] = win[k + 1];
        win[4] = pull(s);
    }
};

// Re-simulates each entry (the generator's FP32 recurrence with accurate
// factors), smooths it, and writes the normalised result with one rounding.
template <bool XONLY>
__global__ void dict_smooth_kernel(SeqDev s, GridDev g, uint8_t *hi, uint8_t *lo, float *norm, float *scale,
                                   int64_t D, int ld, SmoothW sw)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= D) return;
    int lo_a = 0, hi_a = g.n_t1 - 1;
    while (lo_a < hi_a) {
        const int mid = (lo_a + hi_a + 1) >> 1;
        if (__ldg(&g.a_off[mid]) <= e) lo_a = mid; else hi_a = mid - 1;
    }
    const int a = lo_a;
    const int64_t rem = e - __ldg(&g.a_off[a]);
    const int b = (int)(rem / g.n_df), c = (int)(rem % g.n_df);
    const Relax rr = relax_make(__ldg(&g.t1[a]), __ldg(&g.t2[b]), __ldg(&g.df[c]));
    const int n = s.n;
    // pass 1: squared norm of the smoothed entry (FP32 blocks of 32, FP64 total)
    RawStream<XONLY> rs;
    rs.start(s, rr);
    double ss = 0.0;
    float part = 0.f;
    for (int t = 0; t < n; ++t) {
        const float2 z = smoothed(rs.win, t, n, sw);
        part = fmaf(z.x, z.x, fmaf(z.y, z.y, part));
        if ((t & 31) == 31) { ss += part; part = 0.f; }
        rs.advance(s);
    }
    ss += part;
    const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.f;
    // pass 2: the smoothed entry, stored as the dictionary stores entries: the
    // raw signal with scale 1 / ||d|| (MRF_F32: fp16 row and the two e4m3
    // planes of the values and the residuals, lo present), or the unit-norm
    // signal with scale 1 (BF16)
    const float wmul = lo ? 1.f : inv;
    uint8_t *h = hi + (size_t)e * ld * 2;
    uint8_t *l8h = lo ? lo + (size_t)e * ld : nullptr;
    uint8_t *l8l = lo ? lo + (size_t)D * ld + (size_t)e * ld : nullptr;
    rs.start(s, rr);
    for (int t = 0; t < n; ++t) {
        const float2 z = smoothed(rs.win, t, n, sw);
        const float zr = z.x * wmul, zi = z.y * wmul;
        if (lo) {
            const SplitPair sp = split_pair(zr, zi, kSplitHiD);
            *reinterpret_cast<uint32_t *>(h + 4 * t) = sp.hi;
            *reinterpret_cast<uint16_t *>(l8h + 2 * t) = sp.h8;
            *reinterpret_cast<uint16_t *>(l8l + 2 * t) = sp.l8;
        } else {
            *reinterpret_cast<__nv_bfloat162 *>(h + 4 * t) = __floats2bfloat162_rn(zr, zi);
        }
        rs.advance(s);
    }
    norm[e] = (float)sqrt(ss);
    scale[e] = lo ? inv : 1.f;
}

}  // namespace

extern "C" int mrf_smooth(mrf_ctx *ctx, const void *in, void *out, int64_t V, int32_t n, int32_t width, double sigma,
                          void *stream)
{
    if (!ctx) return set_error(MRF_E_INVALID, "NULL argument");
    if (V < 0 || n < 1) return set_error(MRF_E_INVALID, "smooth: V < 0 or n < 1");
    SmoothW sw;
    int rc = make_weights(width, sigma, sw);
    if (rc) return rc;
    if (V == 0) return MRF_OK;
    if (!in || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    if (in == out) return set_error(MRF_E_INVALID, "smooth: input and output must be distinct buffers");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int64_t total = V * (int64_t)n;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->sm_count * 32);
    count_launch(ctx);
    smooth_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const float2 *)in, (float2 *)out, V, n, sw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "smooth launch");
    return MRF_OK;
}

extern "C" int mrf_dict_smooth(mrf_ctx *ctx, mrf_dict *d, int32_t width, double sigma, void *stream)
{
    if (!ctx || !d) return set_error(MRF_E_INVALID, "NULL argument");
    if (d->dtype == MRF_FP8E4M3) return set_error(MRF_E_UNSUPPORTED, "dictionary smoothing needs an MRF_F32 or MRF_BF16 dictionary");
    if (d->smooth_h != 0) return set_error(MRF_E_INVALID, "the dictionary is already smoothed");
    SmoothW sw;
    int rc = make_weights(width, sigma, sw);
    if (rc) return rc;
    if (sw.h == 0) return MRF_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const unsigned blocks = (unsigned)((d->entries + 127) / 128);
    const SeqDev s = d->seq->dev();
    const GridDev g = d->grid.dev();
    count_launch(ctx);
    if (s.xonly)
        dict_smooth_kernel<true><<<blocks, 128, 0, (cudaStream_t)stream>>>(
            s, g, (uint8_t *)d->hi, (uint8_t *)d->lo, d->norm, d->scale, d->entries, d->ld, sw);
    else
        dict_smooth_kernel<false><<<blocks, 128, 0, (cudaStream_t)stream>>>(
            s, g, (uint8_t *)d->hi, (uint8_t *)d->lo, d->norm, d->scale, d->entries, d->ld, sw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dictionary smoothing launch");
    d->smooth_h = sw.h;
    for (int k = 0; k < 3; ++k) d->smooth_w[k] = sw.w[k];
    d->smooth_width = width;
    d->smooth_sigma = sigma;
    return MRF_OK;
}
