// Windowed refinement of per-voxel grid points (Results, Experiment 2: a
// brute-force search in a small window around a ZOOM answer), repeated as a
// hill climb: the centre is compared with the 26 points of its 3 x 3 x 3
// neighbourhood (T1 offset outer, then T2, then df; -1 before +1) and moves
// to the best of them when that is strictly better (the first in that order
// on ties), until the centre wins. It starts from any method's answer -- the
// top-k re-score of a BF16/FP8 brute force, or ZOOM -- and uses the re-score's
// arithmetic: FP32 Bloch recurrence with accurate evolution factors, FP64
// accumulation of <x, d>, ||d||^2 and ||x||^2, FP64 CC.
//
// One warp per voxel: lanes 0..25 simulate the 26 neighbours of a round, lane
// 26 the starting centre in the first round. Points off the grid or with
// T2 >= T1 (when required) are not evaluated.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "bloch.cuh"
#include "mrf_internal.h"

namespace {

constexpr int kRefineThreads = 128;   // 4 voxels (warps) per CTA

__device__ __forceinline__ bool refine_valid(const GridDev &g, int a, int b, int c)
{
    return a >= 0 && a < g.n_t1 && b >= 0 && b < g.n_t2 && c >= 0 && c < g.n_df &&
           (a >= g.a_full || b < __ldg(&g.nb[a]));
}

// <x, d>, ||d||^2 of one point in FP64 (FP32 partial sums over 8 timepoints).
template <bool XONLY, bool SYM>
__device__ __forceinline__ void refine_point(const SeqDev &s, const float2 *__restrict__ x, float T1, float T2,
                                             float df, double &ipr, double &ipi, double &dd)
{
    const Relax r = relax_make(T1, T2, df);
    Bloch st;
    bloch_start(st, s, r);
    ipr = ipi = dd = 0.0;
    const int n = s.n;
    for (int j0 = 0; j0 < n; j0 += 8) {
        float pr = 0.f, pi = 0.f, pd = 0.f;
        const int j1 = min(n, j0 + 8);
        for (int j = j0; j < j1; ++j) {
            bloch_rf<XONLY>(st, s, j, r.f);
            const float2 tau = __ldg(&s.tau[j]);
            float e1, zr, zi;
            relax_factors(r, tau.x, e1, zr, zi);
            bloch_evolve(st, e1, zr, zi);
            const float sr = st.mx, si = st.my;
            if (SYM) {
                bloch_evolve(st, e1, zr, zi);
            } else {
                relax_factors(r, tau.y, e1, zr, zi);
                bloch_evolve(st, e1, zr, zi);
            }
            const float2 z = __ldg(&x[j]);
            // x conj(d) = (xr dr + xi di) + i (xi dr - xr di)
            pr = fmaf(z.x, sr, fmaf(z.y, si, pr));
            pi = fmaf(z.y, sr, fmaf(-z.x, si, pi));
            pd = fmaf(sr, sr, fmaf(si, si, pd));
        }
        ipr += (double)pr;
        ipi += (double)pi;
        dd += (double)pd;
    }
}

template <bool XONLY, bool SYM>
__global__ void __launch_bounds__(kRefineThreads) refine_kernel(SeqDev s, GridDev g, const float2 *x, int64_t V,
                                                                int max_moves, mrf_result *res, int *err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // neighbour of lane q < 26 in the canonical order; lane 26: the centre
    const int k = lane < 13 ? lane : lane + 1;
    const int oa = lane < 26 ? k / 9 - 1 : 0, ob = lane < 26 ? (k / 3) % 3 - 1 : 0, oc = lane < 26 ? k % 3 - 1 : 0;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); v < V; v += warps) {
        const mrf_result in = res[v];
        if (in.index < 0 || !refine_valid(g, in.i_t1, in.i_t2, in.i_df)) continue;   // no start point
        const int n = s.n;
        const float2 *xv = x + (size_t)v * n;
        double xx = 0.0;
        for (int j = lane; j < n; j += 32) {
            const float2 z = __ldg(&xv[j]);
            xx += (double)z.x * z.x + (double)z.y * z.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(FULL, xx, o);
        const double inv_xn = xx > 0.0 ? 1.0 / sqrt(xx) : 0.0;

        int a = in.i_t1, b = in.i_t2, c = in.i_df;
        double centre = -INFINITY, cr = 0.0, ci = 0.0, cd = 0.0;
        int evaluated = 0, moves = 0;
        double mm = INFINITY;
        bool first = true, ok = true;
        for (;;) {
            const int pa = a + oa, pb = b + ob, pc = c + oc;
            const bool want = lane < 26 || (first && lane == 26);
            const bool valid = want && refine_valid(g, pa, pb, pc);
            double ipr, ipi, dd;
            refine_point<XONLY, SYM>(s, xv, valid ? __ldg(&g.t1[pa]) : 1000.f, valid ? __ldg(&g.t2[pb]) : 100.f,
                                     valid ? __ldg(&g.df[pc]) : 0.f, ipr, ipi, dd);
            double val = -INFINITY;
            if (valid) val = (dd > 0.0 && inv_xn > 0.0) ? sqrt(ipr * ipr + ipi * ipi) * inv_xn / sqrt(dd) : 0.0;
            if (first) {
                // the starting centre (lane 26)
                centre = __shfl_sync(FULL, val, 26);
                cr = __shfl_sync(FULL, ipr, 26);
                ci = __shfl_sync(FULL, ipi, 26);
                cd = __shfl_sync(FULL, dd, 26);
                evaluated += 1;
                first = false;
            }
            if (++moves > max_moves) { ok = false; break; }
            // neighbours only (lanes < 26): count, top two with the centre, best (earliest on ties)
            const double nv = lane < 26 ? val : -INFINITY;
            evaluated += __popc(__ballot_sync(FULL, lane < 26 && valid));
            double bv = nv, t1 = nv, t2 = -INFINITY;
            int bl = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(FULL, bv, o);
                const int ol = __shfl_xor_sync(FULL, bl, o);
                if (ov > bv || (ov == bv && ol < bl)) { bv = ov; bl = ol; }
                const double o1 = __shfl_xor_sync(FULL, t1, o), o2 = __shfl_xor_sync(FULL, t2, o);
                const double hi = fmax(t1, o1), lo = fmin(t1, o1);
                t2 = fmax(lo, fmax(t2, o2));
                t1 = hi;
            }
            // the centre joins the decision set
            {
                const double hi = fmax(t1, centre), lo = fmin(t1, centre);
                t2 = fmax(lo, t2);
                t1 = hi;
            }
            if (isfinite(t2)) mm = fmin(mm, t1 - t2);
            const double wr = __shfl_sync(FULL, ipr, bl), wi = __shfl_sync(FULL, ipi, bl),
                         wd = __shfl_sync(FULL, dd, bl);
            if (!(bv > centre)) break;
            const int kk = bl < 13 ? bl : bl + 1;
            a += kk / 9 - 1;
            b += (kk / 3) % 3 - 1;
            c += kk % 3 - 1;
            centre = bv;
            cr = wr; ci = wi; cd = wd;
        }
        if (lane == 0) {
            if (!ok) atomicExch(err, kDeviceErrBounds);
            mrf_result r = in;
            r.index = g.a_off[a] + (int64_t)b * g.n_df + c;
            r.i_t1 = a; r.i_t2 = b; r.i_df = c;
            r.t1_ms = g.t1[a]; r.t2_ms = g.t2[b]; r.df_hz = g.df[c];
            r.cc = (float)centre;
            r.m0 = cd > 0.0 ? (float)(sqrt(cr * cr + ci * ci) / cd) : 0.f;
            r.phase = (float)atan2(ci, cr);
            r.entries_evaluated = (in.entries_evaluated > 0 ? in.entries_evaluated : 0) + evaluated;
            float m = isfinite(mm) ? (float)mm : -1.f;
            if (in.min_margin >= 0.f && (m < 0.f || in.min_margin < m)) m = in.min_margin;
            r.min_margin = m;
            res[v] = r;
        }
    }
}

}  // namespace

extern "C" int mrf_refine(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, const void *fp, int64_t V,
                          int32_t max_moves, mrf_result *res, void *stream_v)
{
    if (!ctx || !seq || !grid) return set_error(MRF_E_INVALID, "NULL argument");
    int rc = grid_validate(grid);
    if (rc) return rc;
    if (V < 0) return set_error(MRF_E_INVALID, "V < 0");
    if (max_moves < 1) return set_error(MRF_E_INVALID, "refine: max_moves must be >= 1");
    if (V == 0) return MRF_OK;
    if (!fp || !res) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t stream = (cudaStream_t)stream_v;
    GridDev gdev;
    void *gblock = nullptr;
    size_t gbytes = 0;
    rc = grid_upload_async(ctx, grid, stream, &gdev, &gblock, &gbytes);
    if (rc) return rc;
    const SeqDev s = seq->dev();
    const int64_t want = (V + kRefineThreads / 32 - 1) / (kRefineThreads / 32);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->sm_count * 16));
    count_launch(ctx);
    if (s.xonly && s.symmetric)
        refine_kernel<true, true><<<blocks, kRefineThreads, 0, stream>>>(s, gdev, (const float2 *)fp, V, max_moves, res, ctx->err_flag);
    else if (s.xonly)
        refine_kernel<true, false><<<blocks, kRefineThreads, 0, stream>>>(s, gdev, (const float2 *)fp, V, max_moves, res, ctx->err_flag);
    else if (s.symmetric)
        refine_kernel<false, true><<<blocks, kRefineThreads, 0, stream>>>(s, gdev, (const float2 *)fp, V, max_moves, res, ctx->err_flag);
    else
        refine_kernel<false, false><<<blocks, kRefineThreads, 0, stream>>>(s, gdev, (const float2 *)fp, V, max_moves, res, ctx->err_flag);
    e = cudaGetLastError();
    cudaFreeAsync(gblock, stream);
    budget_release(ctx, gbytes);
    if (e != cudaSuccess) return cuda_fail(e, "refine launch");
    return MRF_OK;
}
