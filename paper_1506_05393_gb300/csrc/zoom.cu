// MRF-ZOOM (Theory: df search steps 1-4, 1D ZOOM of Fig. 1, 2D ZOOM of
// Fig. 2; Methods, Experiment 2 steps 1-5).
//
// Two searches run the same canonical eager stage machine:
//  * on the fly (no dictionary): zoom_pack_kernel carries eight voxels per
//    warp and gives each lane one candidate per round, whose FP32 Bloch
//    recurrence accumulates <x, d> and ||d||^2 in 16-timepoint FP32 blocks
//    with compensated (Kahan) block sums. mrf_zoom_search splits it in three:
//    the packed kernel runs steps 1-2 and parks each voxel at step 3; the df
//    refinement of step 3 runs batched over the voxels that stopped at the
//    same (T1, T2) (zoom_line_kernel, same arithmetic per candidate and
//    voxel, so the same decisions); the packed kernel then resumes steps 4-5.
//    mrf_zoom_search_static runs all steps in the packed kernel, and so does
//    the spatial-neighbour prior (Methods, Experiment 3: each voxel searched
//    on the box of grid points around a neighbour's result), in two passes
//    of per-voxel boxes;
//  * zoom_dict_kernel reads candidates from a resident dictionary, one warp
//    per voxel, the warp streaming each stored row.
// Decisions take the best candidate with ties to the earliest in the
// canonical scan order, and move only when strictly better than the centre.
// The host turns physical step sizes into whole grid steps (round half up, at
// least 1, consecutive duplicates dropped) exactly as the stage machine
// defines them.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "bloch.cuh"
#include "mrf_internal.h"
#include "split.cuh"

namespace {

constexpr int kMaxLevels = MRF_ZOOM_MAX_LEVELS;
constexpr int kZoomThreads = 256;   // dictionary search: 8 voxels (warps) per CTA
constexpr int kScanW = 2;           // dictionary df scans: positions per lane per round

struct ZoomPlan {
    int a0, b0;          // start of the df search
    int a_raw, b_raw;    // the nearest grid indices of the start before clipping (per-voxel boxes clip them)
    int hA;              // step 1a: coarse df step
    int K1b, hB;         // step 1b: k = -K1b..K1b (k != 0), step hB
    int hC;              // step 1c: probe spacing (omega)
    int W3;              // step 3: half-width at the finest step
    int n_s2;
    int s2_h1[kMaxLevels], s2_h2[kMaxLevels];
    int n_s4;
    int s4_p[kMaxLevels], s4_h[kMaxLevels];
};

// A voxel's search state between the phases of the split on-the-fly search
// (the stages up to the 2D ZOOM, the df refinement of step 3 batched over the
// voxels that share its (T1, T2), then the rest).
struct ZState {
    int a, b, c, evaluated;
    float centre, mm, inv_xn;
    int flags;
};
constexpr int kZOk = 1;      // no level exceeded the move limit
constexpr int kZDone = 2;    // the search ended before step 3; its result is written

// Packed-kernel phases: the whole search, or the stages before step 3 (state
// saved there), or the stages after it (state restored).
enum ZPhase : int { kPhaseAll = 0, kPhaseHead = 1, kPhaseTail = 2 };

struct ZoomArgs {
    SeqDev s;
    GridDev g;
    // factor mode 3 (resident dictionary): the stored rows, bf16 (MRF_BF16)
    // or fp16 with the e4m3 residual plane (MRF_F32: dlo8 non-null)
    const uint8_t *dhi, *dlo8;
    const float *dnorm;      // L2 norm of each un-normalised entry
    const float *dscale;     // per-entry scale: stored row x scale = unit-norm entry
    int ld;                  // row stride in elements
    ZoomPlan plan;
    const float2 *x;
    int64_t V;
    mrf_result *out;
    int *counter;
    int *err;
    int max_moves;
    ZState *state;           // split search only
    int phase;               // ZPhase
    // spatial-neighbour prior: chains of chain_len consecutive voxels (0: off),
    // each voxel after a chain's first searched on the box of +-prior_h steps
    // around its predecessor's result, from that result when prior_start
    int chain_len;
    int prior_h1, prior_h2, prior_h3;
    int prior_start;
    int max_slots;           // slots per warp that take new work (1..kSlots): few chains spread over warps
    unsigned long long *stats;   // work counters: [2] warp rounds, [3] candidates simulated, [4] most rounds of a voxel
};

struct Kahan {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// e^{i 2 pi f tau} on the SFU, argument first reduced to [-1/2, 1/2] cycles.
__device__ __forceinline__ void cis_fast(float f, float tau, float &cs, float &sn) { cis_sfu(f, tau, cs, sn); }

// Start state of a candidate: equilibrium, or inverted and relaxed over the
// inversion delay (transverse magnetisation is zero after an ideal inversion).
__device__ __forceinline__ void start_state(Bloch &st, const SeqDev &s, float k1)
{
    bloch_init(st);
    if (s.inversion) {
        bloch_invert(st);
        st.w *= ex2_fast(k1 * s.inv_delay);
    }
}

struct Acc {   // x conj(d) and ||d||^2 in 16-timepoint FP32 blocks, Kahan-summed
    Kahan kr, ki, kd;
    float pr, pi, pd;
    __device__ __forceinline__ void init() { kr.init(); ki.init(); kd.init(); pr = pi = pd = 0.f; }
    __device__ __forceinline__ void add(float2 z, float sr, float si)
    {
        pr = fmaf(z.x, sr, fmaf(z.y, si, pr));
        pi = fmaf(z.y, sr, fmaf(-z.x, si, pi));
        pd = fmaf(sr, sr, fmaf(si, si, pd));
    }
    __device__ __forceinline__ void flush() { kr.add(pr); ki.add(pi); kd.add(pd); pr = pi = pd = 0.f; }
};

struct Eval {
    float v;                  // CC, -inf if the point is not evaluated
    float ipr, ipi, dd;
};

// One timepoint of C candidates (own factors each) sharing the timepoint's RF
// coefficients. SYM: TE_j equals TR_j - TE_j, so both free evolutions of the
// step share one set of factors (a compile-time choice: the second set is
// never computed).
template <bool XONLY, bool SYM, int C>
__device__ __forceinline__ void step_multi(const SeqDev &s, int j, const float (&k1)[C], const float (&k2)[C],
                                           const float (&f)[C], Bloch (&st)[C], Acc (&acc)[C],
                                           const float2 *const (&x)[C])
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    float q[10];
    float ta, tb = 0.f;
    const bool fin = !XONLY && s.finite;   // finite pulses: each candidate's rotation depends on its df
    if (XONLY) {
        r = __ldg(&s.rfx[j]);
        ta = r.w;
    } else if (fin) {
        r = __ldg(&s.rff[j]);
        ta = __ldg(&s.tau[j]).x;
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(s.rfg + 12 * j);
        const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
        q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
        q[8] = c.x; q[9] = c.y;
        ta = __ldg(&s.tau[j]).x;
    }
    if (!SYM) tb = __ldg(&s.tau[j]).y;
#pragma unroll
    for (int u = 0; u < C; ++u) {
        if (XONLY) bloch_rf_x(st[u], r);
        else if (fin) bloch_rf_finite(st[u], r, f[u]);
        else bloch_rf_general(st[u], q);
        float cs, sn;
        const float e1 = ex2_fast(k1[u] * ta), e2 = ex2_fast(k2[u] * ta);
        cis_fast(f[u], ta, cs, sn);
        bloch_evolve(st[u], e1, e2 * cs, e2 * sn);
        acc[u].add(__ldg(&x[u][j]), st[u].mx, st[u].my);
        if (SYM) {
            bloch_evolve(st[u], e1, e2 * cs, e2 * sn);
        } else {
            const float e1b = ex2_fast(k1[u] * tb), e2b = ex2_fast(k2[u] * tb);
            cis_fast(f[u], tb, cs, sn);
            bloch_evolve(st[u], e1b, e2b * cs, e2b * sn);
        }
    }
}

// Simulate C candidates per lane, each against its own voxel x[u], and take
// their CC: <x, d> and ||d||^2 accumulate in 16-timepoint FP32 blocks with
// compensated (Kahan) block sums. Every candidate's arithmetic is the same
// whichever of the C places it occupies, so a point has one value wherever
// it is simulated.
template <bool XONLY, bool SYM, int C>
__device__ __forceinline__ void sim_multi(const SeqDev &s, const float2 *const (&x)[C], const float (&T1)[C],
                                          const float (&T2)[C], const float (&df)[C], const float (&ixn)[C],
                                          const bool (&ok)[C], Eval (&out)[C])
{
    float k1[C], k2[C], f[C];
    Bloch st[C];
    Acc acc[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
        k1[u] = -1.4426950408889634f / T1[u];
        k2[u] = -1.4426950408889634f / T2[u];
        f[u] = df[u] * 1.0e-3f;
        start_state(st[u], s, k1[u]);
        acc[u].init();
    }
    const int n = s.n;
    int j0 = 0;
    for (; j0 + 16 <= n; j0 += 16) {
        // each voxel's samples four blocks ahead into L1 (lanes read different
        // voxels, whose rows need not stay in L2 while all are in flight)
#pragma unroll
        for (int u = 0; u < C; ++u) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(x[u] + min(j0 + 64, n - 1)));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(x[u] + min(j0 + 79, n - 1)));
        }
#pragma unroll 4
        for (int jj = 0; jj < 16; ++jj) step_multi<XONLY, SYM, C>(s, j0 + jj, k1, k2, f, st, acc, x);
#pragma unroll
        for (int u = 0; u < C; ++u) acc[u].flush();
    }
    for (int j = j0; j < n; ++j) step_multi<XONLY, SYM, C>(s, j, k1, k2, f, st, acc, x);
#pragma unroll
    for (int u = 0; u < C; ++u) {
        acc[u].flush();
        Eval &e = out[u];
        e.ipr = acc[u].kr.s;
        e.ipi = acc[u].ki.s;
        e.dd = acc[u].kd.s;
        if (ok[u]) {
            const float mag = sqrtf(fmaf(e.ipr, e.ipr, e.ipi * e.ipi));
            e.v = (e.dd > 0.f && ixn[u] > 0.f) ? mag * ixn[u] * rsqrtf(e.dd) : 0.f;
        } else {
            e.v = -INFINITY;
        }
    }
}

__device__ __forceinline__ bool point_valid(const GridDev &g, int a, int b, int c)
{
    // T1 indices from a_full on admit every T2 index: no table read there
    return a >= 0 && a < g.n_t1 && b >= 0 && b < g.n_t2 && c >= 0 && c < g.n_df &&
           (a >= g.a_full || b < __ldg(&g.nb[a]));
}

// Per-voxel search state shared (identically) by all lanes of the warp.
struct Search {
    int a, b, c;
    float centre;             // CC of the centre
    float cr, ci, cd;         // <x, d> and ||d||^2 of the centre
    int evaluated;
    float min_margin;
    float inv_xn;
};

// Factor mode 3: CC read from a resident dictionary. The lanes' candidates
// are evaluated one after another by the whole warp: 32 lanes stream the
// stored row (16-byte loads of 8 bf16) against x and reduce by shuffles.
__device__ __forceinline__ Eval eval_dict(const ZoomArgs &A, const float2 *x, float inv_xn, bool ok, int a, int b, int c)
{
    const int lane = threadIdx.x & 31;
    const int n2 = 2 * A.s.n;
    const float *xf = reinterpret_cast<const float *>(x);
    const long long e = ok ? (long long)(__ldg(&A.g.a_off[a]) + (int64_t)b * A.g.n_df + c) : -1;
    Eval mine;
    mine.v = -INFINITY;
    mine.ipr = mine.ipi = mine.dd = 0.f;
    unsigned todo = __ballot_sync(0xffffffffu, ok);
    while (todo) {
        const int q = __ffs(todo) - 1;
        todo &= todo - 1;
        const long long eq = __shfl_sync(0xffffffffu, e, q);
        const uint8_t *hi = A.dhi + (size_t)eq * A.ld * 2;
        const uint8_t *lo = A.dlo8 ? A.dlo8 + (size_t)eq * A.ld : nullptr;
        float re = 0.f, im = 0.f;
#pragma unroll 4
        for (int base = lane * 8; base < n2; base += 256) {
            float d[8];
            const uint4 h = __ldg(reinterpret_cast<const uint4 *>(hi + 2 * (size_t)base));
            if (lo) {
                // value = fp16 part 2^-15 + e4m3 residual 2^-19
                const __half2 *h2 = reinterpret_cast<const __half2 *>(&h);
                const uint2 l = __ldg(reinterpret_cast<const uint2 *>(lo + base));
                const uint16_t *l2 = reinterpret_cast<const uint16_t *>(&l);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __half22float2(h2[k]);
                    const float2 r = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(l2[k], __NV_E4M3)));
                    d[2 * k] = fmaf(r.x, kSplitDecLo, f.x * kSplitDecHi);
                    d[2 * k + 1] = fmaf(r.y, kSplitDecLo, f.y * kSplitDecHi);
                }
            } else {
                const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&h);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __bfloat1622float2(h2[k]);
                    d[2 * k] = f.x;
                    d[2 * k + 1] = f.y;
                }
            }
            if (base + 8 <= n2) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 z = __ldg(reinterpret_cast<const float2 *>(xf + base) + k);
                    // x conj(d)
                    re = fmaf(z.x, d[2 * k], fmaf(z.y, d[2 * k + 1], re));
                    im = fmaf(z.y, d[2 * k], fmaf(-z.x, d[2 * k + 1], im));
                }
            } else {
                for (int k = 0; 2 * k + base < n2; ++k) {
                    const float2 z = __ldg(reinterpret_cast<const float2 *>(xf + base) + k);
                    re = fmaf(z.x, d[2 * k], fmaf(z.y, d[2 * k + 1], re));
                    im = fmaf(z.y, d[2 * k], fmaf(-z.x, d[2 * k + 1], im));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == q) {
            // the stored row times its scale is the unit-norm entry d_hat; <x, d>
            // of the un-normalised entry is the norm times <x, d_hat>
            const float sc = __ldg(&A.dscale[eq]);
            const float hr = re * sc, hi_ = im * sc;
            const float nrm = __ldg(&A.dnorm[eq]);
            mine.ipr = hr * nrm;
            mine.ipi = hi_ * nrm;
            mine.dd = nrm * nrm;
            mine.v = sqrtf(fmaf(hr, hr, hi_ * hi_)) * inv_xn;
        }
    }
    return mine;
}

// Warp argmax: highest value, ties to the smallest position. Returns the lane
// holding it (valid when the value is finite).
__device__ __forceinline__ int warp_best(float v, int pos, float &best)
{
    float bv = v;
    int bp = pos, bl = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (ov > bv || (ov == bv && op < bp)) { bv = ov; bp = op; bl = ol; }
    }
    best = bv;
    return bl;
}

__device__ __forceinline__ void close_margin(Search &S, float t1, float t2)
{
    if (isfinite(t2)) S.min_margin = fminf(S.min_margin, t1 - t2);
}

// Adopt lane `bl`'s evaluation as the new centre.
__device__ __forceinline__ void take(Search &S, const Eval &e, int bl, int na, int nb, int nc, float bv)
{
    S.a = __shfl_sync(0xffffffffu, na, bl);
    S.b = __shfl_sync(0xffffffffu, nb, bl);
    S.c = __shfl_sync(0xffffffffu, nc, bl);
    S.cr = __shfl_sync(0xffffffffu, e.ipr, bl);
    S.ci = __shfl_sync(0xffffffffu, e.ipi, bl);
    S.cd = __shfl_sync(0xffffffffu, e.dd, bl);
    S.centre = bv;
}

// Two largest finite values of a per-lane pair (a >= b) across the warp,
// merged into a running pair.
__device__ __forceinline__ void warp_top2_pair(float a, float b, float &t1, float &t2)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oa = __shfl_xor_sync(0xffffffffu, a, o);
        const float ob = __shfl_xor_sync(0xffffffffu, b, o);
        const float hi = fmaxf(a, oa), lo = fminf(a, oa);
        b = fmaxf(lo, fmaxf(b, ob));
        a = hi;
    }
    const float hi = fmaxf(t1, a), lo = fminf(t1, a);
    t2 = fmaxf(lo, fmaxf(t2, b));
    t1 = hi;
}

// One scan over an ordered candidate list along df at fixed (a, b): list
// position p maps to c = c_start + p * step; `skip` is excluded; positions
// whose c falls off the grid are dropped before batching. Each lane
// simulates four positions per round. The running best (value S.centre at
// S.c) is replaced only by a strictly better value, earliest position first.
__device__ void df_scan(const ZoomArgs &A, const float2 *x, Search &S, int count, int c_start, int step, int skip,
                        bool with_centre)
{
    float t1 = with_centre ? S.centre : -INFINITY, t2 = -INFINITY;
    const int lane = threadIdx.x & 31;
    // positions with 0 <= c < n_df
    int p_lo = c_start >= 0 ? 0 : (-c_start + step - 1) / step;
    int p_hi = min(count - 1, (A.g.n_df - 1 - c_start) >= 0 ? (A.g.n_df - 1 - c_start) / step : -1);
    const bool ab_ok = point_valid(A.g, S.a, S.b, 0);
    for (int base = p_lo; base <= p_hi; base += 32 * kScanW) {
        bool ok[kScanW];
        int pos[kScanW], cc[kScanW];
#pragma unroll
        for (int u = 0; u < kScanW; ++u) {
            pos[u] = base + 32 * u + lane;
            cc[u] = c_start + pos[u] * step;
            ok[u] = ab_ok && pos[u] <= p_hi && cc[u] != skip;
        }
        Eval e[kScanW];
#pragma unroll
        for (int u = 0; u < kScanW; ++u) e[u] = eval_dict(A, x, S.inv_xn, ok[u], S.a, S.b, cc[u]);
        // lane-local best (earliest position on ties) and top two
        int bu = 0;
        float la = -INFINITY, lb = -INFINITY;
#pragma unroll
        for (int u = 0; u < kScanW; ++u) {
            S.evaluated += __popc(__ballot_sync(0xffffffffu, ok[u]));
            const float v = e[u].v;
            if (v > e[bu].v) bu = u;
            if (isfinite(v)) { if (v > la) { lb = la; la = v; } else if (v > lb) lb = v; }
        }
        warp_top2_pair(la, lb, t1, t2);
        Eval best = e[0];
        int bpos = pos[0], bc = cc[0];
#pragma unroll
        for (int u = 1; u < kScanW; ++u)
            if (u == bu) { best = e[u]; bpos = pos[u]; bc = cc[u]; }
        float bv;
        const int bl = warp_best(best.v, bpos, bv);
        if (bv > S.centre) take(S, best, bl, S.a, S.b, bc, bv);
    }
    close_margin(S, t1, t2);
}

// Speculative batches. A round evaluates more points than the next canonical
// decision needs (a whole line of 1D points, a 5x5 block of 2D points); the
// canonical eager decisions are then replayed on those values, lane by lane
// through shuffles, until a decision needs a point outside the batch. The
// replay takes exactly the decisions, margins and evaluation counts of the
// one-move-per-round search: values are deterministic, so a point evaluated
// speculatively has the value the canonical search would compute.

// Points of a 2D speculative batch, in units of (h1, h2) relative to the
// batch origin, for lane l. Without a predicted direction: the 5x5 block
// minus its centre (24 points, 2 moves). With direction (da, db): the 3x3
// neighbourhoods of the origin and of the next positions origin + m (da, db)
// along it -- 8 points, then 3 new ones per straight step or 5 per diagonal
// step (9 or 5 moves in one round). Returns false for an unused lane.
__device__ __forceinline__ bool batch2d_point(int l, int da, int db, int &oa, int &ob)
{
    if (da == 0 && db == 0) {
        if (l >= 24) return false;
        const int k = l < 12 ? l : l + 1;
        oa = k / 5 - 2;
        ob = k % 5 - 2;
        return true;
    }
    if (l < 8) {                              // neighbourhood of the origin
        const int k = l < 4 ? l : l + 1;
        oa = k / 3 - 1;
        ob = k % 3 - 1;
        return true;
    }
    const int r = l - 8;
    if (da == 0 || db == 0) {                 // straight: 3 new points per step
        const int m = 1 + r / 3, j = r % 3 - 1;
        if (da != 0) { oa = (m + 1) * da; ob = j; }
        else { oa = j; ob = (m + 1) * db; }
        return true;                          // m <= 8
    }
    if (r >= 20) return false;                // diagonal: 5 new points per step
    const int m = 1 + r / 5, q = r % 5;
    // around p_m = m (da, db): the far row (u = da, w = -1..1) and the far
    // column (w = db, u = -da, 0)
    int u, w;
    if (q < 3) { u = da; w = q - 1; }
    else { u = q == 3 ? -da : 0; w = db; }
    oa = m * da + u;
    ob = m * db + w;
    return true;
}

// 2D ZOOM at (h1, h2): each round evaluates a speculative batch around the
// current centre (see batch2d_point); the replay visits the 8 neighbours in
// the fixed order (T1 offset outer, -1 before +1), finds each one's lane
// with a warp ballot, and stops the round when a neighbour is missing.
__device__ bool move2d(const ZoomArgs &A, const float2 *x, Search &S, int h1, int h2)
{
    const int lane = threadIdx.x & 31;
    int moves = 0, pda = 0, pdb = 0;          // previous move direction
    for (;;) {
        const int ba = S.a, bb = S.b;         // batch origin (the centre)
        const float bc = S.centre;            // its value (known)
        const float bcr = S.cr, bci = S.ci, bcd = S.cd;
        int oa = 0, ob = 0;
        const bool have = batch2d_point(lane, pda, pdb, oa, ob);
        const int na = ba + oa * h1, nb = bb + ob * h2;
        const Eval e = eval_dict(A, x, S.inv_xn, have && point_valid(A.g, na, nb, S.c), na, nb, S.c);
        int ma = 0, mb = 0;                   // replay position in batch units
        for (;;) {
            if (++moves > A.max_moves) return false;
            float vals[8];
            int srcs[8];
            bool missing = false;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = q < 4 ? q : q + 1;
                const int pa = ma + k / 3 - 1, pb = mb + k % 3 - 1;
                if (pa == 0 && pb == 0) {
                    vals[q] = bc;
                    srcs[q] = -1;
                } else {
                    const unsigned hit = __ballot_sync(0xffffffffu, have && oa == pa && ob == pb);
                    missing |= hit == 0u;
                    srcs[q] = hit ? __ffs(hit) - 1 : 0;
                    vals[q] = __shfl_sync(0xffffffffu, e.v, srcs[q]);
                }
            }
            if (missing) { --moves; break; }  // the next decision needs a new batch
            float best = -INFINITY, t1 = S.centre, t2 = -INFINITY;
            int bq = -1, cnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float v = vals[q];
                if (isfinite(v)) {
                    ++cnt;
                    if (v > t1) { t2 = t1; t1 = v; } else if (v > t2) t2 = v;
                }
                if (v > best) { best = v; bq = q; }
            }
            S.evaluated += cnt;
            close_margin(S, t1, t2);
            if (!(best > S.centre)) return true;      // the centre wins: this level is done
            const int k = bq < 4 ? bq : bq + 1;
            pda = k / 3 - 1;
            pdb = k % 3 - 1;
            ma += pda;
            mb += pdb;
            if (srcs[bq] >= 0) {
                take(S, e, srcs[bq], na, nb, S.c, best);
            } else {                                  // back to the batch origin (values only rise, so unused)
                S.a = ba; S.b = bb; S.centre = best; S.cr = bcr; S.ci = bci; S.cd = bcd;
            }
        }
        // re-plan from the current centre (S.a, S.b were updated by take)
    }
}

// 1D ZOOM along T1 (param 0) or T2 (param 1) at half-width h: each round
// evaluates the points at -16h..16h; the replay compares left then right.
__device__ bool move1d(const ZoomArgs &A, const float2 *x, Search &S, int param, int h)
{
    const int lane = threadIdx.x & 31;
    const int off = lane < 16 ? lane - 16 : lane - 15;      // -16..-1, 1..16
    int moves = 0;
    for (;;) {
        const int ba = S.a, bb = S.b;
        const float bc = S.centre;
        const float bcr = S.cr, bci = S.ci, bcd = S.cd;
        const int na = ba + (param == 0 ? off * h : 0), nb = bb + (param == 1 ? off * h : 0);
        const Eval e = eval_dict(A, x, S.inv_xn, point_valid(A.g, na, nb, S.c), na, nb, S.c);
        int m = 0;
        for (;;) {
            if (m <= -16 || m >= 16) break;
            if (++moves > A.max_moves) return false;
            float vals[2];
            int srcs[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int p = m + (q == 0 ? -1 : 1);
                if (p == 0) { vals[q] = bc; srcs[q] = -1; }
                else {
                    srcs[q] = p < 0 ? p + 16 : p + 15;
                    vals[q] = __shfl_sync(0xffffffffu, e.v, srcs[q]);
                }
            }
            float t1 = S.centre, t2 = -INFINITY;
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float v = vals[q];
                if (isfinite(v)) {
                    ++cnt;
                    if (v > t1) { t2 = t1; t1 = v; } else if (v > t2) t2 = v;
                }
            }
            S.evaluated += cnt;
            close_margin(S, t1, t2);
            const int pick = vals[1] > vals[0] ? 1 : 0;
            const float best = vals[pick];
            if (!(best > S.centre)) return true;
            m += pick == 0 ? -1 : 1;
            if (srcs[pick] >= 0) take(S, e, srcs[pick], na, nb, S.c, best);
            else { S.a = ba; S.b = bb; S.centre = best; S.cr = bcr; S.ci = bci; S.cd = bcd; }
        }
        S.a = ba + (param == 0 ? m * h : 0);
        S.b = bb + (param == 1 ? m * h : 0);
    }
}

__global__ void __launch_bounds__(kZoomThreads) zoom_dict_kernel(ZoomArgs A)
{
    const int lane = threadIdx.x & 31;
    const ZoomPlan &P = A.plan;
    for (;;) {
        int v = 0;
        if (lane == 0) v = atomicAdd(A.counter, 1);
        v = __shfl_sync(0xffffffffu, v, 0);
        if (v >= A.V) break;
        const int n = A.s.n;
        const float2 *x = A.x + (size_t)v * n;
        float xx = 0.f;
        for (int j = lane; j < n; j += 32) {
            const float2 z = __ldg(&x[j]);
            xx = fmaf(z.x, z.x, fmaf(z.y, z.y, xx));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);

        Search S;
        S.a = P.a0; S.b = P.b0; S.c = 0;
        S.centre = -INFINITY;
        S.cr = S.ci = 0.f; S.cd = 0.f;
        S.evaluated = 0;
        S.min_margin = INFINITY;
        S.inv_xn = xx > 0.f ? rsqrtf(xx) : 0.f;
        bool ok = true;

        // step 1a: coarse scan of the whole df range (no prior centre)
        const int nA = (A.g.n_df + P.hA - 1) / P.hA;
        df_scan(A, x, S, nA, 0, P.hA, -1, false);
        // step 1b: window around the optimum
        {
            const int c0 = S.c;
            const int count = 2 * P.K1b + 1;
            df_scan(A, x, S, count, c0 - P.K1b * P.hB, P.hB, c0, true);
        }
        // step 1c: probes at whole multiples of omega
        {
            const int c0 = S.c;
            const int start = c0 - (c0 / P.hC) * P.hC;
            const int count = (A.g.n_df - 1 - start) / P.hC + 1;
            df_scan(A, x, S, count, start, P.hC, c0, true);
        }
        // step 2: 2D ZOOM at the coarse levels
        for (int l = 0; l < P.n_s2 && ok; ++l) ok = move2d(A, x, S, P.s2_h1[l], P.s2_h2[l]);
        // step 3: finest-step df window
        {
            const int c0 = S.c;
            df_scan(A, x, S, 2 * P.W3 + 1, c0 - P.W3, 1, c0, true);
        }
        // step 4: interleaved 1D ZOOMs
        for (int l = 0; l < P.n_s4 && ok; ++l) ok = move1d(A, x, S, P.s4_p[l], P.s4_h[l]);
        // step 5: final 2D ZOOM at the finest step
        if (ok) ok = move2d(A, x, S, 1, 1);
        if (!ok && lane == 0) atomicExch(A.err, kDeviceErrBounds);

        if (lane == 0) {
            mrf_result r;
            const bool have = isfinite(S.centre);
            r.index = have ? A.g.a_off[S.a] + (int64_t)S.b * A.g.n_df + S.c : -1;
            r.i_t1 = S.a; r.i_t2 = S.b; r.i_df = S.c;
            r.t1_ms = A.g.t1[S.a]; r.t2_ms = A.g.t2[S.b]; r.df_hz = A.g.df[S.c];
            r.cc = have ? S.centre : 0.f;
            r.m0 = S.cd > 0.f ? sqrtf(S.cr * S.cr + S.ci * S.ci) / S.cd : 0.f;
            r.phase = atan2f(S.ci, S.cr);
            r.entries_evaluated = S.evaluated;
            r.min_margin = isfinite(S.min_margin) ? S.min_margin : -1.f;
            A.out[v] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// On-the-fly search, packed: a warp carries kSlots voxels and hands out up to
// 2 x 32 candidates afresh every round.
//
// A voxel's next decision lacks only a few values: the unknown points among
// the eight neighbours of a 2D move (3 or 5 after a move), the unknown end of
// a 1D line, or any number of positions of a df scan. Each round lane s <
// kSlots runs the stage machine of slot s as far as the known values allow
// and lists the points its next decision lacks, then points that later
// decisions will want if the walk goes on. Lane 0 fills the round's table:
// first every slot's missing points, then consecutive positions for the
// slots that scan df, then the speculative points. Each lane simulates one
// or two table entries (two when more than 32 are listed) with its own
// (T1, T2, df) and voxel. The values of a move level stay in a per-slot
// window (8 x 8 points of the level's lattice, or 64 points of a 1D line) so
// that no point is simulated twice while it is in reach; the evaluation count
// still counts every visit of the canonical search. The final centre is
// simulated once more for its <x, d> and ||d||^2 (M0, phase).

constexpr int kSlots = 4;
constexpr int kPackWarps = 4;
constexpr int kPackThreads = 32 * kPackWarps;
constexpr int kPerLane = 1;                  // table entries a lane can simulate in one round
constexpr int kTable = 32 * kPerLane;
// every slot's missing decision points (at most 8: a 2D neighbourhood) fit in one round's table
static_assert(kSlots * 8 <= kTable, "round table smaller than the slots' missing points");
constexpr int kWin = 64;
constexpr int kReqMax = 24;                  // listed points per slot and round (8 missing + speculative)
constexpr int kSpecCentres = 5;              // 2D walks: future centres whose neighbourhoods are speculated
// A slot's window holds 8 x 8 lattice points, indexed by (i mod 8, k mod 8): collision free within
// any 8-step span per axis. The current neighbourhood and those of the speculated centres span
// kSpecCentres + 3 steps along a walk; past 8, a speculated point would evict a point the next
// decision needs, which would then be listed again every round.
static_assert(kSpecCentres + 3 <= 8, "speculated neighbourhoods must fit one window span");
// No search comes near this many rounds per voxel (the longest take a few hundred); a slot past it
// is not making progress, and the warp ends with an error instead of looping.
constexpr int kMaxSlotRounds = 1 << 16;
constexpr int kRunPrio = 3;                  // straight 2D run length whose speculation goes first

enum Stage : int { kS1a = 0, kS1b, kS1c, kS2, kS3, kS4, kS5, kFinal, kStop };
enum Tag : int { kTagNone = 0, kTagScan, kTagMove, kTagFinal };

struct Slot {
    int v;                 // voxel, -1 when idle
    int stage, level;
    int a, b, c;           // centre
    float centre;          // its CC (-inf before the first df scan)
    int evaluated;
    float mm;              // smallest decision margin so far
    float inv_xn;
    int ok;                // 0 once a level exceeded the move limit
    int rounds;            // rounds the voxel has been in flight (work counter)
    // df scans: list positions p..p_end, grid point c = start + p * step, `skip` excluded
    int p, p_end, start, step, skip;
    int scan_first, scan_n;  // this round's df positions in the table
    float g1, g2;          // running top two of the scan's decision set
    // move levels: moves so far, lattice origin (la, lb) and steps, the
    // centre's lattice coordinates, the last move (lattice units)
    int moves, la, lb, h1, h2, line, param, ia, ib, da, db;
    int run;               // consecutive moves in the direction (da, db)
    int alo, ahi, blo, bhi, clo, chi;   // the voxel's search box (the whole grid unless a prior bounds it)
    int chain_next, chain_end;          // prior chains: the chain's voxels still to search
    int pa, pb, pc;                     // prior chains: the result of the voxel searched last
    // listed points: ra/rb/rw[0..nreq) missing, then nspec speculative (rw: window index)
    int nreq, nspec;
    int ra[kReqMax], rb[kReqMax], rw[kReqMax];
};

struct PackShared {
    Slot s[kSlots];
    int wa[kSlots][kWin], wb[kSlots][kWin];
    float wv[kSlots][kWin];
    // this round's table and results
    int t_slot[kTable], t_a[kTable], t_b[kTable], t_c[kTable], t_tag[kTable];
    float r_v[kTable], r_ipr[kTable], r_ipi[kTable], r_dd[kTable];
    int used;
    int norm_mask;         // slots whose new voxel still needs ||x||
    int drained;
    int rot;
};

__device__ __forceinline__ bool is_scan(int st) { return st == kS1a || st == kS1b || st == kS1c || st == kS3; }

__device__ __forceinline__ void top2_add(float v, float &t1, float &t2)
{
    if (!isfinite(v)) return;
    if (v > t1) { t2 = t1; t1 = v; } else if (v > t2) t2 = v;
}

// List of a df scan at the current (a, b); positions whose c falls off the
// grid are dropped, and a list holding only the excluded point is empty.
__device__ __forceinline__ bool scan_setup(Slot &S, int count, int start, int step, int skip, bool with_centre)
{
    S.start = start;
    S.step = step;
    S.skip = skip;
    S.p = start >= S.clo ? 0 : (S.clo - start + step - 1) / step;
    S.p_end = min(count - 1, (S.chi - start) >= 0 ? (S.chi - start) / step : -1);
    S.g1 = with_centre ? S.centre : -INFINITY;
    S.g2 = -INFINITY;
    if (S.p == S.p_end && start + S.p * step == skip) return false;
    return S.p <= S.p_end;
}

// Window slot of lattice point (i, k): a torus of 8 x 8 for 2D levels (every
// 7 x 7 block is collision free), 64 along a 1D line.
__device__ __forceinline__ bool win_get(const PackShared &W, int s, int idx, int a, int b, float &v)
{
    if (W.wa[s][idx] != a || W.wb[s][idx] != b) return false;
    v = W.wv[s][idx];
    return true;
}

// Enter `stage` (with S.level for the leveled stages), passing over empty
// scans and exhausted level lists. A move level starts an empty window that
// holds the centre. With `stop3`, reaching step 3 parks the slot (kStop).
__device__ void enter(PackShared &W, int s, int stage, const ZoomPlan &P, int n_df, bool stop3)
{
    Slot &S = W.s[s];
    for (;;) {
        S.stage = stage;
        if (stop3 && stage == kS3) { S.stage = kStop; return; }
        bool nonempty;
        switch (stage) {
        case kS1a: {
            const int n = S.chi - S.clo + 1;
            nonempty = scan_setup(S, (n + P.hA - 1) / P.hA, S.clo, P.hA, -1, false);
            break;
        }
        case kS1b:
            nonempty = scan_setup(S, 2 * P.K1b + 1, S.c - P.K1b * P.hB, P.hB, S.c, true);
            break;
        case kS1c: {
            const int r = S.c - S.clo;
            const int st = S.clo + (r - (r / P.hC) * P.hC);
            nonempty = scan_setup(S, (S.chi - st) / P.hC + 1, st, P.hC, S.c, true);
            break;
        }
        case kS3:
            nonempty = scan_setup(S, 2 * P.W3 + 1, S.c - P.W3, 1, S.c, true);
            break;
        case kS2: case kS4: case kS5:
            if (stage == kS2 && S.level >= P.n_s2) { stage = kS3; continue; }
            if (stage == kS4 && S.level >= P.n_s4) { stage = kS5; continue; }
            S.moves = 0;
            S.line = stage == kS4;
            S.param = stage == kS4 ? P.s4_p[S.level] : 0;
            S.h1 = stage == kS2 ? P.s2_h1[S.level] : stage == kS4 ? P.s4_h[S.level] : 1;
            S.h2 = stage == kS2 ? P.s2_h2[S.level] : stage == kS4 ? P.s4_h[S.level] : 1;
            S.la = S.a;
            S.lb = S.b;
            S.ia = S.ib = S.da = S.db = 0;
            S.run = 0;
            for (int i = 0; i < kWin; ++i) W.wa[s][i] = -1;
            W.wa[s][0] = S.a;
            W.wb[s][0] = S.b;
            W.wv[s][0] = S.centre;
            return;
        default:
            return;
        }
        if (nonempty) return;
        // an empty scan: its decision set is the centre alone (no margin)
        stage = stage == kS1a ? kS1b : stage == kS1b ? kS1c : stage == kS1c ? kS2 : kS4;
        S.level = 0;
    }
}

// A move level's lattice (fixed between level entries), held in registers
// while a slot's decisions run.
struct Lattice {
    int la, lb, h1, h2, c, line, param;
    int alo, ahi, blo, bhi;
};

__device__ __forceinline__ Lattice lattice_of(const Slot &S)
{
    Lattice L;
    L.la = S.la; L.lb = S.lb; L.h1 = S.h1; L.h2 = S.h2; L.c = S.c; L.line = S.line; L.param = S.param;
    L.alo = S.alo; L.ahi = S.ahi; L.blo = S.blo; L.bhi = S.bhi;
    return L;
}

// Points that later decisions of a blocked move level will want if the walk
// goes on, listed by the whole warp, one candidate point per lane, nearest
// first: the points the 3 x 3 neighbourhoods of the next kSpecCentres centres
// along the last move add to the current one (3 per step on a straight walk,
// 5 per diagonal step; before the first move the 16 points at distance 2), or
// the next eight points of a 1D line in the direction of travel (both sides
// before the first move). The long walks of the final 2D ZOOM run straight
// for tens of moves, so a round can settle up to kSpecCentres + 1 moves. These
// points span at most 8 lattice steps along each axis (9 on a line), which the
// window holds without collisions, so every decision a round's results allow
// finds its values. Speculative points fill only lanes that required points
// leave idle (assign). Returns the points listed after the first `nreq`.
__device__ int speculate_warp(PackShared &W, int s, int lane, const GridDev &g, const Lattice &L, int ia, int ib,
                              int da, int db, int nreq, unsigned long long listed)
{
    const unsigned FULL = 0xffffffffu;
    int i = 0, k = 0;
    bool have = false;
    if (L.line) {
        const int d = L.param == 0 ? da : db;
        if (lane < 8) {
            const int t = lane + 2;
            const int m = d != 0 ? d * t : ((t & 1) ? -(t / 2 + 1) : (t / 2 + 1));
            i = ia + (L.param == 0 ? m : 0);
            k = ib + (L.param == 1 ? m : 0);
            have = true;
        }
    } else if (da == 0 && db == 0) {
        if (lane < 16) {   // the ring at distance 2, T1 offset outer, -2 before +2
            int r = lane, ii = 0, kk = 0;
            if (r < 5) { ii = -2; kk = r - 2; }
            else if (r < 11) { r -= 5; ii = -1 + r / 2; kk = (r & 1) ? 2 : -2; }
            else { ii = 2; kk = r - 13; }
            i = ia + ii;
            k = ib + kk;
            have = true;
        }
    } else if (da == 0 || db == 0) {
        if (lane < 3 * kSpecCentres) {   // straight: the three points ahead of centre t
            const int t = 2 + lane / 3, u = lane % 3 - 1;
            i = ia + (da != 0 ? t * da : u);
            k = ib + (db != 0 ? t * db : u);
            have = true;
        }
    } else {
        if (lane < 5 * kSpecCentres) {   // diagonal: the far row and column around centre t
            const int t = 1 + lane / 5, q = lane % 5;
            int u, w;
            if (q < 3) { u = da; w = q - 1; }
            else { u = q == 3 ? -da : 0; w = db; }
            i = ia + t * da + u;
            k = ib + t * db + w;
            have = true;
        }
    }
    int a = 0, b = 0, idx = 0;
    bool want = false;
    if (have) {
        a = L.la + i * L.h1;
        b = L.lb + k * L.h2;
        if (a >= L.alo && a <= L.ahi && b >= L.blo && b <= L.bhi && point_valid(g, a, b, L.c)) {
            idx = L.line ? ((L.param == 0 ? i : k) & (kWin - 1)) : (((i & 7) << 3) | (k & 7));
            float v;
            want = !win_get(W, s, idx, a, b, v) && !((listed >> idx) & 1ull);
        }
    }
    const unsigned m = __ballot_sync(FULL, want);
    const int pos = nreq + __popc(m & ((1u << lane) - 1u));
    if (want && pos < kReqMax) {
        Slot &S = W.s[s];
        S.ra[pos] = a;
        S.rb[pos] = b;
        S.rw[pos] = idx;
    }
    return min(__popc(m), kReqMax - nreq);
}

// Run slot s's decisions as far as the known values allow, by the whole warp:
// the stage machine runs uniformly on every lane (the slot's state in shared
// memory, written by lane 0), each decision's points are looked up one per
// lane, and the missing and speculative points are listed in parallel. On
// return the slot is scanning (positions are handed out elastically), waits
// for its S.nreq listed points, or is idle. Decisions, margins and evaluation
// counts are those of the canonical search: every comparison keeps its order.
__device__ void advance_warp(PackShared &W, int s, int lane, const ZoomPlan &P, const GridDev &g, int max_moves,
                             ZState *state)
{
    const unsigned FULL = 0xffffffffu;
    Slot &S = W.s[s];
    if (lane == 0) { S.nreq = 0; S.nspec = 0; }
    __syncwarp();
    const bool stop3 = state != nullptr;
    for (;;) {
        const int st = S.stage;
        if (S.v < 0) return;
        if (st == kStop) {
            // the stages before step 3 are done: save the search and free the slot
            if (lane == 0) {
                ZState z;
                z.a = S.a; z.b = S.b; z.c = S.c; z.evaluated = S.evaluated;
                z.centre = S.centre; z.mm = S.mm; z.inv_xn = S.inv_xn;
                z.flags = (S.ok ? kZOk : 0) | (S.rounds << 8);
                state[S.v] = z;
                S.v = -1;
            }
            __syncwarp();
            return;
        }
        if (is_scan(st)) {
            if (S.p <= S.p_end) return;
            if (lane == 0) {
                if (isfinite(S.g2)) S.mm = fminf(S.mm, S.g1 - S.g2);
                S.level = 0;
                enter(W, s, st == kS1a ? kS1b : st == kS1b ? kS1c : st == kS1c ? kS2 : kS4, P, g.n_df, stop3);
            }
            __syncwarp();
            continue;
        }
        if (st == kFinal) {
            if (lane == 0) {
                S.ra[0] = S.a;
                S.rb[0] = S.b;
                S.rw[0] = 0;
                S.nreq = 1;
            }
            __syncwarp();
            return;
        }
        // the points of the next decision, in the canonical order (lane q: point q): a
        // 1D line compares left then right, a 2D move the 8 neighbours with the T1 offset
        // outer and -1 before +1
        const Lattice L = lattice_of(S);
        const int ia = S.ia, ib = S.ib;
        const int npts = L.line ? 2 : 8;
        int di = 0, dk = 0;
        if (L.line) {
            const int m = lane == 0 ? -1 : 1;
            di = L.param == 0 ? m : 0;
            dk = L.param == 1 ? m : 0;
        } else {
            const int k = lane < 4 ? lane : lane + 1;
            di = k / 3 - 1;
            dk = k % 3 - 1;
        }
        float v = -INFINITY;
        bool known = true;
        int a = 0, b = 0, idx = 0;
        if (lane < npts) {
            a = L.la + (ia + di) * L.h1;
            b = L.lb + (ib + dk) * L.h2;
            if (a >= L.alo && a <= L.ahi && b >= L.blo && b <= L.bhi && point_valid(g, a, b, L.c)) {
                idx = L.line ? ((L.param == 0 ? ia + di : ib + dk) & (kWin - 1))
                             : ((((ia + di) & 7) << 3) | ((ib + dk) & 7));
                known = win_get(W, s, idx, a, b, v);
            }
        }
        const unsigned miss = __ballot_sync(FULL, lane < npts && !known);
        if (miss) {
            // list the missing points in the decision's order, then the speculative ones
            const int pos = __popc(miss & ((1u << lane) - 1u));
            if (lane < npts && !known) {
                S.ra[pos] = a;
                S.rb[pos] = b;
                S.rw[pos] = idx;
            }
            const int nreq = __popc(miss);
            const unsigned lo = (lane < npts && !known && idx < 32) ? 1u << idx : 0u;
            const unsigned hi = (lane < npts && !known && idx >= 32) ? 1u << (idx - 32) : 0u;
            const unsigned long long listed =
                ((unsigned long long)__reduce_or_sync(FULL, hi) << 32) | __reduce_or_sync(FULL, lo);
            __syncwarp();
            const int nspec = speculate_warp(W, s, lane, g, L, ia, ib, S.da, S.db, nreq, listed);
            __syncwarp();
            if (lane == 0) { S.nreq = nreq; S.nspec = nspec; }
            __syncwarp();
            return;
        }
        // every value known: the decision, on every lane alike
        float vals[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) vals[q] = __shfl_sync(FULL, v, q);
        const bool over = S.moves + 1 > max_moves;
        float t1 = S.centre, t2 = -INFINITY, best = -INFINITY;
        int bq = 0, cnt = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= npts) continue;
            const float vq = vals[q];
            if (isfinite(vq)) { cnt += 1; top2_add(vq, t1, t2); }
            if (vq > best) { best = vq; bq = q; }
        }
        const int bdi = __shfl_sync(FULL, di, bq), bdk = __shfl_sync(FULL, dk, bq);
        const bool moved = best > S.centre;
        __syncwarp();
        if (lane == 0) {
            S.moves += 1;
            if (over) {
                S.ok = 0;
                S.stage = kFinal;
            } else {
                S.evaluated += cnt;
                if (isfinite(t2)) S.mm = fminf(S.mm, t1 - t2);
                if (moved) {
                    S.run = (bdi == S.da && bdk == S.db) ? S.run + 1 : 1;
                    S.ia = ia + bdi;
                    S.ib = ib + bdk;
                    S.da = bdi;
                    S.db = bdk;
                    S.a = L.la + (ia + bdi) * L.h1;
                    S.b = L.lb + (ib + bdk) * L.h2;
                    S.centre = best;
                } else if (st == kS5) {
                    S.stage = kFinal;
                } else {
                    S.level += 1;
                    enter(W, s, st, P, g.n_df, stop3);
                }
            }
        }
        __syncwarp();
    }
}

// Lane 0, rounds with a df scan: consecutive positions for the scanning slots
// from table entry `used` on, shared out elastically over the free entries;
// returns the next free entry.
__device__ int assign_scans(PackShared &W, int used)
{
    const int rot = W.rot;
    int left[kSlots], give[kSlots];
    int active = 0;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const Slot &S = W.s[s];
        left[s] = (S.v >= 0 && is_scan(S.stage)) ? max(0, S.p_end - S.p + 1) : 0;
        give[s] = 0;
        active += left[s] > 0;
    }
    int free_lanes = kTable - used;
    while (free_lanes > 0 && active > 0) {
        const int share = max(1, free_lanes / active);
        active = 0;
        for (int i = 0; i < kSlots && free_lanes > 0; ++i) {
            const int s = (rot + i) % kSlots;
            if (left[s] <= 0) continue;
            const int gv = min(share, min(left[s], free_lanes));
            give[s] += gv;
            left[s] -= gv;
            free_lanes -= gv;
            active += left[s] > 0;
        }
    }
    for (int s = 0; s < kSlots; ++s) {
        Slot &S = W.s[s];
        S.scan_first = used;
        S.scan_n = give[s];
        for (int k = 0; k < give[s]; ++k, ++used) {
            const int c = S.start + (S.p + k) * S.step;
            W.t_slot[used] = s;
            W.t_a[used] = c == S.skip ? -1 : S.a;    // the excluded point is not simulated
            W.t_b[used] = S.b;
            W.t_c[used] = c;
            W.t_tag[used] = kTagScan;
        }
    }
    return used;
}

// The round's table, built by the whole warp: every slot's missing points
// first (rotating slot order), then consecutive df positions for the scanning
// slots, then the speculative points one slot at a time (pass r takes the r-th
// point of each slot that has one, in rotating order), cut at kTable -- first
// for the slots on a straight 2D walk (kRunPrio moves or more in one
// direction, the long final walks that set the search's duration), then for
// the others. Each slot lane computes where its own points go in that order.
// Speculation decides nothing, so the order changes no result.
__device__ void assign(PackShared &W, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int rot = W.rot;
    int nreq = 0, nsp = 0, scanning = 0, tag = kTagMove, ord = kSlots, prio = 0;
    if (lane < kSlots) {
        Slot &S = W.s[lane];
        ord = (lane - rot + kSlots) % kSlots;
        S.scan_n = 0;
        if (S.v >= 0) {
            nreq = S.nreq;
            tag = S.stage == kFinal ? kTagFinal : kTagMove;
            if (is_scan(S.stage)) scanning = S.p <= S.p_end;
            else if (S.stage != kFinal) {
                nsp = S.nspec;
                prio = !S.line && S.run >= kRunPrio;
            }
        }
    }
    int base = 0, nreq_total = 0, nsp_total = 0, nsp_prio = 0;
    int nsp_all[kSlots], ord_all[kSlots], prio_all[kSlots];
#pragma unroll
    for (int t = 0; t < kSlots; ++t) {
        const int nr = __shfl_sync(FULL, nreq, t);
        ord_all[t] = __shfl_sync(FULL, ord, t);
        nsp_all[t] = __shfl_sync(FULL, nsp, t);
        prio_all[t] = __shfl_sync(FULL, prio, t);
        nreq_total += nr;
        nsp_total += nsp_all[t];
        nsp_prio += prio_all[t] ? nsp_all[t] : 0;
        if (ord_all[t] < ord) base += nr;
    }
    if (lane < kSlots) {
        const Slot &S = W.s[lane];
        for (int r = 0; r < nreq; ++r) {
            const int u = base + r;   // at most 8 points per slot: never past kTable
            W.t_slot[u] = lane; W.t_a[u] = S.ra[r]; W.t_b[u] = S.rb[r]; W.t_c[u] = S.c;
            W.t_tag[u] = tag | (S.rw[r] << 8);
        }
    }
    int used = nreq_total;
    if (__any_sync(FULL, scanning)) {
        __syncwarp();
        if (lane == 0) used = assign_scans(W, used);
        used = __shfl_sync(FULL, used, 0);
    }
    if (lane < kSlots && nsp > 0) {
        const Slot &S = W.s[lane];
        const int gbase = used + (prio ? 0 : nsp_prio);
        for (int r = 0; r < nsp; ++r) {
            int u = gbase;
#pragma unroll
            for (int t = 0; t < kSlots; ++t)
                if (prio_all[t] == prio) u += min(r, nsp_all[t]) + ((ord_all[t] < ord && nsp_all[t] > r) ? 1 : 0);
            if (u >= kTable) break;
            const int q = S.nreq + r;
            W.t_slot[u] = lane; W.t_a[u] = S.ra[q]; W.t_b[u] = S.rb[q]; W.t_c[u] = S.c;
            W.t_tag[u] = kTagMove | (S.rw[q] << 8);
        }
    }
    const int fin = min(kTable, used + nsp_total);
    for (int u = fin + lane; u < kTable; u += 32) { W.t_slot[u] = -1; W.t_tag[u] = kTagNone; }
    if (lane == 0) {
        W.used = fin;
        W.rot = (rot + 1) % kSlots;
    }
}

// The round's results, all lanes: move points into their slot's window, a
// final centre's <x, d> into its voxel's result (the slot is then free).
__device__ void ingest(PackShared &W, int lane, const GridDev &g, mrf_result *out, int *err, ZState *state,
                       unsigned long long *stats)
{
    const int used = W.used;
    for (int t = lane; t < used; t += 32) {
        const int s = W.t_slot[t];
        if (s < 0) continue;
        const int tag = W.t_tag[t] & 0xff;
        if (tag == kTagMove) {
            const int idx = W.t_tag[t] >> 8;
            W.wa[s][idx] = W.t_a[t];
            W.wb[s][idx] = W.t_b[t];
            W.wv[s][idx] = W.r_v[t];
        } else if (tag == kTagFinal) {
            Slot &S = W.s[s];
            if (!S.ok) atomicExch(err, kDeviceErrBounds);
            const float cr = W.r_ipr[t], ci = W.r_ipi[t], cd = W.r_dd[t];
            mrf_result r;
            const bool have = isfinite(S.centre);
            r.index = have ? g.a_off[S.a] + (int64_t)S.b * g.n_df + S.c : -1;
            r.i_t1 = S.a; r.i_t2 = S.b; r.i_df = S.c;
            r.t1_ms = g.t1[S.a]; r.t2_ms = g.t2[S.b]; r.df_hz = g.df[S.c];
            r.cc = have ? S.centre : 0.f;
            r.m0 = cd > 0.f ? sqrtf(cr * cr + ci * ci) / cd : 0.f;
            r.phase = atan2f(ci, cr);
            r.entries_evaluated = S.evaluated;
            r.min_margin = isfinite(S.mm) ? S.mm : -1.f;
            out[S.v] = r;
            if (state) state[S.v].flags = kZDone;
            if (stats) atomicMax(&stats[4], (unsigned long long)S.rounds);
            S.pa = S.a; S.pb = S.b; S.pc = S.c;   // the next voxel of a prior chain is bounded by this result
            S.v = -1;
        }
    }
}

// Slot s's df-scan positions of the round, in scan order.
__device__ void ingest_scan(PackShared &W, int s)
{
    Slot &S = W.s[s];
    for (int t = S.scan_first; t < S.scan_first + S.scan_n; ++t) {
        const float v = W.r_v[t];
        if (isfinite(v)) { S.evaluated += 1; top2_add(v, S.g1, S.g2); }
        if (v > S.centre) { S.centre = v; S.c = W.t_c[t]; }
        S.p += 1;
    }
    S.scan_n = 0;
}

// Simulate table entries lane + 32 u (u < C) and store their results.
template <bool XONLY, bool SYM, int C>
__device__ __forceinline__ void eval_entries(PackShared &W, const ZoomArgs &A, int lane)
{
    const float2 *x[C];
    float T1[C], T2[C], df[C], ixn[C];
    bool ok[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
        const int t = lane + 32 * u;
        const int s = W.t_slot[t];
        ok[u] = false;
        T1[u] = 1000.f; T2[u] = 100.f; df[u] = 0.f; ixn[u] = 0.f;
        x[u] = A.x;
        if (s >= 0) {
            const int a = W.t_a[t], b = W.t_b[t], c = W.t_c[t];
            ok[u] = point_valid(A.g, a, b, c);
            if (ok[u]) { T1[u] = __ldg(&A.g.t1[a]); T2[u] = __ldg(&A.g.t2[b]); df[u] = __ldg(&A.g.df[c]); }
            x[u] = A.x + (size_t)W.s[s].v * A.s.n;
            ixn[u] = W.s[s].inv_xn;
        }
    }
    __syncwarp();
    Eval e[C];
    sim_multi<XONLY, SYM, C>(A.s, x, T1, T2, df, ixn, ok, e);
#pragma unroll
    for (int u = 0; u < C; ++u) {
        const int t = lane + 32 * u;
        W.r_v[t] = e[u].v;
        W.r_ipr[t] = e[u].ipr;
        W.r_ipi[t] = e[u].ipi;
        W.r_dd[t] = e[u].dd;
    }
}

// Lane 0: slot s takes work if it is idle -- the next voxel of its prior
// chain, a resumed search (steps 4-5), or a new voxel -- until it has work or
// the voxels run out.
__device__ void refill_slot(PackShared &W, int s, const ZoomArgs &A, const ZoomPlan &P, ZState *head)
{
    Slot &S = W.s[s];
    const bool takes = s < A.max_slots;
    while (S.v < 0 && (S.chain_next < S.chain_end || (takes && !W.drained))) {
        if (A.chain_len > 0 && S.chain_next < S.chain_end) {
            // the next voxel of the chain: the box of the prior's
            // half-widths around the preceding voxel's result, cut
            // by the grid, and (prior_start) that result as start
            S.v = S.chain_next++;
            S.alo = max(0, S.pa - A.prior_h1); S.ahi = min(A.g.n_t1 - 1, S.pa + A.prior_h1);
            S.blo = max(0, S.pb - A.prior_h2); S.bhi = min(A.g.n_t2 - 1, S.pb + A.prior_h2);
            S.clo = max(0, S.pc - A.prior_h3); S.chi = min(A.g.n_df - 1, S.pc + A.prior_h3);
            int a = S.pa, b = S.pb;
            if (!A.prior_start) {
                // the options' start clipped into the box, then moved
                // to a valid point inside it
                a = min(max(P.a_raw, S.alo), S.ahi);
                b = min(max(P.b_raw, S.blo), S.bhi);
                while (b > S.blo && !point_valid(A.g, a, b, S.clo)) --b;
                while (a < S.ahi && !point_valid(A.g, a, b, S.clo)) ++a;
            }
            if (!point_valid(A.g, a, b, S.clo)) atomicExch(A.err, kDeviceErrBounds);
            S.a = a; S.b = b;
            S.c = S.clo;
            S.centre = -INFINITY;
            S.evaluated = 0;
            S.mm = INFINITY;
            S.ok = 1;
            S.rounds = 0;
            S.level = 0;
            atomicOr(&W.norm_mask, 1 << s);
            enter(W, s, kS1a, P, A.g.n_df, false);
            break;
        }
        const int nv = atomicAdd(A.counter, 1);
        const int64_t first = A.chain_len > 0 ? (int64_t)nv * A.chain_len : (int64_t)nv;
        if (first >= A.V) { W.drained = 1; break; }
        if (A.phase == kPhaseTail) {
            // resume after step 3 (voxels finished earlier are skipped)
            const ZState z = A.state[nv];
            S.alo = 0; S.ahi = A.g.n_t1 - 1; S.blo = 0; S.bhi = A.g.n_t2 - 1;
            S.clo = 0; S.chi = A.g.n_df - 1;
            if (z.flags & kZDone) continue;
            S.v = nv;
            S.a = z.a; S.b = z.b; S.c = z.c;
            S.centre = z.centre;
            S.evaluated = z.evaluated;
            S.mm = z.mm;
            S.ok = z.flags & kZOk;
            S.rounds = z.flags >> 8;
            S.inv_xn = z.inv_xn;
            S.level = 0;
            enter(W, s, kS4, P, A.g.n_df, false);
        } else {
            // a voxel (or a prior chain's first voxel) on the whole grid
            S.v = (int)first;
            if (A.chain_len > 0) {
                S.chain_next = (int)first + 1;
                S.chain_end = (int)(first + A.chain_len < A.V ? first + A.chain_len : A.V);
            }
            S.alo = 0; S.ahi = A.g.n_t1 - 1; S.blo = 0; S.bhi = A.g.n_t2 - 1;
            S.clo = 0; S.chi = A.g.n_df - 1;
            S.a = P.a0; S.b = P.b0;
            S.c = S.clo;
            S.centre = -INFINITY;
            S.evaluated = 0;
            S.mm = INFINITY;
            S.ok = 1;
            S.rounds = 0;
            S.level = 0;
            atomicOr(&W.norm_mask, 1 << s);
            enter(W, s, kS1a, P, A.g.n_df, head != nullptr);
        }
    }
}

// Five CTAs per SM as the register target (96 registers, no spills): measured
// against four (121 registers), six (80, some spills) and the compiler's own
// choice (72, spills): 16.5 ms for the 128 x 128 fine-grid slice against 17.1,
// 16.9 and 18.0 ms, the same bits.
template <bool XONLY, bool SYM>
__global__ void __launch_bounds__(kPackThreads, 5) zoom_pack_kernel(ZoomArgs A)
{
    __shared__ ZoomPlan sP;
    __shared__ PackShared sW[kPackWarps];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    PackShared &W = sW[threadIdx.x >> 5];
    if (threadIdx.x == 0) sP = A.plan;
    if (lane < kSlots) { W.s[lane].v = -1; W.s[lane].scan_n = 0; W.s[lane].chain_next = W.s[lane].chain_end = 0; }
    if (lane == 0) { W.drained = 0; W.rot = 0; W.norm_mask = 0; W.used = 0; }
    __syncthreads();
    const ZoomPlan &P = sP;
    const int n = A.s.n;
    ZState *head = A.phase == kPhaseHead ? A.state : nullptr;   // saves at step 3
    unsigned long long w_rounds = 0, w_entries = 0;

    for (;;) {
        // decisions (one lane per slot)
        ingest(W, lane, A.g, A.out, A.err, head, A.stats);
        __syncwarp();
        if (lane < kSlots) ingest_scan(W, lane);
        __syncwarp();
        // every slot in turn: it takes a voxel if idle (lane 0), then the whole warp runs
        // its decisions. A slot parked at step 3 is free at once and takes the next voxel,
        // so no warp leaves with voxels left; a slot in a prior chain goes on with the
        // chain's next voxel.
        for (int s = 0; s < kSlots; ++s) {
            for (;;) {
                if (lane == 0) refill_slot(W, s, A, P, head);
                __syncwarp();
                if (W.s[s].v < 0) break;
                advance_warp(W, s, lane, P, A.g, A.max_moves, head);
                const Slot &S = W.s[s];
                if (S.v >= 0 || ((W.drained || s >= A.max_slots) && S.chain_next >= S.chain_end)) break;
            }
        }
        if (lane < kSlots && W.s[lane].v >= 0) W.s[lane].rounds += 1;
        __syncwarp();
        const bool busy = lane < kSlots && W.s[lane].v >= 0;
        if (!__any_sync(FULL, busy)) break;
        if (__any_sync(FULL, busy && W.s[lane].rounds > kMaxSlotRounds)) {
            if (lane == 0) atomicExch(A.err, kDeviceErrBounds);
            break;
        }
        // ||x|| of the voxels that arrived this round (whole warp)
        int mask = W.norm_mask;
        while (mask) {
            const int s = __ffs(mask) - 1;
            mask &= mask - 1;
            const float2 *x = A.x + (size_t)W.s[s].v * n;
            float xx = 0.f;
            for (int j = lane; j < n; j += 32) {
                const float2 z = __ldg(&x[j]);
                xx = fmaf(z.x, z.x, fmaf(z.y, z.y, xx));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(FULL, xx, o);
            if (lane == 0) W.s[s].inv_xn = xx > 0.f ? rsqrtf(xx) : 0.f;
        }
        if (lane == 0) W.norm_mask = 0;
        assign(W, lane);
        __syncwarp();
        // busy slots always list at least one point; a round with none would
        // repeat forever, so it ends the warp with an error instead
        const int used = W.used;
        if (used == 0) {
            if (lane == 0) atomicExch(A.err, kDeviceErrBounds);
            break;
        }
        w_rounds += 1;
        w_entries += used;
        if (used > 32) eval_entries<XONLY, SYM, 2>(W, A, lane);
        else eval_entries<XONLY, SYM, 1>(W, A, lane);
        __syncwarp();
    }
    if (lane == 0 && A.stats) {
        atomicAdd(&A.stats[2], w_rounds);
        atomicAdd(&A.stats[3], w_entries);
    }
}

// ---------------------------------------------------------------------------
// Step 3 batched over the voxels that share (T1, T2).
//
// Step 3 scans df at the (T1, T2) where the 2D ZOOM of step 2 stopped, over
// the window c0 - W3 .. c0 + W3 around the voxel's df index c0. Every voxel
// that stopped at the same (a, b) scans the same line of candidates, and the
// coarse lattice of step 2 has few points, so the voxels group into few
// lines with many voxels each. zoom_line_kernel simulates each line's
// candidates once per tile of kLineVox voxels and correlates each simulated
// sample with all of them: a candidate's recurrence is shared by 16 voxels,
// and the inner loop is four FMAs per voxel and timepoint.
//
// Every (voxel, candidate) value is computed with the same FP32 operations
// in the same order as the packed kernel (16-timepoint blocks, Kahan block
// sums, the voxel's own 1/||x||), so the scan decides what the voxel's own
// scan would. A voxel's scan outcome -- the first position with the largest
// CC, the top two CC values with the centre, the number of evaluated
// positions -- is reduced per 128-position chunk and then merged over the
// chunks in scan order.

constexpr int kLineVox = 16;        // voxels of a tile
constexpr int kLineEntries = 128;   // df positions of a chunk (one per thread)
constexpr int kLineTJ = 64;         // timepoints of a staged block of samples
constexpr int kLineThreads = kLineEntries;

struct LinePart {                   // one voxel's scan outcome over one chunk
    float t1;                       // largest CC (-inf when none)
    int c1;                         // its first position
    float t2;                       // second largest (as a multiset)
    int cnt;                        // finite values
};

struct LineArgs {
    SeqDev s;
    GridDev g;
    const float2 *x;
    const ZState *state;
    const int *order;               // voxels grouped by line
    const int2 *tiles;              // (first position in `order`, voxels)
    const int *n_tiles;
    int *item_counter;
    int n_chunks, W3;
    LinePart *part;                 // [voxel][chunk]
    int *vlo;                       // [voxel] first position of its tile's chunk 0
    unsigned long long *stats;      // [1] += candidates simulated
};

__device__ __forceinline__ void s3_window(int c0, int W3, int n_df, int &lo, int &hi)
{
    lo = max(0, c0 - W3);
    hi = min(n_df - 1, c0 + W3);
}

// First-position-of-the-maximum and top-two merge of two partial outcomes,
// (t1, c1, t2, cnt) <- (t1, c1, t2, cnt) + (u1, d1, u2, dn).
__device__ __forceinline__ void part_merge(float &t1, int &c1, float &t2, int &cnt, float u1, int d1, float u2, int dn)
{
    t2 = fmaxf(fmaxf(t2, u2), fminf(t1, u1));
    if (u1 > t1 || (u1 == t1 && d1 < c1)) { t1 = u1; c1 = d1; }
    cnt += dn;
}

// Voxels grouped by the (a, b) of their step 3: an open-addressing table of
// H (a power of two, at least twice the voxels) keys; each voxel learns its
// line's slot, and its rank within one of kLineBuckets df bands of the line
// (c0 binned), so that a line's voxels are laid out by df and a tile's
// windows overlap.
constexpr int kLineBuckets = 32;

__device__ __forceinline__ int line_bucket(int c0, int n_df)
{
    return (int)(((int64_t)c0 * kLineBuckets) / n_df);
}

__global__ void line_hash_kernel(const ZState *state, int64_t V, int W3, int n_df, int n_t2, int H,
                                 unsigned long long *hkey, int *hcnt, int *hist, int *vslot, int *vrank, int *err)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const ZState z = state[v];
    int lo, hi;
    s3_window(z.c, W3, n_df, lo, hi);
    vslot[v] = -1;
    if ((z.flags & kZDone) || lo >= hi) return;   // finished, or a scan of the centre alone
    const unsigned long long key = (unsigned long long)z.a * (unsigned long long)n_t2 + (unsigned long long)z.b;
    unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 32) & (unsigned)(H - 1);
    for (int probe = 0; probe < H; ++probe) {
        const unsigned long long prev = atomicCAS(&hkey[h], ~0ull, key);
        if (prev == ~0ull || prev == key) {
            vslot[v] = (int)h;
            atomicAdd(&hcnt[h], 1);
            const int bk = line_bucket(z.c, n_df);
            vrank[v] = atomicAdd(&hist[(size_t)h * kLineBuckets + bk], 1) | (bk << 24);
            return;
        }
        h = (h + 1) & (unsigned)(H - 1);
    }
    atomicExch(err, kDeviceErrBounds);   // cannot happen: the table has room for every voxel
}

// One CTA: each line's first position in `order` and its tiles of at most
// kLineVox voxels. Thread t owns slots [t H / T, (t + 1) H / T).
constexpr int kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads) line_plan_kernel(int H, const int *hcnt, int *hbase, int2 *tiles,
                                                                 int *n_tiles)
{
    __shared__ int sv[kPlanThreads], st[kPlanThreads];
    const int t = threadIdx.x;
    const int per = (H + kPlanThreads - 1) / kPlanThreads;
    const int h0 = min(H, t * per), h1 = min(H, h0 + per);
    int nv = 0, nt = 0;
    for (int h = h0; h < h1; ++h) {
        const int c = hcnt[h];
        nv += c;
        nt += (c + kLineVox - 1) / kLineVox;
    }
    sv[t] = nv;
    st[t] = nt;
    __syncthreads();
    // inclusive scan (Hillis-Steele)
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        const int av = t >= o ? sv[t - o] : 0, at = t >= o ? st[t - o] : 0;
        __syncthreads();
        sv[t] += av;
        st[t] += at;
        __syncthreads();
    }
    int vb = sv[t] - nv, tb = st[t] - nt;
    for (int h = h0; h < h1; ++h) {
        const int c = hcnt[h];
        hbase[h] = vb;
        for (int i = 0; i < c; i += kLineVox) tiles[tb++] = make_int2(vb + i, min(kLineVox, c - i));
        vb += c;
    }
    if (t == kPlanThreads - 1) *n_tiles = st[t];
}

__global__ void line_scatter_kernel(int64_t V, const int *vslot, const int *vrank, const int *hbase, const int *hist,
                                    int *order)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int h = vslot[v];
    if (h < 0) return;
    const int r = vrank[v] & 0xffffff, bk = vrank[v] >> 24;
    int off = hbase[h] + r;
    for (int b = 0; b < bk; ++b) off += hist[(size_t)h * kLineBuckets + b];
    order[off] = (int)v;
}

// Work items are (tile, chunk) pairs taken from a counter; the chunks of one
// tile are consecutive items, so its voxels' samples are read from L2.
template <bool XONLY, bool SYM>
__global__ void __launch_bounds__(kLineThreads, 4) zoom_line_kernel(LineArgs L)
{
    __shared__ __align__(16) float2 xs[kLineTJ][kLineVox];
    __shared__ float4 s_rf[3 * kLineTJ];   // x rotation (c, s, 1 - c, TE), or 12 floats of a general rotation
    __shared__ float2 s_tau[kLineTJ];
    __shared__ int s_item, s_vid[kLineVox], s_c0[kLineVox];
    __shared__ float s_ixn[kLineVox];
    __shared__ LinePart s_red[kLineThreads / 32][kLineVox];
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = L.s.n, n_df = L.g.n_df;
    const int n_items = *L.n_tiles * L.n_chunks;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(L.item_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int t = item / L.n_chunks, k = item - t * L.n_chunks;
        const int2 tl = L.tiles[t];
        const int nv = tl.y;
        if (tid < kLineVox) {
            int v = -1, c0 = 0;
            float ixn = 0.f;
            if (tid < nv) {
                v = L.order[tl.x + tid];
                c0 = L.state[v].c;
                ixn = L.state[v].inv_xn;
            }
            s_vid[tid] = v;
            s_c0[tid] = c0;
            s_ixn[tid] = ixn;
        }
        __syncthreads();
        int lo = n_df, hi = -1;
        for (int i = 0; i < nv; ++i) {
            int l, h;
            s3_window(s_c0[i], L.W3, n_df, l, h);
            lo = min(lo, l);
            hi = max(hi, h);
        }
        const int cbase = lo + k * kLineEntries;   // chunks tile the union of the tile's windows
        if (cbase > hi) {
            __syncthreads();
            continue;
        }
        if (k == 0 && tid < nv) L.vlo[s_vid[tid]] = lo;
        const int c = cbase + tid;
        const bool act = c >= lo && c <= hi;
        if (tid == 0)
            atomicAdd(&L.stats[1], (unsigned long long)(min(hi, cbase + kLineEntries - 1) - cbase + 1));
        const int a = L.state[s_vid[0]].a, b = L.state[s_vid[0]].b;
        const float T1 = __ldg(&L.g.t1[a]), T2 = __ldg(&L.g.t2[b]);
        const float df = act ? __ldg(&L.g.df[c]) : 0.f;
        const float k1 = -1.4426950408889634f / T1, k2 = -1.4426950408889634f / T2, f = df * 1.0e-3f;
        Bloch st;
        start_state(st, L.s, k1);
        Kahan kr[kLineVox], ki[kLineVox], kd;
        float pr[kLineVox], pi[kLineVox], pd = 0.f;
#pragma unroll
        for (int i = 0; i < kLineVox; ++i) { kr[i].init(); ki[i].init(); pr[i] = 0.f; pi[i] = 0.f; }
        kd.init();
        auto flush = [&]() {
#pragma unroll
            for (int i = 0; i < kLineVox; ++i) { kr[i].add(pr[i]); ki[i].add(pi[i]); pr[i] = 0.f; pi[i] = 0.f; }
            kd.add(pd);
            pd = 0.f;
        };
        // one timepoint, the operations of step_multi for one candidate; the
        // block's samples and RF coefficients come from shared memory
        auto step = [&](int jj) {
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            float q[10];
            float ta, tb = 0.f;
            const bool fin = !XONLY && L.s.finite;
            if (XONLY) {
                r = s_rf[jj];
                ta = r.w;
            } else if (fin) {
                r = s_rf[3 * jj];
                ta = s_tau[jj].x;
            } else {
                const float4 a4 = s_rf[3 * jj], b4 = s_rf[3 * jj + 1], c4 = s_rf[3 * jj + 2];
                q[0] = a4.x; q[1] = a4.y; q[2] = a4.z; q[3] = a4.w;
                q[4] = b4.x; q[5] = b4.y; q[6] = b4.z; q[7] = b4.w;
                q[8] = c4.x; q[9] = c4.y;
                ta = s_tau[jj].x;
            }
            if (!SYM) tb = s_tau[jj].y;
            if (XONLY) bloch_rf_x(st, r);
            else if (fin) bloch_rf_finite(st, r, f);
            else bloch_rf_general(st, q);
            float cs, sn;
            const float e1 = ex2_fast(k1 * ta), e2 = ex2_fast(k2 * ta);
            cis_fast(f, ta, cs, sn);
            bloch_evolve(st, e1, e2 * cs, e2 * sn);
            const float sr = st.mx, si = st.my;
            const float4 *xv = reinterpret_cast<const float4 *>(&xs[jj][0]);
#pragma unroll
            for (int i2 = 0; i2 < kLineVox / 2; ++i2) {
                const float4 z = xv[i2];
                pr[2 * i2] = fmaf(z.x, sr, fmaf(z.y, si, pr[2 * i2]));
                pi[2 * i2] = fmaf(z.y, sr, fmaf(-z.x, si, pi[2 * i2]));
                pr[2 * i2 + 1] = fmaf(z.z, sr, fmaf(z.w, si, pr[2 * i2 + 1]));
                pi[2 * i2 + 1] = fmaf(z.w, sr, fmaf(-z.z, si, pi[2 * i2 + 1]));
            }
            pd = fmaf(sr, sr, fmaf(si, si, pd));
            if (SYM) {
                bloch_evolve(st, e1, e2 * cs, e2 * sn);
            } else {
                const float e1b = ex2_fast(k1 * tb), e2b = ex2_fast(k2 * tb);
                cis_fast(f, tb, cs, sn);
                bloch_evolve(st, e1b, e2b * cs, e2b * sn);
            }
        };
        for (int j0 = 0; j0 < n; j0 += kLineTJ) {
            const int len = min(kLineTJ, n - j0);
            __syncthreads();   // the previous block of samples is consumed
            for (int q = tid; q < kLineVox * kLineTJ; q += kLineThreads) {
                const int i = q & (kLineVox - 1), jj = q / kLineVox;
                float2 z = make_float2(0.f, 0.f);
                if (i < nv && jj < len) z = __ldg(&L.x[(size_t)s_vid[i] * n + j0 + jj]);
                xs[jj][i] = z;
            }
            if (tid < len) {
                if (XONLY) {
                    s_rf[tid] = __ldg(&L.s.rfx[j0 + tid]);
                } else if (L.s.finite) {
                    s_rf[3 * tid] = __ldg(&L.s.rff[j0 + tid]);
                } else {
                    const float4 *p = reinterpret_cast<const float4 *>(L.s.rfg + 12 * (j0 + tid));
                    s_rf[3 * tid] = __ldg(p);
                    s_rf[3 * tid + 1] = __ldg(p + 1);
                    s_rf[3 * tid + 2] = __ldg(p + 2);
                }
                s_tau[tid] = __ldg(&L.s.tau[j0 + tid]);
            }
            __syncthreads();
            // 16-timepoint blocks (block boundaries at multiples of 16, as in
            // the packed kernel); a block cut by the end of the sequence is
            // flushed once after the loop
            for (int jb = 0; jb < len; jb += 16) {
                if (jb + 16 <= len) {
#pragma unroll 4
                    for (int u = 0; u < 16; ++u) step(jb + u);
                    flush();
                } else {
                    for (int u = jb; u < len; ++u) step(u);
                }
            }
        }
        flush();   // the tail block (the packed kernel flushes once more after its last full block)
        // each voxel's CC at this position, -inf outside its window or at its centre
        const float dd = kd.s;
#pragma unroll
        for (int i = 0; i < kLineVox; ++i) {
            float v = -INFINITY;
            if (act && i < nv) {
                int l, h;
                s3_window(s_c0[i], L.W3, n_df, l, h);
                if (c >= l && c <= h && c != s_c0[i]) {
                    const float ipr = kr[i].s, ipi = ki[i].s, ixn = s_ixn[i];
                    const float mag = sqrtf(fmaf(ipr, ipr, ipi * ipi));
                    v = (dd > 0.f && ixn > 0.f) ? mag * ixn * rsqrtf(dd) : 0.f;
                }
            }
            float t1 = v, t2 = -INFINITY;
            int c1 = c, cnt = isfinite(v) ? 1 : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float u1 = __shfl_xor_sync(FULL, t1, o), u2 = __shfl_xor_sync(FULL, t2, o);
                const int d1 = __shfl_xor_sync(FULL, c1, o), dn = __shfl_xor_sync(FULL, cnt, o);
                part_merge(t1, c1, t2, cnt, u1, d1, u2, dn);
            }
            if (lane == 0) s_red[warp][i] = LinePart{t1, c1, t2, cnt};
        }
        __syncthreads();
        if (tid < nv) {
            LinePart r = s_red[0][tid];
#pragma unroll
            for (int w = 1; w < kLineThreads / 32; ++w) {
                const LinePart u = s_red[w][tid];
                part_merge(r.t1, r.c1, r.t2, r.cnt, u.t1, u.c1, u.t2, u.cnt);
            }
            L.part[(size_t)s_vid[tid] * L.n_chunks + k] = r;
        }
        __syncthreads();
    }
}

// Each voxel's step 3 from its chunks, in scan order: the first position of
// the largest CC moves the centre if strictly better; the decision set's top
// two (with the centre) give the margin.
__global__ void line_merge_kernel(int64_t V, int W3, int n_df, int n_chunks, const int *vslot, const LinePart *part,
                                  const int *vlo, ZState *state, unsigned long long *stats)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V || vslot[v] < 0) return;
    ZState z = state[v];
    int lo, hi;
    s3_window(z.c, W3, n_df, lo, hi);
    float best = z.centre, g1 = z.centre, g2 = -INFINITY;
    int bc = z.c, cnt = 0;
    const int tlo = vlo[v];
    for (int k = (lo - tlo) / kLineEntries; k <= (hi - tlo) / kLineEntries; ++k) {
        const LinePart p = part[(size_t)v * n_chunks + k];
        if (p.t1 > best) { best = p.t1; bc = p.c1; }
        top2_add(p.t1, g1, g2);
        top2_add(p.t2, g1, g2);
        cnt += p.cnt;
    }
    if (isfinite(g2)) z.mm = fminf(z.mm, g1 - g2);
    z.evaluated += cnt;
    const unsigned m = __activemask();
    const unsigned tot = __reduce_add_sync(m, (unsigned)cnt);
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&stats[0], (unsigned long long)tot);
    z.centre = best;
    z.c = bc;
    state[v] = z;
}

int snap(double h_phys, double step)
{
    const int h = (int)floor(h_phys / step + 0.5);
    return h < 1 ? 1 : h;
}

// Grid of the packed kernel: every resident CTA slot of the device, but no
// more CTAs than the voxels need (kSlots voxels in flight per warp). The four
// instantiations share one resource footprint up to a few registers.
unsigned pack_blocks(const mrf_ctx *ctx, int64_t V)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zoom_pack_kernel<true, true>, kPackThreads, 0);
    per_sm = std::max(1, per_sm);
    const int64_t per_cta = (int64_t)kSlots * kPackWarps;
    const int64_t blocks = std::min<int64_t>((int64_t)per_sm * ctx->sm_count, (V + per_cta - 1) / per_cta);
    return (unsigned)std::max<int64_t>(blocks, 1);
}

// Launch the packed kernel instantiated for the sequence's RF form and symmetry.
void launch_pack(const ZoomArgs &A, unsigned blocks, cudaStream_t stream)
{
    if (A.s.xonly && A.s.symmetric) zoom_pack_kernel<true, true><<<blocks, kPackThreads, 0, stream>>>(A);
    else if (A.s.xonly) zoom_pack_kernel<true, false><<<blocks, kPackThreads, 0, stream>>>(A);
    else if (A.s.symmetric) zoom_pack_kernel<false, true><<<blocks, kPackThreads, 0, stream>>>(A);
    else zoom_pack_kernel<false, false><<<blocks, kPackThreads, 0, stream>>>(A);
}

// Line kernel: a persistent grid over the (tile, chunk) items, no more CTAs
// than the items can need.
void launch_line(const mrf_ctx *ctx, const LineArgs &L, int64_t max_items, cudaStream_t stream)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zoom_line_kernel<true, true>, kLineThreads, 0);
    per_sm = std::max(1, per_sm);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * ctx->sm_count, max_items));
    if (L.s.xonly && L.s.symmetric) zoom_line_kernel<true, true><<<blocks, kLineThreads, 0, stream>>>(L);
    else if (L.s.xonly) zoom_line_kernel<true, false><<<blocks, kLineThreads, 0, stream>>>(L);
    else if (L.s.symmetric) zoom_line_kernel<false, true><<<blocks, kLineThreads, 0, stream>>>(L);
    else zoom_line_kernel<false, false><<<blocks, kLineThreads, 0, stream>>>(L);
}

}  // namespace

namespace {

// MRF-ZOOM with the spatial-neighbour prior (Methods, Experiment 3): the
// voxels, in their given (raster) order, form chains of opts->prior_chain
// consecutive voxels (the whole slice when it is V or more: the paper's
// single chain); a chain's first voxel is searched on the whole grid, every
// later one on the grid overlapped with the prior's ranges around the result
// of the voxel before it, started there (prior_start) or at the options'
// start clipped into those ranges. Each chain runs in one slot of the packed
// kernel, every step in that kernel; chains run in parallel.
int zoom_with_chains(mrf_ctx *ctx, const ZoomPlan &P, const SeqDev &sd, const GridDev &gdev,
                     const mrf_grid_desc *gd, const mrf_zoom_opts *o, const void *fp, int64_t V, mrf_result *out,
                     cudaStream_t stream)
{
    const int64_t L = std::min<int64_t>(o->prior_chain, std::max<int64_t>(V, 1));
    const int64_t chains = (V + L - 1) / L;
    const size_t total = 256;
    int rc = budget_charge(ctx, total);
    if (rc) return rc;
    int *counter = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&counter, total, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, total, stream);
    if (e != cudaSuccess) {
        if (counter) cudaFreeAsync(counter, stream);
        budget_release(ctx, total);
        return cuda_fail(e, "zoom prior scratch");
    }
    ZoomArgs A;
    A.s = sd;
    A.g = gdev;
    A.dhi = A.dlo8 = nullptr;
    A.dnorm = nullptr;
    A.dscale = nullptr;
    A.ld = 0;
    A.plan = P;
    A.x = (const float2 *)fp;
    A.V = V;
    A.out = out;
    A.counter = counter;
    A.err = ctx->err_flag;
    A.max_moves = 1 << 20;
    A.state = nullptr;
    A.phase = kPhaseAll;
    A.chain_len = (int)L;
    // half-widths in whole grid steps (an axis's length at most: wider windows change nothing)
    auto steps = [](double half, double step, int n) { return (int)std::min<double>(floor(half / step + 1e-9), n); };
    A.prior_h1 = steps(o->prior_t1_ms, gd->t1_step, gd->n_t1);
    A.prior_h2 = steps(o->prior_t2_ms, gd->t2_step, gd->n_t2);
    A.prior_h3 = steps(o->prior_df_hz, gd->df_step, gd->n_df);
    A.prior_start = o->prior_start;
    A.stats = ctx->dev_stats;
    // chains run one voxel after another: spread them over the resident warps,
    // as few per warp as fill the device (a warp's candidate table then serves
    // fewer chains, which advance in fewer rounds)
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zoom_pack_kernel<true, true>, kPackThreads, 0);
    const int64_t warps = (int64_t)std::max(1, per_sm) * ctx->sm_count * kPackWarps;
    A.max_slots = (int)std::min<int64_t>(kSlots, std::max<int64_t>(1, (chains + warps - 1) / warps));
    const int64_t per_cta = (int64_t)A.max_slots * kPackWarps;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(warps / kPackWarps, (chains + per_cta - 1) / per_cta));
    {
        ProfScope prof(ctx, kProfZoom, stream);
        launch_pack(A, blocks, stream);
    }
    e = cudaGetLastError();
    cudaFreeAsync(counter, stream);
    budget_release(ctx, total);
    if (e != cudaSuccess) return cuda_fail(e, "zoom (prior) launch");
    return MRF_OK;
}

}  // namespace

// The search plan on the host, in FP64, with the stage machine's snapping
// rules (every on-the-fly and dictionary-backed search uses this one).
static int plan_zoom(const mrf_seq *seq, const mrf_grid_desc *gd, const mrf_zoom_opts *o, ZoomPlan &P)
{
    const double omega = o->omega_hz > 0 ? o->omega_hz : 1000.0 / seq->min_tr;
    P = ZoomPlan{};
    int a = (int)floor((o->t1_init_ms - gd->t1_min) / gd->t1_step + 0.5);
    int b = (int)floor((o->t2_init_ms - gd->t2_min) / gd->t2_step + 0.5);
    P.a_raw = a;
    P.b_raw = b;
    a = std::max(0, std::min(a, gd->n_t1 - 1));
    b = std::max(0, std::min(b, gd->n_t2 - 1));
    auto valid = [&](int aa, int bb) {
        return !gd->require_t2_lt_t1 || gd->t2_min + (double)bb * gd->t2_step < gd->t1_min + (double)aa * gd->t1_step;
    };
    while (b > 0 && !valid(a, b)) --b;
    while (a < gd->n_t1 - 1 && !valid(a, b)) ++a;
    if (!valid(a, b)) return set_error(MRF_E_INVALID, "zoom: the grid has no valid starting point");
    P.a0 = a;
    P.b0 = b;
    P.hA = snap(o->s1a_step_frac * omega, gd->df_step);
    P.hB = snap(o->s1b_step_frac * omega, gd->df_step);
    P.K1b = (int)floor(o->s1b_half_frac * omega / gd->df_step + 0.5) / P.hB;
    P.hC = snap(omega, gd->df_step);
    P.W3 = (int)floor(o->s3_half_frac * omega / gd->df_step + 0.5);
    for (int l = 0, p1 = -1, p2 = -1; l < o->n_s2; ++l) {
        const int h1 = snap(o->s2_t1_ms[l], gd->t1_step), h2 = snap(o->s2_t2_ms[l], gd->t2_step);
        if (h1 == p1 && h2 == p2) continue;
        p1 = h1; p2 = h2;
        P.s2_h1[P.n_s2] = h1; P.s2_h2[P.n_s2] = h2; P.n_s2++;
    }
    for (int l = 0, pp = -1, ph = -1; l < o->n_s4; ++l) {
        const int p = o->s4_param[l], h = snap(o->s4_ms[l], p == 0 ? gd->t1_step : gd->t2_step);
        if (p == pp && h == ph) continue;
        pp = p; ph = h;
        P.s4_p[P.n_s4] = p; P.s4_h[P.n_s4] = h; P.n_s4++;
    }
    return MRF_OK;
}

int run_zoom(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *gd, const mrf_zoom_opts *o, const void *fp,
             int64_t V, mrf_result *out, cudaStream_t stream)
{
    ZoomPlan P;
    int rc = plan_zoom(seq, gd, o, P);
    if (rc) return rc;

    GridDev gdev;
    void *gblock = nullptr;
    size_t gbytes = 0;
    rc = grid_upload_async(ctx, gd, stream, &gdev, &gblock, &gbytes);
    if (rc) return rc;

    if (o->prior_chain > 0) {
        rc = zoom_with_chains(ctx, P, seq->dev(), gdev, gd, o, fp, V, out, stream);
        cudaFreeAsync(gblock, stream);
        budget_release(ctx, gbytes);
        return rc;
    }

    // Split search (step 3 batched by line) unless step 3 never scans. Scratch,
    // one block: counters + line counts | state | keys | line bases | per-voxel
    // slot, rank, order | tiles | chunk outcomes.
    const int n_chunks = (gd->n_df + kLineEntries - 1) / kLineEntries;
    // (a window of fewer than 64 positions leaves the line kernel's lanes mostly idle)
    const bool split = std::min(2 * P.W3 + 1, gd->n_df) >= 64 && V * (int64_t)n_chunks < (int64_t)INT32_MAX / 2 &&
                       V < (1 << 24);
    int H = 1024;
    while (split && (int64_t)H < 2 * V) H <<= 1;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t Vs = (size_t)V;
    const size_t o_hcnt = 256, o_hist = o_hcnt + al(4 * (size_t)H);
    const size_t o_state = o_hist + al(4 * (size_t)H * kLineBuckets), o_hkey = o_state + al(sizeof(ZState) * Vs);
    const size_t o_hbase = o_hkey + al(8 * (size_t)H), o_vslot = o_hbase + al(4 * (size_t)H);
    const size_t o_vrank = o_vslot + al(4 * Vs), o_order = o_vrank + al(4 * Vs), o_tiles = o_order + al(4 * Vs);
    const size_t o_vlo = o_tiles + al(8 * Vs), o_part = o_vlo + al(4 * Vs);
    const size_t total = o_part + al(sizeof(LinePart) * Vs * n_chunks);
    const size_t scratch = split ? total : 256;
    rc = budget_charge(ctx, scratch);
    if (rc) { cudaFreeAsync(gblock, stream); budget_release(ctx, gbytes); return rc; }
    uint8_t *sb = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sb, scratch, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb, 0, split ? o_state : 256, stream);
    if (e == cudaSuccess && split) e = cudaMemsetAsync(sb + o_hkey, 0xFF, 8 * (size_t)H, stream);
    if (e != cudaSuccess) {
        if (sb) cudaFreeAsync(sb, stream);
        budget_release(ctx, scratch);
        cudaFreeAsync(gblock, stream);
        budget_release(ctx, gbytes);
        return cuda_fail(e, "zoom scratch");
    }
    int *counters = (int *)sb;   // [0] head / whole search, [1] tail, [2] tiles, [3] line items
    ZoomArgs A;
    A.s = seq->dev();
    A.g = gdev;
    A.dhi = A.dlo8 = nullptr;
    A.dnorm = nullptr;
    A.dscale = nullptr;
    A.ld = 0;
    A.plan = P;
    A.x = (const float2 *)fp;
    A.V = V;
    A.out = out;
    A.counter = counters;
    A.err = ctx->err_flag;
    A.max_moves = 1 << 20;
    A.chain_len = 0;
    A.prior_h1 = A.prior_h2 = A.prior_h3 = 0;
    A.prior_start = 0;
    A.max_slots = kSlots;
    A.state = split ? (ZState *)(sb + o_state) : nullptr;
    A.phase = split ? kPhaseHead : kPhaseAll;
    A.stats = ctx->dev_stats;
    const unsigned blocks = pack_blocks(ctx, V);
    {
        ProfScope prof(ctx, kProfZoom, stream);
        launch_pack(A, blocks, stream);
        if (split) {
            ZState *state = (ZState *)(sb + o_state);
            unsigned long long *hkey = (unsigned long long *)(sb + o_hkey);
            int *hcnt = (int *)(sb + o_hcnt), *hbase = (int *)(sb + o_hbase), *hist = (int *)(sb + o_hist);
            int *vlo = (int *)(sb + o_vlo);
            int *vslot = (int *)(sb + o_vslot), *vrank = (int *)(sb + o_vrank), *order = (int *)(sb + o_order);
            int2 *tiles = (int2 *)(sb + o_tiles);
            LinePart *part = (LinePart *)(sb + o_part);
            const unsigned vb = (unsigned)((V + 255) / 256);
            line_hash_kernel<<<vb, 256, 0, stream>>>(state, V, P.W3, gd->n_df, gd->n_t2, H, hkey, hcnt, hist,
                                                     vslot, vrank, ctx->err_flag);
            line_plan_kernel<<<1, kPlanThreads, 0, stream>>>(H, hcnt, hbase, tiles, counters + 2);
            line_scatter_kernel<<<vb, 256, 0, stream>>>(V, vslot, vrank, hbase, hist, order);
            LineArgs L;
            L.s = A.s;
            L.g = gdev;
            L.x = A.x;
            L.state = state;
            L.order = order;
            L.tiles = tiles;
            L.n_tiles = counters + 2;
            L.item_counter = counters + 3;
            L.n_chunks = n_chunks;
            L.W3 = P.W3;
            L.part = part;
            L.vlo = vlo;
            L.stats = ctx->dev_stats;
            {
                ProfScope lp(ctx, kProfZoomLine, stream);
                launch_line(ctx, L, V * (int64_t)n_chunks, stream);
            }
            line_merge_kernel<<<vb, 256, 0, stream>>>(V, P.W3, gd->n_df, n_chunks, vslot, part, vlo, state,
                                                      ctx->dev_stats);
            A.counter = counters + 1;
            A.phase = kPhaseTail;
            launch_pack(A, blocks, stream);
            count_launch(ctx, 5);   // hash, plan, scatter, merge, tail (head and line kernels counted above)
        }
    }
    e = cudaGetLastError();
    cudaFreeAsync(sb, stream);
    cudaFreeAsync(gblock, stream);
    budget_release(ctx, scratch + gbytes);
    if (e != cudaSuccess) return cuda_fail(e, "zoom launch");
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// MRF-ZOOM over a resident dictionary (Experiment 2's "full pre-made
// dictionary" variant): the same search on the dictionary's grid, every
// candidate's CC read from the stored normalised entry.

extern "C" int mrf_zoom_search_dict(mrf_ctx *ctx, const mrf_dict *d, const mrf_zoom_opts *opts, const void *fp,
                                    int64_t V, mrf_result *out, void *stream_v)
{
    if (!ctx || !d) return set_error(MRF_E_INVALID, "NULL argument");
    if (d->dtype != MRF_F32 && d->dtype != MRF_BF16)
        return set_error(MRF_E_UNSUPPORTED, "zoom over a dictionary needs an MRF_F32 or MRF_BF16 dictionary");
    if (opts && opts->prior_chain != 0)
        return set_error(MRF_E_UNSUPPORTED, "zoom over a dictionary: the spatial-neighbour prior is mrf_zoom_search's");
    if (V < 0 || V > INT32_MAX) return set_error(MRF_E_INVALID, "zoom: V must be in [0, 2^31 - 1]");
    mrf_zoom_opts def;
    if (!opts) { mrf_zoom_opts_default(&def); opts = &def; }
    if (opts->n_s2 < 0 || opts->n_s2 > MRF_ZOOM_MAX_LEVELS || opts->n_s4 < 0 || opts->n_s4 > MRF_ZOOM_MAX_LEVELS)
        return set_error(MRF_E_INVALID, "zoom: level counts out of range");
    for (int i = 0; i < opts->n_s4; ++i)
        if (opts->s4_param[i] != 0 && opts->s4_param[i] != 1) return set_error(MRF_E_INVALID, "zoom: s4_param must be 0/1");
    if (!(opts->s1a_step_frac > 0) || !(opts->s1b_step_frac > 0) || opts->s1b_half_frac < 0 || opts->s3_half_frac < 0)
        return set_error(MRF_E_INVALID, "zoom: bad df search fractions");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    cudaSetDevice(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_v;
    ZoomPlan P;
    int rc = plan_zoom(d->seq, &d->grid.desc, opts, P);
    if (rc) return rc;
    rc = budget_charge(ctx, 256);
    if (rc) return rc;
    int *counter = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&counter, 256, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) { budget_release(ctx, 256); return cuda_fail(e, "zoom scratch"); }
    ZoomArgs A;
    A.s = d->seq->dev();
    A.g = d->grid.dev();
    A.dhi = (const uint8_t *)d->hi;
    A.dlo8 = d->lo ? (const uint8_t *)d->lo + (size_t)d->entries * d->ld : nullptr;   // the residual plane
    A.dnorm = d->norm;
    A.dscale = d->scale;
    A.ld = d->ld;
    A.plan = P;
    A.x = (const float2 *)fp;
    A.V = V;
    A.out = out;
    A.counter = counter;
    A.err = ctx->err_flag;
    A.max_moves = 1 << 20;
    A.chain_len = 0;
    A.prior_h1 = A.prior_h2 = A.prior_h3 = 0;
    A.prior_start = 0;
    A.max_slots = kSlots;
    A.state = nullptr;
    A.phase = kPhaseAll;
    A.stats = nullptr;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zoom_dict_kernel, kZoomThreads, 0);
    per_sm = std::max(1, per_sm);
    int64_t blocks = std::min<int64_t>((int64_t)per_sm * ctx->sm_count, (V + 7) / 8);
    blocks = std::max<int64_t>(blocks, 1);
    {
        ProfScope prof(ctx, kProfZoom, stream);
        zoom_dict_kernel<<<(unsigned)blocks, kZoomThreads, 0, stream>>>(A);
    }
    e = cudaGetLastError();
    cudaFreeAsync(counter, stream);
    budget_release(ctx, 256);
    if (e != cudaSuccess) return cuda_fail(e, "zoom (dictionary) launch");
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free ZOOM search.
//
// Some callers cannot let a library allocate device memory while they run:
// a host framework that reserved the GPU's memory up front for its own pool
// (a cudaMalloc from here could fail or fragment that pool), or a
// reconstruction loop that matches slice after slice and must never pay
// allocation latency or meet an out-of-memory error in the middle of a scan.
// For them, mrf_zoom_search_static keeps all per-call scratch of the ZOOM
// search -- the voxel work counter and the grid's axis/offset tables -- in
// the fixed device array below, so a call allocates nothing: it copies the
// tables into the array, clears the counter and launches the same kernel as
// mrf_zoom_search. The caller still passes its fingerprints and result
// buffer.
//
// The array lives in every GPU that loads this library until the process
// exits. All calls share it and it keeps the last call's contents, so calls
// whose work overlaps on the GPU (different streams, or host threads racing)
// corrupt each other: serialise them. The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, with that device current);
// make that first call before any stream capture.

namespace {

constexpr size_t kZoomStaticBytes = MRF_ZOOM_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) uint8_t g_zoom_static_scratch[kZoomStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;                         // guards the address table and the host staging
void *g_static_addr[kMaxDevices] = {nullptr};
alignas(256) uint8_t g_static_host[kZoomStaticBytes];   // host staging for the table copy

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int mrf_zoom_search_static(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *gd,
                                      const mrf_zoom_opts *opts, const void *fp, int64_t V, mrf_result *out,
                                      void *stream_v)
{
    if (!ctx || !seq || !gd) return set_error(MRF_E_INVALID, "NULL argument");
    int rc = grid_validate(gd);
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
    if (opts->prior_chain != 0)
        return set_error(MRF_E_UNSUPPORTED, "zoom (static scratch): the spatial-neighbour prior needs mrf_zoom_search");
    // scratch layout: [counter][t1][t2][df][a_off][nb], 256-byte aligned pieces
    const size_t nt1 = gd->n_t1, nt2 = gd->n_t2, ndf = gd->n_df;
    const size_t o_t1 = 256, o_t2 = o_t1 + al256(4 * nt1), o_df = o_t2 + al256(4 * nt2);
    const size_t o_ao = o_df + al256(4 * ndf), o_nb = o_ao + al256(8 * (nt1 + 1)), need = o_nb + al256(4 * nt1);
    if (need > kZoomStaticBytes)
        return set_error(MRF_E_INVALID, "zoom (static scratch): the grid needs " + std::to_string(need) +
                                            " bytes of tables, more than the fixed " +
                                            std::to_string(kZoomStaticBytes) + "-byte scratch array; use mrf_zoom_search");
    if (V == 0) return MRF_OK;
    if (!fp || !out) return set_error(MRF_E_INVALID, "NULL device buffer");
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return set_error(MRF_E_INVALID, "device index out of range");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t stream = (cudaStream_t)stream_v;

    // the plan of mrf_zoom_search
    ZoomPlan P;
    rc = plan_zoom(seq, gd, opts, P);
    if (rc) return rc;
    auto t1v = [&](int i) { return gd->t1_min + (double)i * gd->t1_step; };
    auto t2v = [&](int i) { return gd->t2_min + (double)i * gd->t2_step; };
    auto valid = [&](int aa, int bb) { return !gd->require_t2_lt_t1 || t2v(bb) < t1v(aa); };

    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[ctx->device]) {
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_zoom_static_scratch);
        if (e != cudaSuccess || !addr) return cuda_fail(e, "cudaGetSymbolAddress(static ZOOM scratch)");
        g_static_addr[ctx->device] = addr;
    }
    uint8_t *dev = (uint8_t *)g_static_addr[ctx->device];
    // tables into the host staging, then one copy into the array
    float *t1 = (float *)(g_static_host + o_t1), *t2 = (float *)(g_static_host + o_t2);
    float *df = (float *)(g_static_host + o_df);
    int64_t *ao = (int64_t *)(g_static_host + o_ao);
    int32_t *nb = (int32_t *)(g_static_host + o_nb);
    for (int i = 0; i < gd->n_t1; ++i) t1[i] = (float)t1v(i);
    for (int i = 0; i < gd->n_t2; ++i) t2[i] = (float)t2v(i);
    for (int i = 0; i < gd->n_df; ++i) df[i] = (float)(gd->df_min + (double)i * gd->df_step);
    ao[0] = 0;
    for (int i = 0; i < gd->n_t1; ++i) {
        int32_t k = 0;
        for (int j = 0; j < gd->n_t2; ++j) if (valid(i, j)) k = j + 1;
        nb[i] = k;
        ao[i + 1] = ao[i] + (int64_t)k * gd->n_df;
    }
    // pageable source: the copy is staged before the call returns, so the
    // host staging may be refilled by the next call
    e = cudaMemcpyAsync(dev + o_t1, g_static_host + o_t1, need - o_t1, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, 256, stream);   // voxel work counter starts at 0
    if (e != cudaSuccess) return cuda_fail(e, "static ZOOM scratch upload");

    ZoomArgs A;
    A.s = seq->dev();
    A.g.n_t1 = gd->n_t1; A.g.n_t2 = gd->n_t2; A.g.n_df = gd->n_df;
    A.g.t1 = (const float *)(dev + o_t1);
    A.g.t2 = (const float *)(dev + o_t2);
    A.g.df = (const float *)(dev + o_df);
    A.g.a_off = (const int64_t *)(dev + o_ao);
    A.g.nb = (const int32_t *)(dev + o_nb);
    A.g.count = ao[gd->n_t1];
    A.g.a_full = gd->n_t1;
    while (A.g.a_full > 0 && nb[A.g.a_full - 1] == gd->n_t2) --A.g.a_full;
    A.dhi = A.dlo8 = nullptr;
    A.dnorm = nullptr;
    A.dscale = nullptr;
    A.ld = 0;
    A.plan = P;
    A.x = (const float2 *)fp;
    A.V = V;
    A.out = out;
    A.counter = (int *)dev;
    A.err = ctx->err_flag;
    A.max_moves = 1 << 20;
    A.chain_len = 0;
    A.prior_h1 = A.prior_h2 = A.prior_h3 = 0;
    A.prior_start = 0;
    A.max_slots = kSlots;
    A.state = nullptr;
    A.phase = kPhaseAll;   // one kernel: the split search's scratch grows with V
    A.stats = ctx->dev_stats;
    const unsigned blocks = pack_blocks(ctx, V);
    launch_pack(A, blocks, stream);
    count_launch(ctx);   // no profile events here: creating them is not allocation-free
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "zoom launch (static scratch)");
    return MRF_OK;
}
