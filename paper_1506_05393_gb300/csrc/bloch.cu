// Bloch-recurrence kernels: dictionary generation (normalise + quantise) and
// on-the-fly simulation of arbitrary parameter triples.
//
// Dictionary generation (Theory: brute-force DGS simulates every grid entry;
// entries normalised to unit norm so CC is |inner product|):
//   one thread per entry, FP32 recurrence in registers (bloch.cuh);
//   MRF_F32 (fp16 row plus e4m3 planes of the values and of the fp16
//   residuals, split.cuh): one pass writes the raw signal and accumulates
//   ||d||^2; the entry's scale 1 / ||d|| makes it unit norm;
//   BF16 / FP8: pass 1 accumulates ||d||^2 (and max |d| for FP8), pass 2
//   re-runs the recurrence and writes the normalised (BF16, scale 1) or
//   scaled e4m3 (FP8) row.
// Rows are staged per warp in shared memory (32 entries x 128 bytes, XOR
// swizzled on 16-byte chunks) and leave as full 128-byte lines of 16-byte
// stores, so the kernel streams HBM writes at one pass of the output.
// Symmetric x-rotation sequences (the randomised IR-bSSFP train) take the
// df-major kernel dict_gen_xsym_kernel: a warp's lanes share the df index, so
// e^{i theta} is a broadcast load from a [df][j] table, E1 / E2 are exp2f of
// TE_j, and the RF of each row chunk is staged per warp. Other sequences take
// dict_gen_kernel, whose evolution factors come from tables indexed by grid
// axis (E1 by T1, E2 by T2, e^{i theta} by df), built once per dictionary with
// CUDA's expf/sincospif.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "bloch.cuh"
#include "mrf_internal.h"
#include "split.cuh"

namespace {

constexpr int kGenThreads = 128;

// Factor tables. General sequences keep both intervals of a step, TE_j and
// TR_j - TE_j; a symmetric sequence (TE_j = TR_j - TE_j) keeps one, and its
// tables are half the size (e1s, e2s, ciss).
struct Tables {
    const float2 *e1;    // [n_t1][n]: (E1 over TE_j, E1 over TR_j - TE_j)
    const float2 *e2;    // [n_t2][n]
    const float4 *cis;   // [n][n_df]: (cos, sin) over TE_j, then over TR_j - TE_j
    const float *e1s;    // symmetric: [n_t1][n] E1 over TE_j
    const float *e2s;    // symmetric: [n_t2][n]
    const float2 *ciss;  // symmetric: [n][n_df] (cos, sin) over TE_j
    const float *e1_inv; // [n_t1]: E1 over the inversion delay
};

__global__ void tables_kernel(SeqDev s, GridDev g, float2 *e1, float2 *e2, float4 *cis, float *e1_inv)
{
    // symmetric sequences: the same storage holds the one-interval tables
    float *e1s = reinterpret_cast<float *>(e1), *e2s = reinterpret_cast<float *>(e2);
    float2 *ciss = reinterpret_cast<float2 *>(cis);
    const bool sym = s.symmetric;
    const int64_t n = s.n;
    const int64_t n1 = (int64_t)g.n_t1 * n, n2 = (int64_t)g.n_t2 * n, n3 = n * g.n_df;
    const int64_t total = n1 + n2 + n3 + g.n_t1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n1) {
            const int a = (int)(i / n), j = (int)(i % n);
            const float2 t = s.tau[j];
            const float T1 = g.t1[a];
            if (sym) e1s[i] = expf(-t.x / T1);
            else e1[i] = make_float2(expf(-t.x / T1), expf(-t.y / T1));
        } else if (i < n1 + n2) {
            const int64_t k = i - n1;
            const int b = (int)(k / n), j = (int)(k % n);
            const float2 t = s.tau[j];
            const float T2 = g.t2[b];
            if (sym) e2s[k] = expf(-t.x / T2);
            else e2[k] = make_float2(expf(-t.x / T2), expf(-t.y / T2));
        } else if (i < n1 + n2 + n3) {
            const int64_t k = i - n1 - n2;
            const int j = (int)(k / g.n_df), c = (int)(k % g.n_df);
            const float2 t = s.tau[j];
            const float f = g.df[c] * 1.0e-3f;
            float ta = f * t.x, tb = f * t.y;
            ta -= rintf(ta);
            tb -= rintf(tb);
            float sa, ca, sb, cb;
            sincospif(2.0f * ta, &sa, &ca);
            if (sym) {
                ciss[k] = make_float2(ca, sa);
            } else {
                sincospif(2.0f * tb, &sb, &cb);
                cis[k] = make_float4(ca, sa, cb, sb);
            }
        } else {
            const int a = (int)(i - n1 - n2 - n3);
            e1_inv[a] = expf(-s.inv_delay / g.t1[a]);
        }
    }
}

// Linear entry index -> (a, b, c): binary search over the T1 offsets.
__device__ __forceinline__ void unravel(const GridDev &g, int64_t e, int &a, int &b, int &c)
{
    int lo = 0, hi = g.n_t1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&g.a_off[mid]) <= e) lo = mid; else hi = mid - 1;
    }
    a = lo;
    const int64_t rem = e - __ldg(&g.a_off[a]);
    b = (int)(rem / g.n_df);
    c = (int)(rem % g.n_df);
}

// One timepoint with tabulated factors (SYM: one factor set for both
// intervals of the step).
template <bool XONLY, bool SYM>
__device__ __forceinline__ void step_tab(Bloch &st, const SeqDev &s, const Tables &t, int n, int n_df, int a, int b,
                                         int c, int j, float fdf, float &sr, float &si)
{
    bloch_rf<XONLY>(st, s, j, fdf);
    if (SYM) {
        const float e1 = __ldg(&t.e1s[(int64_t)a * n + j]);
        const float e2 = __ldg(&t.e2s[(int64_t)b * n + j]);
        const float2 z = __ldg(&t.ciss[(int64_t)j * n_df + c]);
        const float zr = e2 * z.x, zi = e2 * z.y;
        bloch_evolve(st, e1, zr, zi);
        sr = st.mx;
        si = st.my;
        bloch_evolve(st, e1, zr, zi);
    } else {
        const float2 e1 = __ldg(&t.e1[(int64_t)a * n + j]);
        const float2 e2 = __ldg(&t.e2[(int64_t)b * n + j]);
        const float4 z = __ldg(&t.cis[(int64_t)j * n_df + c]);
        bloch_evolve(st, e1.x, e2.x * z.x, e2.x * z.y);
        sr = st.mx;
        si = st.my;
        bloch_evolve(st, e1.y, e2.y * z.z, e2.y * z.w);
    }
}

// Symmetric sequences: the factors of kFacG consecutive timepoints, fetched a
// group ahead of their use so that one group's table loads overlap the
// previous group's recurrence.
constexpr int kFacG = 8;

struct FacGroup {
    float e1[kFacG], e2[kFacG];
    float2 z[kFacG];
};

// An entry's rows of the symmetric tables; the tables carry kFacG samples of
// padding past their end, so a group may run past the last timepoint.
struct FacRows {
    const float *e1, *e2;    // E1 / E2 of this entry's T1 / T2, by timepoint
    const float2 *z;         // e^{i theta} of this entry's df at timepoint 0; stride n_df
    int n_df;
};

__device__ __forceinline__ void fac_load(FacGroup &f, const FacRows &r, int jb)
{
    const float2 *z = r.z + (size_t)jb * r.n_df;
#pragma unroll
    for (int g = 0; g < kFacG; ++g) {
        f.e1[g] = __ldg(r.e1 + jb + g);
        f.e2[g] = __ldg(r.e2 + jb + g);
        f.z[g] = __ldg(z);
        z += r.n_df;
    }
}

// One timepoint from preloaded symmetric factors (the same arithmetic as step_tab).
template <bool XONLY>
__device__ __forceinline__ void step_fac(Bloch &st, const SeqDev &s, const FacGroup &f, int g, int j, float fdf,
                                         float &sr, float &si)
{
    bloch_rf<XONLY>(st, s, j, fdf);
    const float zr = f.e2[g] * f.z[g].x, zi = f.e2[g] * f.z[g].y;
    bloch_evolve(st, f.e1[g], zr, zi);
    sr = st.mx;
    si = st.my;
    bloch_evolve(st, f.e1[g], zr, zi);
}

// Packs timepoint values into 16-byte vectors for the staged row writer.
template <int OUT>
struct Packer;

// F32: the fp16 pair (4 bytes per timepoint) in `hi`; in `lo`, words 0-1 the
// e4m3 value pairs and words 2-3 the e4m3 residual pairs of the four slots.
template <>
struct Packer<MRF_F32> {
    static constexpr int kBpt = 4;
    uint32_t hi[4], lo[4];
    __device__ __forceinline__ void put(int slot, float vr, float vi, float)
    {
        const SplitPair p = split_pair(vr, vi, kSplitHiD);
        hi[slot] = p.hi;
        const int w = slot >> 1, sh = 16 * (slot & 1);
        lo[w] |= (uint32_t)p.h8 << sh;
        lo[2 + w] |= (uint32_t)p.l8 << sh;
    }
};

// BF16: 4 bytes per timepoint.

template <>
struct Packer<MRF_BF16> {
    static constexpr int kBpt = 4;
    uint32_t hi[4], lo[4];
    __device__ __forceinline__ void put(int slot, float vr, float vi, float)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(vr, vi);
        hi[slot] = *reinterpret_cast<uint32_t *>(&h);
    }
};

// FP8 e4m3: 2 bytes per timepoint; values multiplied by the per-entry 1/scale.
template <>
struct Packer<MRF_FP8E4M3> {
    static constexpr int kBpt = 2;
    uint32_t hi[4], lo[4];
    __device__ __forceinline__ void put(int slot, float vr, float vi, float qs)
    {
        __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(make_float2(vr * qs, vi * qs), __NV_SATFINITE, __NV_E4M3);
        const int word = slot >> 1, half = slot & 1;
        if (half == 0) hi[word] = (uint32_t)q;
        else hi[word] |= ((uint32_t)q) << 16;
    }
};

// The F32 form's two e4m3 planes (the values, then the residuals; D x ld
// bytes each) for one 32-timepoint row chunk: lane piece qq < 4 writes 16
// bytes (8 timepoints) of the value plane, qq >= 4 of the residual plane,
// gathered from the two staged vectors that hold those timepoints (stage
// slots swizzled by r7, the row's index mod 8).
__device__ __forceinline__ void store_split_lo(uint8_t *out_lo, int64_t D, int ld, int64_t row, int j0, int qq,
                                               const uint4 *srow, int r7)
{
    const int sel = qq >> 2, p = qq & 3;
    const uint4 v0 = srow[(2 * p) ^ r7], v1 = srow[(2 * p + 1) ^ r7];
    const uint4 o = sel ? make_uint4(v0.z, v0.w, v1.z, v1.w) : make_uint4(v0.x, v0.y, v1.x, v1.y);
    __stcs(reinterpret_cast<uint4 *>(out_lo + (size_t)sel * D * ld + (size_t)row * ld + (size_t)j0 * 2 + p * 16), o);
}

template <int OUT, bool XONLY, bool SYM>
__global__ void __launch_bounds__(kGenThreads) dict_gen_kernel(SeqDev s, GridDev g, Tables t, int64_t D, int ld,
                                                               uint8_t *out_hi, uint8_t *out_lo, float *norm_out,
                                                               float *scale_out, int *err)
{
    using P = Packer<OUT>;
    constexpr int kBpt = P::kBpt;               // bytes per timepoint per array
    constexpr int kPerVec = 16 / kBpt;          // timepoints per 16-byte vector
    constexpr int kJ = 128 / kBpt;              // timepoints per 128-byte row chunk
    constexpr bool kTwo = (OUT == MRF_F32);

    __shared__ uint4 stage_hi[kGenThreads / 32][32][8];
    __shared__ uint4 stage_lo[kTwo ? kGenThreads / 32 : 1][32][8];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * kGenThreads + threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * kGenThreads + warp * 32;
    const bool live = e < D;
    const int n = s.n;
    int a = 0, b = 0, c = 0;
    if (live) unravel(g, e, a, b, c);
    const float fdf = live && s.finite ? __ldg(&g.df[c]) * 1.0e-3f : 0.f;   // finite pulses: RF depends on df
    const float e1inv = live && s.inversion ? __ldg(&t.e1_inv[a]) : 1.f;
    FacRows fr;
    if (SYM) {
        fr.e1 = t.e1s + (size_t)a * n;
        fr.e2 = t.e2s + (size_t)b * n;
        fr.z = t.ciss + c;
        fr.n_df = g.n_df;
    }

    // MRF_F32 stores the raw signal and the scale 1 / ||d||, so it needs a
    // single pass (the norm accumulates while the row is written); BF16 and
    // FP8 store normalised or scaled values and take the norm first.
    constexpr bool kOnePass = (OUT == MRF_F32);

    // pass 1: norm (blocked FP32 partial sums, Kahan-compensated total)
    float tot = 0.f, comp = 0.f, amax = 0.f;
    Bloch st;
    if (live && !kOnePass) {
        bloch_init(st);
        if (s.inversion) { bloch_invert(st); st.w *= e1inv; }
        if constexpr (SYM) {
            FacGroup cur, nxt;
            fac_load(cur, fr, 0);
            float part = 0.f;
            for (int j0 = 0; j0 < n; j0 += kFacG) {
                fac_load(nxt, fr, j0 + kFacG);
#pragma unroll
                for (int q = 0; q < kFacG; ++q) {
                    const int j = j0 + q;
                    if (j < n) {
                        float sr, si;
                        step_fac<XONLY>(st, s, cur, q, j, fdf, sr, si);
                        part = fmaf(sr, sr, fmaf(si, si, part));
                        if (OUT == MRF_FP8E4M3) amax = fmaxf(amax, fmaxf(fabsf(sr), fabsf(si)));
                    }
                }
                if ((j0 + kFacG) % 32 == 0 || j0 + kFacG >= n) {   // 32-timepoint blocks
                    const float y = part - comp;
                    const float tt = tot + y;
                    comp = (tt - tot) - y;
                    tot = tt;
                    part = 0.f;
                }
                cur = nxt;
            }
        } else {
            for (int j0 = 0; j0 < n; j0 += 32) {
                float part = 0.f;
                const int j1 = min(n, j0 + 32);
#pragma unroll 8
                for (int j = j0; j < j1; ++j) {
                    float sr, si;
                    step_tab<XONLY, SYM>(st, s, t, n, g.n_df, a, b, c, j, fdf, sr, si);
                    part = fmaf(sr, sr, fmaf(si, si, part));
                    if (OUT == MRF_FP8E4M3) amax = fmaxf(amax, fmaxf(fabsf(sr), fabsf(si)));
                }
                const float y = part - comp;
                const float tt = tot + y;
                comp = (tt - tot) - y;
                tot = tt;
            }
        }
    }
    float qs = 1.f;
    if (live && !kOnePass) {
        const float nrm = sqrtf(tot);
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
        norm_out[e] = nrm;
        if (OUT == MRF_FP8E4M3) {
            const float mx = amax * inv;                      // max |normalised component|
            const float scale = mx > 0.f ? mx / 448.0f : 1.0f;
            qs = inv / scale;                                 // raw value -> e4m3 code scale
            scale_out[e] = scale;
        } else {
            qs = inv;                                         // BF16: normalised values
            scale_out[e] = 1.0f;
        }
    }

    // pass 2: (re-)run and write the rows through the warp stage
    if (live) {
        bloch_init(st);
        if (s.inversion) { bloch_invert(st); st.w *= e1inv; }
    }
    const int row_bytes = ld * (OUT == MRF_FP8E4M3 ? 1 : 2);
    const int tp_row = row_bytes / kBpt;      // timepoint slots per row (incl. padding)
    FacGroup cur, nxt;
    if constexpr (SYM) fac_load(cur, fr, 0);
    float part1 = 0.f;                        // one-pass norm: this chunk's partial sum
    for (int j0 = 0; j0 < tp_row; j0 += kJ) {
        if constexpr (SYM) {
            // groups of kFacG timepoints: 8 / kPerVec vectors each
            constexpr int kVecs = kFacG / kPerVec;
#pragma unroll 1
            for (int gq = 0; gq < kJ / kFacG; ++gq) {
                const int jg = j0 + gq * kFacG;
                // the row's padding slots past n need no factors (and the
                // tables' padding covers only 2 x kFacG timepoints past n)
                if (jg + kFacG < n) fac_load(nxt, fr, jg + kFacG);
                float vr[kFacG], vi[kFacG];
#pragma unroll
                for (int q = 0; q < kFacG; ++q) {
                    const int j = jg + q;
                    vr[q] = 0.f;
                    vi[q] = 0.f;
                    if (live && j < n) {
                        step_fac<XONLY>(st, s, cur, q, j, fdf, vr[q], vi[q]);
                        if (kOnePass) part1 = fmaf(vr[q], vr[q], fmaf(vi[q], vi[q], part1));
                    }
                }
#pragma unroll
                for (int vq = 0; vq < kVecs; ++vq) {
                    P pk;
#pragma unroll
                    for (int u = 0; u < 4; ++u) { pk.hi[u] = 0u; pk.lo[u] = 0u; }
#pragma unroll
                    for (int u = 0; u < kPerVec; ++u) {
                        const float xr = vr[vq * kPerVec + u], xi = vi[vq * kPerVec + u];
                        pk.put(u, xr * (OUT == MRF_FP8E4M3 ? 1.f : qs), xi * (OUT == MRF_FP8E4M3 ? 1.f : qs),
                               OUT == MRF_FP8E4M3 ? qs : 1.f);
                    }
                    const int q = gq * kVecs + vq;
                    const int pq = q ^ (lane & 7);
                    stage_hi[warp][lane][pq] = make_uint4(pk.hi[0], pk.hi[1], pk.hi[2], pk.hi[3]);
                    if (kTwo) stage_lo[kTwo ? warp : 0][lane][pq] = make_uint4(pk.lo[0], pk.lo[1], pk.lo[2], pk.lo[3]);
                }
                cur = nxt;
            }
        } else {
#pragma unroll 2
            for (int q = 0; q < 8; ++q) {
                P pk;
#pragma unroll
                for (int u = 0; u < 4; ++u) { pk.hi[u] = 0u; pk.lo[u] = 0u; }
#pragma unroll
                for (int u = 0; u < kPerVec; ++u) {
                    const int j = j0 + q * kPerVec + u;
                    float vr = 0.f, vi = 0.f;
                    if (live && j < n) {
                        float sr, si;
                        step_tab<XONLY, SYM>(st, s, t, n, g.n_df, a, b, c, j, fdf, sr, si);
                        vr = sr;
                        vi = si;
                        if (kOnePass) part1 = fmaf(sr, sr, fmaf(si, si, part1));
                    }
                    pk.put(u, vr * (OUT == MRF_FP8E4M3 ? 1.f : qs), vi * (OUT == MRF_FP8E4M3 ? 1.f : qs),
                           OUT == MRF_FP8E4M3 ? qs : 1.f);
                }
                const int pq = q ^ (lane & 7);
                stage_hi[warp][lane][pq] = make_uint4(pk.hi[0], pk.hi[1], pk.hi[2], pk.hi[3]);
                if (kTwo) stage_lo[kTwo ? warp : 0][lane][pq] = make_uint4(pk.lo[0], pk.lo[1], pk.lo[2], pk.lo[3]);
            }
        }
        if (kOnePass) {   // 32-timepoint blocks (kJ = 32 for 4-byte timepoints)
            const float y = part1 - comp;
            const float tt = tot + y;
            comp = (tt - tot) - y;
            tot = tt;
            part1 = 0.f;
        }
        __syncwarp();
        const int qq = lane & 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i * 4 + (lane >> 3);
            const int64_t row = row0 + r;
            if (row < D && mrf_in_bounds((size_t)j0 * kBpt + qq * 16 + 16 <= (size_t)row_bytes, err)) {
                const size_t off = (size_t)row * row_bytes + (size_t)j0 * kBpt + qq * 16;
                const uint4 vh = stage_hi[warp][r][qq ^ (r & 7)];
                __stcs(reinterpret_cast<uint4 *>(out_hi + off), vh);
                if (kTwo) store_split_lo(out_lo, D, ld, row, j0, qq, stage_lo[kTwo ? warp : 0][r], r & 7);
            }
        }
        __syncwarp();
    }
    if (kOnePass && live) {
        const float nrm = sqrtf(tot);
        norm_out[e] = nrm;
        scale_out[e] = nrm > 0.f ? 1.0f / nrm : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Symmetric x-rotation sequences (every RF phase 0 or pi, TE_j = TR_j - TE_j:
// the randomised IR-bSSFP train of the experiments). Threads walk the grid
// df-major: thread t takes df index c = t / P and (T1, T2) pair p = t mod P
// (P = D / n_df valid pairs), i.e. entry p * n_df + c, so the lanes of a warp
// share c and e^{i theta_j} is one broadcast 16-byte load per two timepoints
// from a [c][j] table. E1 and E2 come from exp2f of TE_j, and the RF rotation
// and TE_j of each row chunk are staged per warp in shared memory (one
// coalesced load per chunk, fetched a chunk ahead). The recurrence and the
// evolution factors are those of the on-the-fly simulator (bloch_start,
// relax_factors), with E1 and E2 taken from the SFU's ex2 as in the ZOOM
// kernels.

// e^{i theta_j} of df index c over TE_j at zt[c * ldz + j]; ldz is a multiple of
// 8 with at least 8 slots past n (a look-ahead group reads past the end).
__global__ void ztable_kernel(SeqDev s, GridDev g, float2 *zt, int ldz)
{
    const int64_t n = s.n, total = n * g.n_df;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(k / n), j = (int)(k % n);
        const float f = g.df[c] * 1.0e-3f;
        float ta = f * s.tau[j].x;
        ta -= rintf(ta);
        float sa, ca;
        sincospif(2.0f * ta, &sa, &ca);
        zt[(size_t)c * ldz + j] = make_float2(ca, sa);
    }
}

struct ZGroup {
    float2 z[kFacG];
};

__device__ __forceinline__ void zgroup_load(ZGroup &f, const float2 *zrow, int jb)
{
    const float4 *p = reinterpret_cast<const float4 *>(zrow + jb);
#pragma unroll
    for (int k = 0; k < kFacG / 2; ++k) {
        const float4 v = __ldg(p + k);
        f.z[2 * k] = make_float2(v.x, v.y);
        f.z[2 * k + 1] = make_float2(v.z, v.w);
    }
}

// One timepoint: RF (c, s, 1 - c, TE_j), then E1 / E2 e^{i theta} over TE_j,
// the sample, and the same factors again over TR_j - TE_j = TE_j.
__device__ __forceinline__ void step_xsym(Bloch &st, float4 rf, float k1, float k2, float2 z, float &sr, float &si)
{
    bloch_rf_x(st, rf);
    const float e1 = ex2_fast(k1 * rf.w), e2 = ex2_fast(k2 * rf.w);
    const float zr = e2 * z.x, zi = e2 * z.y;
    bloch_evolve(st, e1, zr, zi);
    sr = st.mx;
    si = st.my;
    bloch_evolve(st, e1, zr, zi);
}

// RF of timepoints j0 + lane + 32 u (zero past n), one chunk of kJ timepoints.
template <int kJ>
__device__ __forceinline__ void rf_fetch(float4 (&r)[kJ / 32], const SeqDev &s, int j0, int lane)
{
#pragma unroll
    for (int u = 0; u < kJ / 32; ++u) {
        const int j = j0 + lane + 32 * u;
        r[u] = j < s.n ? __ldg(&s.rfx[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int OUT>
__global__ void __launch_bounds__(kGenThreads) dict_gen_xsym_kernel(SeqDev s, GridDev g, const float2 *zt, int ldz,
                                                                    int64_t D, int ld, uint8_t *out_hi,
                                                                    uint8_t *out_lo, float *norm_out, float *scale_out,
                                                                    int *err)
{
    using P = Packer<OUT>;
    constexpr int kBpt = P::kBpt;               // bytes per timepoint per array
    constexpr int kPerVec = 16 / kBpt;          // timepoints per 16-byte vector
    constexpr int kJ = 128 / kBpt;              // timepoints per 128-byte row chunk
    constexpr int kVecs = kFacG / kPerVec;      // 16-byte vectors per look-ahead group
    constexpr bool kTwo = (OUT == MRF_F32);
    constexpr bool kOnePass = (OUT == MRF_F32);
    static_assert(kJ % (2 * kFacG) == 0 && 32 % (2 * kFacG) == 0 && kVecs >= 1, "chunk / group mismatch");

    __shared__ uint4 stage_hi[kGenThreads / 32][32][8];
    __shared__ uint4 stage_lo[kTwo ? kGenThreads / 32 : 1][32][8];
    __shared__ float4 stage_rf[kGenThreads / 32][kJ];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tid = (int64_t)blockIdx.x * kGenThreads + threadIdx.x;
    const bool live = tid < D;
    const int n = s.n;
    const int64_t pairs = D / g.n_df;
    int64_t e = 0;
    int a = 0, b = 0, c = 0;
    if (live) {
        c = (int)(tid / pairs);
        e = (tid - (int64_t)c * pairs) * g.n_df + c;
        unravel(g, e, a, b, c);
    }
    // lanes past D run the recurrence of entry 0 and write nothing
    const Relax rx = relax_make(__ldg(&g.t1[a]), __ldg(&g.t2[b]), 0.f);
    const float2 *zrow = zt + (size_t)c * ldz;
    const float4 *srf = stage_rf[warp];
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // kFacG timepoints from jg on (FULL: all below n), with the next group's
    // e^{i theta} fetched into zn; the last look-ahead of a full chunk may
    // read up to 7 slots past n, inside the table's padding
    auto run_group = [&](auto full, Bloch &st, const ZGroup &zc, ZGroup &zn, int jg, int j0, float (&vr)[kFacG],
                         float (&vi)[kFacG]) {
        constexpr bool FULL = decltype(full)::value;
        if ((FULL || jg + kFacG < n) && mrf_in_bounds(jg + 2 * kFacG <= ldz && c < g.n_df, err))
            zgroup_load(zn, zrow, jg + kFacG);
#pragma unroll
        for (int q = 0; q < kFacG; ++q) {
            vr[q] = 0.f;
            vi[q] = 0.f;
            if (FULL || jg + q < n) step_xsym(st, srf[jg + q - j0], rx.k1, rx.k2, zc.z[q], vr[q], vi[q]);
        }
    };

    // pass 1 (BF16, FP8): ||d||^2 in 32-timepoint blocks (Kahan-compensated
    // total) and, for FP8, max |component|
    float tot = 0.f, comp = 0.f, amax = 0.f;
    Bloch st;
    if constexpr (!kOnePass) {
        bloch_start(st, s, rx);
        ZGroup za, zb;
        zgroup_load(za, zrow, 0);
        float4 rfn[1];
        rf_fetch<32>(rfn, s, 0, lane);
        for (int j0 = 0; j0 < n; j0 += 32) {
            stage_rf[warp][lane] = rfn[0];
            __syncwarp();
            rf_fetch<32>(rfn, s, j0 + 32, lane);
            float part = 0.f;
            auto acc = [&](const float (&vr)[kFacG], const float (&vi)[kFacG]) {
#pragma unroll
                for (int q = 0; q < kFacG; ++q) {
                    part = fmaf(vr[q], vr[q], fmaf(vi[q], vi[q], part));
                    if (OUT == MRF_FP8E4M3) amax = fmaxf(amax, fmaxf(fabsf(vr[q]), fabsf(vi[q])));
                }
            };
            float vr[kFacG], vi[kFacG];
            if (j0 + 32 <= n) {
#pragma unroll 1
                for (int jg = j0; jg < j0 + 32; jg += 2 * kFacG) {
                    run_group(std::true_type{}, st, za, zb, jg, j0, vr, vi);
                    acc(vr, vi);
                    run_group(std::true_type{}, st, zb, za, jg + kFacG, j0, vr, vi);
                    acc(vr, vi);
                }
            } else {
#pragma unroll 1
                for (int jg = j0; jg < j0 + 32; jg += 2 * kFacG) {
                    run_group(std::false_type{}, st, za, zb, jg, j0, vr, vi);
                    acc(vr, vi);
                    run_group(std::false_type{}, st, zb, za, jg + kFacG, j0, vr, vi);
                    acc(vr, vi);
                }
            }
            const float y = part - comp;
            const float tt = tot + y;
            comp = (tt - tot) - y;
            tot = tt;
            __syncwarp();
        }
    }
    float qs = 1.f;
    if (live && !kOnePass) {
        const float nrm = sqrtf(tot);
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
        norm_out[e] = nrm;
        if (OUT == MRF_FP8E4M3) {
            const float mx = amax * inv;                      // max |normalised component|
            const float scale = mx > 0.f ? mx / 448.0f : 1.0f;
            qs = inv / scale;                                 // raw value -> e4m3 code scale
            scale_out[e] = scale;
        } else {
            qs = inv;                                         // BF16: normalised values
            scale_out[e] = 1.0f;
        }
    }

    // pass 2: (re-)run and write the rows through the warp stage
    bloch_start(st, s, rx);
    const int row_bytes = ld * (OUT == MRF_FP8E4M3 ? 1 : 2);
    const int tp_row = row_bytes / kBpt;      // timepoint slots per row (incl. padding)
    const int erow = live ? (int)e : -1;      // dictionaries hold fewer than 2^31 entries
    ZGroup za, zb;
    zgroup_load(za, zrow, 0);
    float4 rfn[kJ / 32];
    rf_fetch<kJ>(rfn, s, 0, lane);
    float part1 = 0.f;                        // one-pass norm: this chunk's partial sum
    // pack one group into the stage (vectors gq * kVecs ...)
    auto put_group = [&](const float (&vr)[kFacG], const float (&vi)[kFacG], int gq) {
#pragma unroll
        for (int q = 0; q < kFacG; ++q)
            if (kOnePass) part1 = fmaf(vr[q], vr[q], fmaf(vi[q], vi[q], part1));
#pragma unroll
        for (int vq = 0; vq < kVecs; ++vq) {
            P pk;
#pragma unroll
            for (int u = 0; u < 4; ++u) { pk.hi[u] = 0u; pk.lo[u] = 0u; }
#pragma unroll
            for (int u = 0; u < kPerVec; ++u) {
                const float xr = vr[vq * kPerVec + u], xi = vi[vq * kPerVec + u];
                pk.put(u, xr * (OUT == MRF_FP8E4M3 ? 1.f : qs), xi * (OUT == MRF_FP8E4M3 ? 1.f : qs),
                       OUT == MRF_FP8E4M3 ? qs : 1.f);
            }
            const int pq = (gq * kVecs + vq) ^ (lane & 7);
            stage_hi[warp][lane][pq] = make_uint4(pk.hi[0], pk.hi[1], pk.hi[2], pk.hi[3]);
            if (kTwo) stage_lo[kTwo ? warp : 0][lane][pq] = make_uint4(pk.lo[0], pk.lo[1], pk.lo[2], pk.lo[3]);
        }
    };
    for (int j0 = 0; j0 < tp_row; j0 += kJ) {
#pragma unroll
        for (int u = 0; u < kJ / 32; ++u) stage_rf[warp][lane + 32 * u] = rfn[u];
        __syncwarp();
        rf_fetch<kJ>(rfn, s, j0 + kJ, lane);
        float vr[kFacG], vi[kFacG];
        if (j0 + kJ <= n) {
#pragma unroll 1
            for (int gq = 0; gq < kJ / kFacG; gq += 2) {
                run_group(std::true_type{}, st, za, zb, j0 + gq * kFacG, j0, vr, vi);
                put_group(vr, vi, gq);
                run_group(std::true_type{}, st, zb, za, j0 + (gq + 1) * kFacG, j0, vr, vi);
                put_group(vr, vi, gq + 1);
            }
        } else {
#pragma unroll 1
            for (int gq = 0; gq < kJ / kFacG; gq += 2) {
                run_group(std::false_type{}, st, za, zb, j0 + gq * kFacG, j0, vr, vi);
                put_group(vr, vi, gq);
                run_group(std::false_type{}, st, zb, za, j0 + (gq + 1) * kFacG, j0, vr, vi);
                put_group(vr, vi, gq + 1);
            }
        }
        if (kOnePass) {   // 32-timepoint blocks (kJ = 32 for 4-byte timepoints)
            const float y = part1 - comp;
            const float tt = tot + y;
            comp = (tt - tot) - y;
            tot = tt;
            part1 = 0.f;
        }
        __syncwarp();
        // the warp's rows are its lanes' entries (df-major order: not consecutive)
        const int qq = lane & 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i * 4 + (lane >> 3);
            const int row = __shfl_sync(0xffffffffu, erow, r);
            const size_t off = (size_t)row * row_bytes + (size_t)j0 * kBpt + qq * 16;
            if (row >= 0 && mrf_in_bounds(row < D && (size_t)j0 * kBpt + qq * 16 + 16 <= (size_t)row_bytes, err)) {
                const uint4 vh = stage_hi[warp][r][qq ^ (r & 7)];
                __stcs(reinterpret_cast<uint4 *>(out_hi + off), vh);
                if (kTwo) store_split_lo(out_lo, D, ld, row, j0, qq, stage_lo[kTwo ? warp : 0][r], r & 7);
            }
        }
        __syncwarp();
    }
    if (kOnePass && live) {
        const float nrm = sqrtf(tot);
        norm_out[e] = nrm;
        scale_out[e] = nrm > 0.f ? 1.0f / nrm : 0.f;
    }
}

// Arbitrary (T1, T2, df) per thread, complex64 rows of n timepoints, not normalised.
template <bool XONLY>
__global__ void __launch_bounds__(128) simulate_kernel(SeqDev s, int64_t count, const float *t1, const float *t2,
                                                       const float *df, float2 *out, int staged)
{
    __shared__ uint4 stage[4][32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * 128 + warp * 32;
    const bool live = e < count;
    const int n = s.n;
    Relax r = relax_make(live ? t1[e] : 1.f, live ? t2[e] : 1.f, live ? df[e] : 0.f);
    Bloch st;
    bloch_start(st, s, r);
    if (staged) {
        // staged (n even, out 16-byte aligned): 16 timepoints (128 bytes) per
        // row chunk, 2 per 16-byte vector
        for (int j0 = 0; j0 < n; j0 += 16) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = j0 + 2 * q + u;
                    if (live && j < n) bloch_step_otf<XONLY>(st, s, r, j, v[2 * u], v[2 * u + 1]);
                }
                stage[warp][lane][q ^ (lane & 7)] = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]),
                                                               __float_as_uint(v[2]), __float_as_uint(v[3]));
            }
            __syncwarp();
            const int qq = lane & 7;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = i * 4 + (lane >> 3);
                const int64_t row = row0 + rr;
                const int j = j0 + 2 * qq;
                if (row < count && j < n) {
                    const uint4 val = stage[warp][rr][qq ^ (rr & 7)];
                    *reinterpret_cast<uint4 *>(out + (size_t)row * n + j) = val;
                }
            }
            __syncwarp();
        }
    } else if (live) {
        for (int j = 0; j < n; ++j) {
            float sr, si;
            bloch_step_otf<XONLY>(st, s, r, j, sr, si);
            out[(size_t)e * n + j] = make_float2(sr, si);
        }
    }
}

}  // namespace

int launch_dict_generate(mrf_ctx *ctx, mrf_dict *d, cudaStream_t stream)
{
    const SeqDev s = d->seq->dev();
    const GridDev g = d->grid.dev();
    const int n = s.n;
    uint8_t *hi = (uint8_t *)d->hi, *lo = (uint8_t *)d->lo;
    const int64_t blocks = (d->entries + kGenThreads - 1) / kGenThreads;
    if (s.xonly && s.symmetric) {
        // df-major kernel: only the [c][j] e^{i theta} table
        const int ldz = ((n + 7) & ~7) + 8;
        const size_t zb = sizeof(float2) * (size_t)ldz * g.n_df;
        int rc = budget_charge(ctx, zb);
        if (rc) return rc;
        float2 *zt = nullptr;
        cudaError_t e = cudaMallocAsync((void **)&zt, zb, stream);
        if (e != cudaSuccess) { budget_release(ctx, zb); return cuda_fail(e, "table scratch"); }
        ztable_kernel<<<4 * ctx->sm_count, 256, 0, stream>>>(s, g, zt, ldz);
        count_launch(ctx);
        {
            ProfScope prof(ctx, kProfDictGen, stream);
#define MRF_XGEN(OUT) dict_gen_xsym_kernel<OUT><<<(unsigned)blocks, kGenThreads, 0, stream>>>(s, g, zt, ldz, d->entries, d->ld, hi, lo, d->norm, d->scale, ctx->err_flag)
            if (d->dtype == MRF_F32) MRF_XGEN(MRF_F32);
            else if (d->dtype == MRF_BF16) MRF_XGEN(MRF_BF16);
            else MRF_XGEN(MRF_FP8E4M3);
#undef MRF_XGEN
        }
        e = cudaGetLastError();
        cudaFreeAsync(zt, stream);
        budget_release(ctx, zb);
        if (e != cudaSuccess) return cuda_fail(e, "dictionary generation launch");
        return MRF_OK;
    }
    // evolution-factor tables in stream-ordered scratch
    // each table is followed by room for 2 x kFacG timepoints of padding (a
    // look-ahead group of the last entry reads past its end)
    const size_t b1 = sizeof(float2) * ((size_t)g.n_t1 * n + 2 * kFacG);
    const size_t b2 = sizeof(float2) * ((size_t)g.n_t2 * n + 2 * kFacG);
    const size_t b3 = sizeof(float4) * ((size_t)n + 2 * kFacG) * g.n_df, b4 = sizeof(float) * (size_t)g.n_t1;
    const size_t tb = b1 + b2 + b3 + b4 + 256 * 4;
    int rc = budget_charge(ctx, tb);
    if (rc) return rc;
    uint8_t *tab = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tab, tb, stream);
    if (e != cudaSuccess) { budget_release(ctx, tb); return cuda_fail(e, "table scratch"); }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    float2 *e1 = (float2 *)tab;
    float2 *e2 = (float2 *)(tab + al(b1));
    float4 *cis = (float4 *)(tab + al(b1) + al(b2));
    float *e1i = (float *)(tab + al(b1) + al(b2) + al(b3));
    tables_kernel<<<4 * ctx->sm_count, 256, 0, stream>>>(s, g, e1, e2, cis, e1i);
    count_launch(ctx);
    Tables t{e1, e2, cis, (const float *)e1, (const float *)e2, (const float2 *)cis, e1i};
#define MRF_GEN(OUT, XO, SY) dict_gen_kernel<OUT, XO, SY><<<(unsigned)blocks, kGenThreads, 0, stream>>>(s, g, t, d->entries, d->ld, hi, lo, d->norm, d->scale, ctx->err_flag)
#define MRF_GEN_DT(XO, SY)                                        \
    do {                                                          \
        if (d->dtype == MRF_F32) MRF_GEN(MRF_F32, XO, SY);        \
        else if (d->dtype == MRF_BF16) MRF_GEN(MRF_BF16, XO, SY); \
        else MRF_GEN(MRF_FP8E4M3, XO, SY);                        \
    } while (0)
    {
    ProfScope prof(ctx, kProfDictGen, stream);
    if (s.xonly) MRF_GEN_DT(true, false);
    else if (s.symmetric) MRF_GEN_DT(false, true);
    else MRF_GEN_DT(false, false);
    }
#undef MRF_GEN_DT
#undef MRF_GEN
    e = cudaGetLastError();
    cudaFreeAsync(tab, stream);
    budget_release(ctx, tb);
    if (e != cudaSuccess) return cuda_fail(e, "dictionary generation launch");
    return MRF_OK;
}

int launch_simulate(mrf_ctx *ctx, const mrf_seq *seq, int64_t count, const float *t1, const float *t2,
                    const float *df, void *out, cudaStream_t stream)
{
    count_launch(ctx);
    const SeqDev s = seq->dev();
    const int64_t blocks = (count + 127) / 128;
    const int staged = (s.n % 2 == 0) && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    if (s.xonly) simulate_kernel<true><<<(unsigned)blocks, 128, 0, stream>>>(s, count, t1, t2, df, (float2 *)out, staged);
    else simulate_kernel<false><<<(unsigned)blocks, 128, 0, stream>>>(s, count, t1, t2, df, (float2 *)out, staged);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "simulate launch");
    return MRF_OK;
}
