// Brute-force DGS matcher (Theory: argmax of Eq. 1 over every grid entry).
//
// With unit-norm voxels x and entries d, CC(x, d) = |sum_j x_j conj(d_j)|.
// Writing each voxel as two real rows of length 2n over interleaved (re, im)
// timepoints,
//     row 2v   = ( xr_0,  xi_0,  xr_1,  xi_1, ...)
//     row 2v+1 = ( xi_0, -xr_0,  xi_1, -xr_1, ...)
// and each entry as (dr_0, di_0, dr_1, di_1, ...), the product of the 2V x 2n
// voxel matrix with the n-row-major dictionary gives Re <x, d> in row 2v and
// Im <x, d> in row 2v+1: the complex correlation is one real GEMM whose 2 x 2
// blocks are the complex products.
//
// The GEMM runs on the 5th-generation tensor cores: 128 voxel rows (64
// voxels) x 256 entries per tile, fp32 accumulators in TMEM (two 256-column
// buffers), operand tiles staged by TMA with 128-byte swizzle. A persistent
// warp-specialised CTA per SM: warp 0 issues TMA, warp 1 issues tcgen05.mma,
// warps 2-5 read the accumulators (tcgen05.ld), form CC^2 = Re^2 + Im^2 and
// keep each voxel's running top-k in registers. The V x D score matrix never
// leaves the SM; each (voxel block, dictionary chunk) work unit writes only
// its top-k, merged across chunks afterwards.
//
// Precisions: MRF_F32 = the split form of split.cuh over raw entries: an
// fp16 product and two e4m3 products of the fp16 residuals (per term at most
// about 2^-13, rms about 2^-16 relative), the e4m3 ones accumulated first,
// the entry's scale 1 / ||d|| applied to CC^2 (generated tiles: the bf16
// hi/lo split, hi.hi + hi.lo + lo.hi); MRF_BF16 = one bf16 product of
// unit-norm entries; MRF_FP8E4M3 = one e4m3 product (kind::f8f6f4) with
// per-entry and per-voxel scales applied to CC^2.
//
// Re-score (Discussion: normalised-CC errors fixed by a non-normalised final
// comparison): each voxel's candidates are re-simulated in FP32 and their CC
// taken with FP64 accumulation; the best (ties to the smaller index) wins.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "bloch.cuh"
#include "mrf_internal.h"
#include "split.cuh"
#include "tc.cuh"

namespace {

constexpr int BM = 128;          // voxel rows per tile (64 voxels)
constexpr int BN = 256;          // dictionary entries per tile
constexpr uint64_t kWaitLimitNs = 4000000000ull;   // 4 s per barrier wait

// Kernel form of MRF_F32 over a stored dictionary (the split form of
// split.cuh); MRF_F32 itself is the form of generated tiles (bf16 hi / lo).
constexpr int kModeSplit = 3;

template <int MODE>
struct Cfg;
// MRF_F32, generated tiles: hi and lo of both operands, one voxel block per CTA
template <>
struct Cfg<MRF_F32> {
    static constexpr int kBK = 64, kStages = 2, kOps = 2, kNB = 1;
};
// split form: two voxel blocks per CTA share each dictionary tile, as BF16;
// a stage holds one operand plane of 128 bytes per row (e4m3 residual or
// value plane, or one fp16 K block)
template <>
struct Cfg<kModeSplit> {
    static constexpr int kBK = 64, kStages = 3, kOps = 1, kNB = 2;
};
// BF16 / FP8: two voxel blocks per CTA share each dictionary tile (two
// accumulators), which halves the dictionary bytes per flop through L2
template <>
struct Cfg<MRF_BF16> {
    static constexpr int kBK = 64, kStages = 3, kOps = 1, kNB = 2;
};
template <>
struct Cfg<MRF_FP8E4M3> {
    static constexpr int kBK = 128, kStages = 3, kOps = 1, kNB = 2;
};

constexpr int kTileA = BM * 128;   // bytes of one A operand tile (128 rows x 128 B)
constexpr int kTileB = BN * 128;   // bytes of one B operand tile (256 rows x 128 B)

template <int MODE>
constexpr int stage_bytes() { return Cfg<MODE>::kOps * (Cfg<MODE>::kNB * kTileA + kTileB); }
template <int MODE>
constexpr int smem_bytes() { return Cfg<MODE>::kStages * stage_bytes<MODE>() + 1024; }
// Generated dictionary tiles (mrf_match_bruteforce_fused): kSimWarps warps
// simulate each tile's entries into the B stages, two entries per thread.
constexpr int kSimWarps = 4;
template <int MODE, bool GEN = false>
constexpr int threads_of() { return 64 + 128 * Cfg<MODE>::kNB + (GEN ? 32 * kSimWarps : 0); }

struct MatchParams {
    int64_t D;           // dictionary entries
    int64_t V;           // voxels
    int n_tiles;         // ceil(D / BN)
    int n_vu;            // voxel units (kNB voxel blocks of 64 voxels each)
    int n_chunks;        // dictionary chunks per voxel unit
    int group_vu;        // voxel units per group: a group's voxel operands stay in L2
                         // while the dictionary streams past them once
    int k_blocks;        // K blocks of 128 bytes
    int last_ksteps;     // MMA k-steps in the last K block (rest is zero padding)
    int k_blocks16;      // split form: fp16 K blocks of 64 elements (k_blocks: e4m3 blocks of 128)
    int last_ks16;       // split form: k-steps in the last fp16 K block
    const float *colscale;   // per-entry scale (stored value x scale = unit-norm entry), nullptr when 1
    int col_stride;      // dictionary entry of tile column c is c * col_stride (sampled pre-pass)
    const float *thr0;   // per-voxel lower bound on the K-th best CC^2 (thr0[v * thr0_stride]), or nullptr
    int thr0_stride;
    float *thr_live;     // per-voxel bound shared by the CTAs of one pass (atomic max of their K-th bests), or nullptr
    float2 *part;        // [V][n_chunks][K]: (cc2, idx bits)
    int *err;
    // generated tiles (GEN): the entries' sequence and grid, timepoints
    SeqDev s;
    GridDev g;
    int n;
};

// order: higher cc2 first, then smaller index
__device__ __forceinline__ bool before(float c, int i, float oc, int oi)
{
    return c > oc || (c == oc && i < oi);
}

// Sorted (descending) top-K list in registers. Insertion computes the slot
// with K independent comparisons and shifts with selects (no serial chain).
template <int K>
struct TopK {
    float v[K];
    int i[K];
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int q = 0; q < K; ++q) { v[q] = -1.0f; i[q] = 0x7fffffff; }
    }
    __device__ __forceinline__ void insert(float c, int idx)
    {
        int pos = 0;
#pragma unroll
        for (int q = 0; q < K; ++q) pos += before(v[q], i[q], c, idx) ? 1 : 0;
        if (pos >= K) return;
#pragma unroll
        for (int q = K - 1; q > 0; --q) {
            const bool sh = q > pos, here = q == pos;
            v[q] = sh ? v[q - 1] : (here ? c : v[q]);
            i[q] = sh ? i[q - 1] : (here ? idx : i[q]);
        }
        if (pos == 0) { v[0] = c; i[0] = idx; }
    }
};

// Work unit u -> (dictionary chunk, voxel unit). Units run group by group;
// inside a group chunk-major, so concurrent CTAs share dictionary tiles.
__device__ __forceinline__ void decode_unit(const MatchParams &p, int u, int &chunk, int &vu)
{
    const int per_group = p.group_vu * p.n_chunks;
    const int n_groups = (p.n_vu + p.group_vu - 1) / p.group_vu;
    const int g = min(u / per_group, n_groups - 1);
    const int r = u - g * per_group;
    const int gsize = (g == n_groups - 1) ? p.n_vu - g * p.group_vu : p.group_vu;
    chunk = r / gsize;
    vu = g * p.group_vu + r % gsize;
}

__device__ __forceinline__ float sel16(const float (&a)[16], int q)
{
    float r = a[0];
#pragma unroll
    for (int k = 1; k < 16; ++k) r = (q == k) ? a[k] : r;
    return r;
}

// Linear entry index -> grid indices (a, b, c): binary search over the T1 offsets.
__device__ __forceinline__ void unravel_dev(const GridDev &g, int64_t e, int &a, int &b, int &c)
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

// GEN: the dictionary is not read but generated. kSimWarps simulation warps
// run each tile's entries through the Bloch recurrence (FP32, factors on the
// fly) and write the raw entries, 32 timepoints per K block, as bf16 (hi, and
// lo for MRF_F32) straight into the B stages in the 128-byte-swizzled K-major
// layout TMA would produce; each entry's 1 / ||d|| becomes its column scale.
// The voxel operands still arrive by TMA. No dictionary reaches HBM.
template <int MODE, int K, bool GEN>
__global__ void __launch_bounds__(threads_of<MODE, GEN>(), 1)
    match_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapA2,
                 const __grid_constant__ CUtensorMap mapA3, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ CUtensorMap mapB2, const __grid_constant__ CUtensorMap mapB3, MatchParams p)
{
    using C = Cfg<MODE>;
    // Split form (MRF_F32 over a stored dictionary): per tile, first 2
    // p.k_blocks e4m3 stages, for each 128-element K block the pair (x
    // residuals with d values, x values with d residuals), then p.k_blocks16
    // fp16 stages of 64 elements; every stage holds both voxel blocks' A
    // tiles and one B tile.
    constexpr bool kSplit = MODE == kModeSplit;
    static_assert(!kSplit || !GEN, "generated tiles use the bf16 hi / lo split");
    constexpr uint32_t kIdescF16 = make_idesc(0, 0, BM, BN);   // kind::f16 with fp16 operands
    constexpr uint32_t kIdescE4 = make_idesc(0, 0, BM, BN);    // kind::f8f6f4 with e4m3 operands
    // squared column scales carry the split form's 2^-54 (2^-27 per operand side; exact)
    constexpr float kColMul2 = kSplit ? kSplitUnscale * kSplitUnscale : 1.0f;
    constexpr int S = C::kStages;
    constexpr int NB = C::kNB;                  // voxel blocks per CTA
    constexpr int NBUF = NB == 1 ? 2 : 1;       // accumulator buffers (TMEM holds 512 columns)
    constexpr int NEPI = 4 * NB;                // epilogue warps
    constexpr uint32_t kStageBytes = stage_bytes<MODE>();
    // bytes TMA brings into a stage (GEN: the voxel operands only)
    constexpr uint32_t kTmaBytes = GEN ? (uint32_t)(C::kOps * NB * kTileA) : kStageBytes;
    constexpr uint32_t kIdesc = MODE == MRF_FP8E4M3 ? make_idesc(0, 0, BM, BN) : make_idesc(1, 1, BM, BN);
    constexpr bool kScaled = MODE != MRF_BF16 || GEN;   // columns carry a scale (stored x scale = unit norm)
    static_assert(!GEN || MODE != MRF_FP8E4M3, "generated tiles are bf16 (hi, lo)");

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], tfull_bar[NBUF], tempty_bar[NBUF], drain_bar;
    __shared__ __align__(8) uint64_t scale_bar[GEN ? NBUF : 1];   // GEN: a tile's column scales are written
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    // per epilogue warp: the column scales of its current tile, fetched while
    // the tile's MMAs run (GEN: written by the simulation warps, per accumulator buffer)
    __shared__ __align__(16) float sc_tile[GEN ? 1 : NEPI][kScaled && !GEN ? BN : 1];
    __shared__ __align__(16) float sc_gen[GEN ? NBUF : 1][GEN ? BN : 1];
    // GEN: per simulation warp, the sequence coefficients of the current K block's 32
    // timepoints (RF rotation: rfx, or the general matrix in 3 float4, or the finite-
    // pulse parameters; TE_j and TR_j - TE_j), staged once per K block
    __shared__ __align__(16) float4 sim_rf[GEN ? kSimWarps : 1][GEN ? 3 * 32 : 1];
    __shared__ __align__(16) float2 sim_tau[GEN ? kSimWarps : 1][GEN ? 32 : 1];

    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // stage s: [A(block 0..NB-1, hi) | A lo? | B hi | B lo?]
    auto tileA = [&](int s, int op, int i) { return smem + s * kStageBytes + (op * NB + i) * kTileA; };
    auto tileB = [&](int s, int op) { return smem + s * kStageBytes + C::kOps * NB * kTileA + op * kTileB; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // GEN: a stage is full once TMA's bytes and every simulation warp have arrived
        for (int q = 0; q < S; ++q) { mbar_init(&full_bar[q], GEN ? 1 + kSimWarps : 1); mbar_init(&empty_bar[q], 1); }
        for (int a = 0; a < NBUF; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], NEPI); }
        if (GEN)
            for (int a = 0; a < NBUF; ++a) mbar_init(&scale_bar[a], kSimWarps);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&mapA);
        if (!GEN) tma_prefetch_desc(&mapB);
        if (C::kOps == 2) {
            tma_prefetch_desc(&mapA2);
            if (!GEN) tma_prefetch_desc(&mapB2);
        }
        if (kSplit) {
            tma_prefetch_desc(&mapA2);
            tma_prefetch_desc(&mapA3);
            tma_prefetch_desc(&mapB2);
            tma_prefetch_desc(&mapB3);
        }
    }
    if (warp == 1) {
        tmem_alloc(&tmem_slot, 2 * BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_slot;

    const int n_units = p.n_vu * p.n_chunks;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            // voxel operands are re-read for every dictionary tile: keep them in L2
            const uint64_t keep = l2_policy_keep();
            int s = 0;
            uint32_t ph = 0;
            bool issued[S];
            uint32_t issued_ph[S];
            for (int q = 0; q < S; ++q) { issued[q] = false; issued_ph[q] = 0; }
            for (int u = blockIdx.x; u < n_units && !abort_flag; u += gridDim.x) {
                int chunk, vu;
                decode_unit(p, u, chunk, vu);
                const int t0 = (int)((int64_t)chunk * p.n_tiles / p.n_chunks);
                const int t1 = (int)((int64_t)(chunk + 1) * p.n_tiles / p.n_chunks);
                for (int t = t0; t < t1; ++t) {
                    const int n_st = kSplit ? 2 * p.k_blocks + p.k_blocks16 : p.k_blocks;
                    for (int kb = 0; kb < n_st; ++kb) {
                        if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kWaitLimitNs)) goto producer_done;
                        mbar_arrive_expect_tx(&full_bar[s], kTmaBytes);
                        if (kSplit) {
                            // e4m3 stages: x residuals with d values (even), x values with
                            // d residuals (odd), 128 elements; then fp16 blocks of 64
                            const bool e4 = kb < 2 * p.k_blocks;
                            const int kx = e4 ? (kb >> 1) * 128 : (kb - 2 * p.k_blocks) * 64;
                            const CUtensorMap *ma = e4 ? ((kb & 1) ? &mapA3 : &mapA2) : &mapA;
                            const CUtensorMap *mb = e4 ? ((kb & 1) ? &mapB3 : &mapB2) : &mapB;
#pragma unroll
                            for (int i = 0; i < NB; ++i)
                                tma_load_2d_hint(tileA(s, 0, i), ma, &full_bar[s], kx, (vu * NB + i) * BM, keep);
                            tma_load_2d(tileB(s, 0), mb, &full_bar[s], kx, t * BN);
                            issued[s] = true;
                            issued_ph[s] = ph;
                            if (++s == S) { s = 0; ph ^= 1; }
                            continue;
                        }
                        const int kx = kb * C::kBK;
#pragma unroll
                        for (int i = 0; i < NB; ++i) {
                            const int row = (vu * NB + i) * BM;
                            tma_load_2d_hint(tileA(s, 0, i), &mapA, &full_bar[s], kx, row, keep);
                            if (C::kOps == 2) tma_load_2d_hint(tileA(s, 1, i), &mapA2, &full_bar[s], kx, row, keep);
                        }
                        if (!GEN) {
                            tma_load_2d(tileB(s, 0), &mapB, &full_bar[s], kx, t * BN);
                            if (C::kOps == 2) tma_load_2d(tileB(s, 1), &mapB2, &full_bar[s], kx, t * BN);
                        }
                        issued[s] = true;
                        issued_ph[s] = ph;
                        if (++s == S) { s = 0; ph ^= 1; }
                    }
                }
            }
        producer_done:
            // every load issued into shared memory must land before the CTA exits
            for (int q = 0; q < S; ++q) {
                if (!issued[q]) continue;
                const uint64_t t0 = global_timer_ns();
                while (!mbar_try_wait(&full_bar[q], issued_ph[q])) {
                    if (global_timer_ns() - t0 > kWaitLimitNs) { atomicExch(p.err, 1); break; }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int s = 0, buf = 0;
            uint32_t ph = 0, buf_ph = 0;
            bool any = false;
            for (int u = blockIdx.x; u < n_units && !abort_flag; u += gridDim.x) {
                int chunk, vu;
                decode_unit(p, u, chunk, vu);
                (void)vu;
                const int t0 = (int)((int64_t)chunk * p.n_tiles / p.n_chunks);
                const int t1 = (int)((int64_t)(chunk + 1) * p.n_tiles / p.n_chunks);
                for (int t = t0; t < t1; ++t) {
                    if (!mbar_wait_bounded(&tempty_bar[buf], buf_ph ^ 1, &abort_flag, p.err, kWaitLimitNs)) goto mma_done;
                    tc_fence_after();
                    const int n_st = kSplit ? 2 * p.k_blocks + p.k_blocks16 : p.k_blocks;
                    for (int kb = 0; kb < n_st; ++kb) {
                        if (!mbar_wait_bounded(&full_bar[s], ph, &abort_flag, p.err, kWaitLimitNs)) goto mma_done;
                        tc_fence_after();
                        if (kSplit) {
                            // the e4m3 products of the whole K range first, then the fp16 product
                            const bool e4 = kb < 2 * p.k_blocks;
                            const int nk = e4 ? ((kb >> 1) == p.k_blocks - 1 ? p.last_ksteps : 4)
                                              : (kb == n_st - 1 ? p.last_ks16 : 4);
                            const uint64_t b0 = smem_desc_sw128(tileB(s, 0));
                            // one loop per instruction kind (32 bytes of K per MMA in both)
                            if (e4) {
                                for (int kk = 0; kk < nk; ++kk) {
                                    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                                    const uint32_t accum = (kb | kk) != 0;
#pragma unroll
                                    for (int i = 0; i < NB; ++i)
                                        mma_f8(tmem_base + (uint32_t)((buf * NB + i) * BN),
                                               smem_desc_sw128(tileA(s, 0, i)) + adv, b0 + adv, kIdescE4, accum);
                                }
                            } else {
                                for (int kk = 0; kk < nk; ++kk) {
                                    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
#pragma unroll
                                    for (int i = 0; i < NB; ++i)
                                        mma_f16(tmem_base + (uint32_t)((buf * NB + i) * BN),
                                                smem_desc_sw128(tileA(s, 0, i)) + adv, b0 + adv, kIdescF16, 1u);
                                }
                            }
                            mma_commit(&empty_bar[s]);
                            any = true;
                            if (++s == S) { s = 0; ph ^= 1; }
                            continue;
                        }
                        const uint64_t b0 = smem_desc_sw128(tileB(s, 0));
                        const int nk = (kb == p.k_blocks - 1) ? p.last_ksteps : 4;
                        for (int kk = 0; kk < nk; ++kk) {
                            // advance 32 bytes along K inside the swizzled 128-byte rows
                            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                            const uint32_t accum = (kb | kk) != 0;
#pragma unroll
                            for (int i = 0; i < NB; ++i) {
                                const uint32_t d_tmem = tmem_base + (uint32_t)((buf * NB + i) * BN);
                                const uint64_t a0 = smem_desc_sw128(tileA(s, 0, i));
                                if (MODE == MRF_FP8E4M3) {
                                    mma_f8(d_tmem, a0 + adv, b0 + adv, kIdesc, accum);
                                } else {
                                    mma_f16(d_tmem, a0 + adv, b0 + adv, kIdesc, accum);
                                    if (MODE == MRF_F32) {
                                        const uint64_t a1 = smem_desc_sw128(tileA(s, 1, i));
                                        const uint64_t b1 = smem_desc_sw128(tileB(s, 1));
                                        mma_f16(d_tmem, a0 + adv, b1 + adv, kIdesc, 1u);
                                        mma_f16(d_tmem, a1 + adv, b0 + adv, kIdesc, 1u);
                                    }
                                }
                            }
                        }
                        mma_commit(&empty_bar[s]);   // frees the stage when these MMAs finish
                        any = true;
                        if (++s == S) { s = 0; ph ^= 1; }
                    }
                    mma_commit(&tfull_bar[buf]);     // accumulators ready for the epilogue
                    if (++buf == NBUF) { buf = 0; buf_ph ^= 1; }
                }
            }
        mma_done:
            if (any) {
                // all issued MMAs must finish before TMEM is released
                mma_commit(&drain_bar);
                const uint64_t t0 = global_timer_ns();
                while (!mbar_try_wait(&drain_bar, 0)) {
                    if (global_timer_ns() - t0 > kWaitLimitNs) { atomicExch(p.err, 1); break; }
                }
            }
        }
    } else if (GEN && warp >= 2 + NEPI) {
        // ---------------- simulation: generated B tiles ----------------
        // thread r simulates rows r and r + 128 of each tile (entries t * BN + row)
        const int r0 = threadIdx.x - 32 * (2 + NEPI);
        const int wsim = warp - (2 + NEPI);
        const int n = p.n;
        // one timepoint jj of the staged K block; evolution factors from the SFU
        // (the candidates are ranked here and re-scored exactly afterwards)
        auto sim_step = [&](Bloch &bs, const Relax &rr, int jj, float &sr, float &si) {
            if (p.s.xonly) {
                bloch_rf_x(bs, sim_rf[wsim][jj]);
            } else if (p.s.finite) {
                bloch_rf_finite(bs, sim_rf[wsim][jj], rr.f);
            } else {
                const float4 a4 = sim_rf[wsim][3 * jj], b4 = sim_rf[wsim][3 * jj + 1], c4 = sim_rf[wsim][3 * jj + 2];
                const float qm[10] = {a4.x, a4.y, a4.z, a4.w, b4.x, b4.y, b4.z, b4.w, c4.x, c4.y};
                bloch_rf_general(bs, qm);
            }
            const float2 tau = sim_tau[wsim][jj];
            float cs, sn;
            cis_sfu(rr.f, tau.x, cs, sn);
            float e1 = ex2_fast(rr.k1 * tau.x), e2 = ex2_fast(rr.k2 * tau.x);
            bloch_evolve(bs, e1, e2 * cs, e2 * sn);
            sr = bs.mx;
            si = bs.my;
            if (!p.s.symmetric) {
                cis_sfu(rr.f, tau.y, cs, sn);
                e1 = ex2_fast(rr.k1 * tau.y);
                e2 = ex2_fast(rr.k2 * tau.y);
            }
            bloch_evolve(bs, e1, e2 * cs, e2 * sn);
        };
        int s = 0, buf = 0;
        uint32_t ph = 0, buf_ph = 0;
        for (int u = blockIdx.x; u < n_units && !abort_flag; u += gridDim.x) {
            int chunk, vu;
            decode_unit(p, u, chunk, vu);
            (void)vu;
            const int t0 = (int)((int64_t)chunk * p.n_tiles / p.n_chunks);
            const int t1 = (int)((int64_t)(chunk + 1) * p.n_tiles / p.n_chunks);
            for (int t = t0; t < t1; ++t) {
                Bloch st[2];
                Relax rx[2];
                bool live[2];
                float tot[2], comp[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t e = (int64_t)t * BN + r0 + 128 * h;
                    live[h] = e < p.D;
                    int a = 0, b = 0, c = 0;
                    if (live[h]) unravel_dev(p.g, e, a, b, c);
                    rx[h] = relax_make(live[h] ? __ldg(&p.g.t1[a]) : 1000.f, live[h] ? __ldg(&p.g.t2[b]) : 100.f,
                                       live[h] ? __ldg(&p.g.df[c]) : 0.f);
                    bloch_start(st[h], p.s, rx[h]);
                    tot[h] = 0.f;
                    comp[h] = 0.f;
                }
                for (int kb = 0; kb < p.k_blocks; ++kb) {
                    // this K block's sequence coefficients, fetched before waiting for the stage
                    __syncwarp();
                    {
                        const int jl = kb * 32 + lane;
                        if (jl < n) {
                            if (p.s.xonly) {
                                sim_rf[wsim][lane] = __ldg(&p.s.rfx[jl]);
                            } else if (p.s.finite) {
                                sim_rf[wsim][lane] = __ldg(&p.s.rff[jl]);
                            } else {
                                const float4 *gq = reinterpret_cast<const float4 *>(p.s.rfg + 12 * (size_t)jl);
                                sim_rf[wsim][3 * lane] = __ldg(gq);
                                sim_rf[wsim][3 * lane + 1] = __ldg(gq + 1);
                                sim_rf[wsim][3 * lane + 2] = __ldg(gq + 2);
                            }
                            sim_tau[wsim][lane] = __ldg(&p.s.tau[jl]);
                        }
                    }
                    __syncwarp();   // the staged coefficients are visible to every lane of the warp
                    const bool ok = mbar_wait_bounded(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kWaitLimitNs);
                    if (!__all_sync(0xffffffffu, ok)) goto sim_done;   // leave as a whole warp
                    // the two entries interleaved (independent recurrences)
                    float part[2] = {0.f, 0.f};
#pragma unroll 1
                    for (int q = 0; q < 8; ++q) {
                        uint32_t hi4[2][4], lo4[2][4];
#pragma unroll
                        for (int u4 = 0; u4 < 4; ++u4) {
                            const int j = kb * 32 + q * 4 + u4;
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float sr = 0.f, si = 0.f;
                                if (live[h] && j < n) {
                                    sim_step(st[h], rx[h], q * 4 + u4, sr, si);
                                    part[h] = fmaf(sr, sr, fmaf(si, si, part[h]));
                                }
                                const __nv_bfloat162 hv = __floats2bfloat162_rn(sr, si);
                                const float2 hf = __bfloat1622float2(hv);
                                const __nv_bfloat162 lv = __floats2bfloat162_rn(sr - hf.x, si - hf.y);
                                hi4[h][u4] = *reinterpret_cast<const uint32_t *>(&hv);
                                lo4[h][u4] = *reinterpret_cast<const uint32_t *>(&lv);
                            }
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // 16-byte chunk q of the row, 128-byte swizzle (chunk index ^ row % 8)
                            const int row = r0 + 128 * h;
                            const int pq = q ^ (row & 7);
                            *reinterpret_cast<uint4 *>(tileB(s, 0) + row * 128 + pq * 16) =
                                make_uint4(hi4[h][0], hi4[h][1], hi4[h][2], hi4[h][3]);
                            if (C::kOps == 2)
                                *reinterpret_cast<uint4 *>(tileB(s, C::kOps - 1) + row * 128 + pq * 16) =
                                    make_uint4(lo4[h][0], lo4[h][1], lo4[h][2], lo4[h][3]);
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // the norm: 32-timepoint FP32 blocks, compensated total
                        const float y = part[h] - comp[h];
                        const float tt = tot[h] + y;
                        comp[h] = (tt - tot[h]) - y;
                        tot[h] = tt;
                    }
                    // the generic-proxy stores must be visible to the tensor core's reads
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full_bar[s]);
                    if (++s == S) { s = 0; ph ^= 1; }
                }
                // the tile's column scales, once the epilogue is done with this buffer's previous ones
                const bool ok = mbar_wait_bounded(&tempty_bar[buf], buf_ph ^ 1, &abort_flag, p.err, kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) goto sim_done;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // the squared column scale (1 / ||d||)^2, as the epilogue applies it
                    const float sc = (live[h] && tot[h] > 0.f) ? rsqrtf(tot[h]) : 0.f;
                    sc_gen[GEN ? buf : 0][GEN ? r0 + 128 * h : 0] = sc * sc;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&scale_bar[GEN ? buf : 0]);
                if (++buf == NBUF) { buf = 0; buf_ph ^= 1; }
            }
        }
    sim_done:;
    } else {
        // ---------------- epilogue: TMEM -> CC^2 -> running top-k ----------------
        const int blk = (warp - 2) / 4;            // which voxel block of the unit
        const int quad = warp & 3;                 // TMEM lane quadrant this warp may access
        const int row = quad * 32 + lane;          // voxel row within the tile
        const int par = row & 1;                   // 0: Re row, 1: Im row
        int buf = 0;
        uint32_t buf_ph = 0;
        TopK<K> tk;
        for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
            if (__any_sync(0xffffffffu, abort_flag != 0)) break;
            int chunk, vu;
            decode_unit(p, u, chunk, vu);
            const int t0 = (int)((int64_t)chunk * p.n_tiles / p.n_chunks);
            const int t1 = (int)((int64_t)(chunk + 1) * p.n_tiles / p.n_chunks);
            tk.reset();
            // Values below a lower bound on the voxel's K-th best CC^2 over the
            // whole dictionary (the K-th best of a subset of it, slightly
            // lowered for rounding) cannot be among its K best: they are
            // filtered before the list ever sees them.
            float seed = -1.0f;
            if (p.thr0) {
                const int64_t vs = (int64_t)(vu * NB + blk) * (BM / 2) + (row >> 1);
                const float lb = vs < p.V ? __ldg(&p.thr0[vs * p.thr0_stride]) : -1.0f;
                if (lb > 0.f) seed = lb * (1.0f - 1.0e-6f);
            }
            float thr = seed;                      // current K-th best (or the bound)
            const int64_t vrow = (int64_t)(vu * NB + blk) * (BM / 2) + (row >> 1);
            const bool vlive = vrow < p.V;
            for (int t = t0; t < t1; ++t) {
                if (kScaled && !GEN) {
                    float *sct = sc_tile[GEN ? 0 : warp - 2];
                    for (int q = lane; q < BN; q += 32) {
                        const int col = t * BN + q;
                        const float sc = col < p.D ? __ldg(&p.colscale[(int64_t)col * p.col_stride]) : 0.f;
                        sct[q] = sc * sc * kColMul2;   // squared, as the epilogue applies it
                    }
                    __syncwarp();
                }
                bool ok = mbar_wait_bounded(&tfull_bar[buf], buf_ph, &abort_flag, p.err, kWaitLimitNs);
                if (GEN && ok) ok = mbar_wait_bounded(&scale_bar[GEN ? buf : 0], buf_ph, &abort_flag, p.err, kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) goto epi_done;   // leave as a whole warp
                tc_fence_after();
                const uint32_t tbase =
                    tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)((buf * NB + blk) * BN);
#pragma unroll 1
                for (int ch = 0; ch < BN / 32; ++ch) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tbase + ch * 32, r);
                    tmem_wait_ld();
                    const int col0 = t * BN + ch * 32 + (par ? 16 : 0);
                    float c2v[16];
                    float sc16[16];
                    if (kScaled) {
                        const float *scs = GEN ? &sc_gen[GEN ? buf : 0][GEN ? ch * 32 + (par ? 16 : 0) : 0]
                                               : &sc_tile[GEN ? 0 : warp - 2][GEN ? 0 : ch * 32 + (par ? 16 : 0)];
                        const float4 *s4 = reinterpret_cast<const float4 *>(scs);
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const float4 f = s4[q4];
                            sc16[4 * q4] = f.x; sc16[4 * q4 + 1] = f.y; sc16[4 * q4 + 2] = f.z; sc16[4 * q4 + 3] = f.w;
                        }
                    }
                    uint32_t mask = 0;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float mine_lo = __uint_as_float(r[q]);
                        const float mine_hi = __uint_as_float(r[16 + q]);
                        const float send = par ? mine_lo : mine_hi;
                        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                        const float re = par ? recv : mine_lo;
                        const float im = par ? mine_hi : recv;
                        float c2 = fmaf(re, re, im * im);
                        if (kScaled) c2 *= sc16[q];   // squared column scale
                        c2v[q] = c2;
                        mask |= c2 > thr ? (1u << q) : 0u;
                    }
                    // columns past the dictionary (the last tile) take no part
                    const int64_t lim = p.D - col0;
                    if (lim < 16) mask &= lim <= 0 ? 0u : ((1u << lim) - 1u);
                    // columns arrive in increasing index order: strictly better enters
                    while (mask) {
                        const int q = __ffs(mask) - 1;
                        mask &= mask - 1;
                        tk.insert(sel16(c2v, q), col0 + q);
                        thr = fmaxf(seed, tk.v[K - 1]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty_bar[buf]);
                if (++buf == NBUF) { buf = 0; buf_ph ^= 1; }
                if (p.thr_live && vlive) {
                    // this lane's K-th best covers a subset of the dictionary, so it
                    // bounds the voxel's K-th best; share it with the other chunks
                    // (non-negative floats order like their bit patterns)
                    int *cell = reinterpret_cast<int *>(p.thr_live + vrow);
                    if (tk.v[K - 1] > 0.f) atomicMax(cell, __float_as_int(tk.v[K - 1]));
                    const float lb = __int_as_float(__ldcg(cell));
                    if (lb > 0.f) seed = fmaxf(seed, lb * (1.0f - 1.0e-6f));
                    thr = fmaxf(seed, tk.v[K - 1]);
                }
            }
            // merge the Re/Im pair's lists (each covered half of the columns):
            // only the even lane inserts, so the odd lane's list stays intact
            // while it is being read
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const float ov = __shfl_xor_sync(0xffffffffu, tk.v[q], 1);
                const int oi = __shfl_xor_sync(0xffffffffu, tk.i[q], 1);
                if (par == 0 && oi != 0x7fffffff) tk.insert(ov, oi);
            }
            const int64_t v = (int64_t)(vu * NB + blk) * (BM / 2) + (row >> 1);
            if (par == 0 && v < p.V) {
                float2 *dst = p.part + ((size_t)v * p.n_chunks + chunk) * K;
#pragma unroll
                for (int q = 0; q < K; ++q) dst[q] = make_float2(tk.v[q], __int_as_float(tk.i[q]));
            }
        }
    epi_done:;
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 2 * BN);
    }
}

// ---------------------------------------------------------------------------
// voxel prep: normalise and lay out the two real rows per voxel. SPLIT
// (MRF_F32 over a stored dictionary): fp16 rows in a_hi, and in a_lo the e4m3
// residual plane followed, plane8 bytes on, by the e4m3 value plane.

template <int MODE, bool SPLIT = false>
__global__ void __launch_bounds__(256) voxel_prep_kernel(const float2 *x, int64_t V, int n, int ld, uint8_t *a_hi,
                                                         uint8_t *a_lo, float *row_scale, size_t plane8)
{
    const int64_t v = blockIdx.x;
    __shared__ float red[2][8];
    float ss = 0.f, mx = 0.f;
    const bool live = v < V;
    if (live) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const float2 z = x[(size_t)v * n + j];
            ss = fmaf(z.x, z.x, fmaf(z.y, z.y, ss));
            mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.y)));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ss; red[1][threadIdx.x >> 5] = mx; }
    __syncthreads();
    ss = 0.f; mx = 0.f;
    for (int w = 0; w < 8; ++w) { ss += red[0][w]; mx = fmaxf(mx, red[1][w]); }
    const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
    float qs = inv;
    if (MODE == MRF_FP8E4M3) {
        const float m = mx * inv;
        const float scale = m > 0.f ? m / 448.0f : 1.0f;
        qs = inv / scale;
        if (threadIdx.x == 0) row_scale[v] = live ? scale : 0.f;
    }
    const int half = ld / 2;   // timepoint slots per row
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
        float xr = 0.f, xi = 0.f;
        if (live && j < n) {
            const float2 z = x[(size_t)v * n + j];
            xr = z.x * qs;
            xi = z.y * qs;
        }
        const size_t r0 = (size_t)(2 * v) * ld, r1 = (size_t)(2 * v + 1) * ld;
        if (SPLIT) {
            const SplitPair p0 = split_pair(xr, xi, kSplitHiX), p1 = split_pair(xi, -xr, kSplitHiX);
            reinterpret_cast<uint32_t *>(a_hi + 2 * r0)[j] = p0.hi;
            reinterpret_cast<uint32_t *>(a_hi + 2 * r1)[j] = p1.hi;
            reinterpret_cast<uint16_t *>(a_lo + r0)[j] = p0.l8;
            reinterpret_cast<uint16_t *>(a_lo + r1)[j] = p1.l8;
            reinterpret_cast<uint16_t *>(a_lo + plane8 + r0)[j] = p0.h8;
            reinterpret_cast<uint16_t *>(a_lo + plane8 + r1)[j] = p1.h8;
        } else if (MODE == MRF_FP8E4M3) {
            __nv_fp8x2_storage_t q0 = __nv_cvt_float2_to_fp8x2(make_float2(xr, xi), __NV_SATFINITE, __NV_E4M3);
            __nv_fp8x2_storage_t q1 = __nv_cvt_float2_to_fp8x2(make_float2(xi, -xr), __NV_SATFINITE, __NV_E4M3);
            reinterpret_cast<__nv_fp8x2_storage_t *>(a_hi + r0)[j] = q0;
            reinterpret_cast<__nv_fp8x2_storage_t *>(a_hi + r1)[j] = q1;
        } else {
            __nv_bfloat162 h0 = __floats2bfloat162_rn(xr, xi);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(xi, -xr);
            reinterpret_cast<__nv_bfloat162 *>(a_hi + 2 * r0)[j] = h0;
            reinterpret_cast<__nv_bfloat162 *>(a_hi + 2 * r1)[j] = h1;
            if (MODE == MRF_F32) {
                const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
                reinterpret_cast<__nv_bfloat162 *>(a_lo + 2 * r0)[j] = __floats2bfloat162_rn(xr - f0.x, xi - f0.y);
                reinterpret_cast<__nv_bfloat162 *>(a_lo + 2 * r1)[j] = __floats2bfloat162_rn(xi - f1.x, -xr - f1.y);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// merge the per-chunk top-k lists of each voxel (one warp per voxel)

template <int K>
__global__ void merge_kernel(const float2 *part, int64_t V, int n_chunks, const float *row_scale, int64_t *idx_out,
                             float *cc2_out)
{
    const int64_t v = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= V) return;
    const int total = n_chunks * K;
    const float2 *src = part + (size_t)v * total;
    const float rs = row_scale ? row_scale[v] : 1.f;
    const float rs2 = rs * rs;
    int last_i = -1;
    float last_c = 3.4e38f;
    for (int q = 0; q < K; ++q) {
        // best candidate strictly after (last_c, last_i) in the order
        float bc = -2.f;
        int bi = 0x7fffffff;
        for (int k = lane; k < total; k += 32) {
            const float2 e = src[k];
            const float c = e.x;
            const int i = __float_as_int(e.y);
            if (i == 0x7fffffff) continue;
            if (before(last_c, last_i, c, i) && before(c, i, bc, bi)) { bc = c; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (before(oc, oi, bc, bi)) { bc = oc; bi = oi; }
        }
        if (lane == 0) {
            idx_out[(size_t)v * K + q] = bi == 0x7fffffff ? -1 : (int64_t)bi;
            cc2_out[(size_t)v * K + q] = bi == 0x7fffffff ? -1.f : bc * rs2;
        }
        last_c = bc;
        last_i = bi;
    }
}

// ---------------------------------------------------------------------------
// re-score: FP32 re-simulation of each candidate, FP64 accumulation of the
// inner product and norms, best by FP64 CC (ties to the smaller index)


// Temporal smoothing of the re-simulated candidates (the dictionary's own,
// see mrf_dict_smooth): half-width h and weights w[k], k = 0..h.
struct RescoreSmooth {
    int h;
    float w[3];
};

template <bool XONLY>
// A warp re-scores 32 / W voxels, W = the candidates per voxel (a power of
// two): lane l takes candidate l mod W of voxel l / W, so every lane
// simulates (W = 1 for the rank-1 form: 32 voxels per warp).
__global__ void rescore_kernel(SeqDev s, GridDev g, const float2 *x, int64_t V, int K, const int64_t *cand,
                               const float *cand_cc2, int rank, int64_t D, RescoreSmooth sm, mrf_result *out,
                               int *err)
{
    const int lane = threadIdx.x & 31;
    const int ncand = rank ? K : 1;   // 1, 2, 4, ..., 32
    const int W = ncand, per_warp = 32 / W;
    const int64_t v0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * per_warp;
    if (v0 >= V) return;   // whole warps only
    const int grp = lane / W, sub = lane % W;
    const int64_t v = v0 + grp;
    const bool vlive = v < V;
    const int n = s.n;
    const float2 *xv = x + (size_t)(vlive ? v : v0) * n;
    // ||x||^2 in FP64, each voxel's sum taken by the whole warp in the same
    // order whatever W is
    double xx = 0.0;
    for (int p = 0; p < per_warp && v0 + p < V; ++p) {
        const float2 *xp = x + (size_t)(v0 + p) * n;
        double t = 0.0;
        for (int j = lane; j < n; j += 32) {
            const float2 z = xp[j];
            t += (double)z.x * z.x + (double)z.y * z.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (p == grp) xx = t;
    }

    const int64_t e = vlive ? cand[(size_t)v * K + sub] : -1;
    const bool live = e >= 0 && mrf_in_bounds(e < D, err);
    int a = 0, b = 0, c = 0;
    if (live) unravel_dev(g, e, a, b, c);
    Relax r = relax_make(live ? g.t1[a] : 1.f, live ? g.t2[b] : 1.f, live ? g.df[c] : 0.f);
    Bloch st;
    bloch_start(st, s, r);
    double ipr = 0.0, ipi = 0.0, dd = 0.0;
    if (sm.h == 0) {
        for (int j0 = 0; j0 < n; j0 += 8) {
            float pr = 0.f, pi = 0.f, pd = 0.f;
            const int j1 = min(n, j0 + 8);
            for (int j = j0; j < j1; ++j) {
                float sr, si;
                bloch_step_otf<XONLY>(st, s, r, j, sr, si);
                const float2 z = __ldg(&xv[j]);
                // x conj(d) = (xr dr + xi di) + i (xi dr - xr di)
                pr = fmaf(z.x, sr, fmaf(z.y, si, pr));
                pi = fmaf(z.y, sr, fmaf(-z.x, si, pi));
                pd = fmaf(sr, sr, fmaf(si, si, pd));
            }
            ipr += (double)pr;
            ipi += (double)pi;
            dd += (double)pd;
        }
    } else {
        // raw samples pass through a five-sample ring (ring[4] newest); sample t
        // is smoothed once s_{t+h} exists, with weights renormalised at the ends
        float2 ring[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) ring[k] = make_float2(0.f, 0.f);
        float pr = 0.f, pi = 0.f, pd = 0.f;
        int cnt = 0;
        auto emit = [&](int t, int newest) {
            float sr = 0.f, si = 0.f, ws = 0.f;
            for (int k = -sm.h; k <= sm.h; ++k) {
                const int tk = t + k;
                if (tk < 0 || tk > newest) continue;
                const float2 zz = ring[4 - (newest - tk)];
                const float w = sm.w[k < 0 ? -k : k];
                sr = fmaf(w, zz.x, sr);
                si = fmaf(w, zz.y, si);
                ws += w;
            }
            sr /= ws;
            si /= ws;
            const float2 z = __ldg(&xv[t]);
            pr = fmaf(z.x, sr, fmaf(z.y, si, pr));
            pi = fmaf(z.y, sr, fmaf(-z.x, si, pi));
            pd = fmaf(sr, sr, fmaf(si, si, pd));
            if (++cnt == 8) {
                ipr += (double)pr; ipi += (double)pi; dd += (double)pd;
                pr = pi = pd = 0.f;
                cnt = 0;
            }
        };
        for (int j = 0; j < n; ++j) {
            float sr, si;
            bloch_step_otf<XONLY>(st, s, r, j, sr, si);
#pragma unroll
            for (int k = 0; k < 4; ++k) ring[k] = ring[k + 1];
            ring[4] = make_float2(sr, si);
            if (j >= sm.h) emit(j - sm.h, j);
        }
        for (int t = max(0, n - sm.h); t < n; ++t) emit(t, n - 1);
        ipr += (double)pr;
        ipi += (double)pi;
        dd += (double)pd;
    }
    const double mag = sqrt(ipr * ipr + ipi * ipi);
    double cc = (live && dd > 0.0 && xx > 0.0) ? mag / sqrt(xx * dd) : -1.0;
    // best by FP64 CC within the voxel's W lanes, ties to the smaller index;
    // also the runner-up CC
    double bc = cc, sc = -2.0;
    int64_t bi = live ? e : INT64_MAX;
    int bl = lane;
    for (int o = W / 2; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const double os = __shfl_xor_sync(0xffffffffu, sc, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        const bool take = oc > bc || (oc == bc && oi < bi);
        const double lose = take ? bc : oc;
        sc = fmax(fmax(sc, os), lose);
        if (take) { bc = oc; bi = oi; bl = ol; }
    }
    const double wr = __shfl_sync(0xffffffffu, ipr, bl);
    const double wi = __shfl_sync(0xffffffffu, ipi, bl);
    const double wd = __shfl_sync(0xffffffffu, dd, bl);
    const int wa = __shfl_sync(0xffffffffu, a, bl), wb = __shfl_sync(0xffffffffu, b, bl),
              wc = __shfl_sync(0xffffffffu, c, bl);
    if (sub == 0 && vlive) {
        mrf_result res;
        if (bi == INT64_MAX || bc < 0.0) {
            res.index = -1; res.i_t1 = res.i_t2 = res.i_df = -1;
            res.t1_ms = res.t2_ms = res.df_hz = 0.f;
            res.cc = 0.f; res.m0 = 0.f; res.phase = 0.f;
        } else {
            res.index = bi;
            res.i_t1 = wa; res.i_t2 = wb; res.i_df = wc;
            res.t1_ms = g.t1[wa]; res.t2_ms = g.t2[wb]; res.df_hz = g.df[wc];
            res.cc = (float)bc;
            res.m0 = wd > 0.0 ? (float)(sqrt(wr * wr + wi * wi) / wd) : 0.f;
            res.phase = (float)atan2(wi, wr);
        }
        res.entries_evaluated = (int32_t)D;
        res.min_margin = (ncand > 1 && sc > -1.5) ? (float)(bc - sc) : -1.f;
        (void)cand_cc2;
        out[v] = res;
    }
}

// Chunked brute force (mrf_match_bruteforce_grid): per voxel, the range's
// answer moves to whole-grid indices and replaces the running one if its CC
// is higher (ties keep the earlier range, i.e. the smaller linear index); the
// runner-up is the best CC among all other candidates the ranges re-scored.
__global__ void chunk_merge_kernel(mrf_result *best, float *second, const mrf_result *part, int64_t V, int64_t base,
                                   int a0)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    mrf_result p = part ? part[v] : best[v];
    if (p.index >= 0) {
        p.index += base;
        p.i_t1 += a0;
    }
    const float c1 = p.index >= 0 ? p.cc : -1.f;
    const float c2 = (p.index >= 0 && p.min_margin >= 0.f) ? p.cc - p.min_margin : -1.f;
    mrf_result b = p;
    float s = c2;
    if (part) {
        b = best[v];
        s = second[v];
        const float b1 = b.index >= 0 ? b.cc : -1.f;
        const int64_t ev = (int64_t)b.entries_evaluated + p.entries_evaluated;
        if (c1 > b1) {
            s = fmaxf(b1, c2);
            b = p;
        } else {
            s = fmaxf(s, c1);
        }
        b.entries_evaluated = (int32_t)min(ev, (int64_t)INT32_MAX);
    }
    b.min_margin = (b.index >= 0 && s > -0.5f) ? b.cc - s : -1.f;
    second[v] = s;
    best[v] = b;
}

// ---------------------------------------------------------------------------
// host side

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2D K-major map: rows x ld elements, box = (128 bytes of K) x box_rows, 128-byte swizzle.
// 2D tensor map over `rows` rows of `ld` elements; consecutive map rows are
// `row_step` stored rows apart (1: dense; > 1: a strided sample).
int make_map(CUtensorMap *m, const void *base, int64_t rows, int ld, int elem_bytes, int box_rows, int row_step = 1)
{
    auto enc = get_encode();
    if (!enc) return set_error(MRF_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * elem_bytes * (cuuint64_t)row_step};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MRF_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return MRF_OK;
}

int gcd_i(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }

// Operand maps of one launch: A (voxels) and B (dictionary), each up to three planes.
struct MatchMaps {
    CUtensorMap a, a2, a3, b, b2, b3;
};

template <int MODE, int K, bool GEN>
int launch_match_k(mrf_ctx *ctx, const MatchMaps &m, const MatchParams &p, cudaStream_t stream)
{
    // the opt-in for large dynamic shared memory is a property of the kernel on
    // one device: set once per instantiation and device, under the matcher mutex
    // (devices past the table set it on every launch)
    constexpr int kDevs = 64;
    static bool attr_set[kDevs] = {};
    const int dev = ctx->device;
    if (dev < 0 || dev >= kDevs || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(match_kernel<MODE, K, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes<MODE>());
        if (e != cudaSuccess) return cuda_fail(e, "matcher shared-memory attribute");
        if (dev >= 0 && dev < kDevs) attr_set[dev] = true;
    }
    const int units = p.n_vu * p.n_chunks;
    const int grid = std::min(units, ctx->sm_count);
    match_kernel<MODE, K, GEN><<<grid, threads_of<MODE, GEN>(), smem_bytes<MODE>(), stream>>>(m.a, m.a2, m.a3, m.b, m.b2,
                                                                                           m.b3, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matcher launch");
    return MRF_OK;
}

template <int MODE, bool GEN = false>
int launch_match_mode(mrf_ctx *ctx, int K, const MatchMaps &m, const MatchParams &p, cudaStream_t stream)
{
    switch (K) {
    case 1: return launch_match_k<MODE, 1, GEN>(ctx, m, p, stream);
    case 2: return launch_match_k<MODE, 2, GEN>(ctx, m, p, stream);
    case 4: return launch_match_k<MODE, 4, GEN>(ctx, m, p, stream);
    case 8: return launch_match_k<MODE, 8, GEN>(ctx, m, p, stream);
    case 16: return launch_match_k<MODE, 16, GEN>(ctx, m, p, stream);
    case 32: return launch_match_k<MODE, 32, GEN>(ctx, m, p, stream);
    }
    return set_error(MRF_E_INVALID, "top_k");
}

}  // namespace

std::mutex g_match_attr_mu;

int launch_chunk_merge(mrf_result *best, float *second, const mrf_result *part, int64_t V, int64_t base, int a0,
                       cudaStream_t stream)
{
    const int64_t blocks = (V + 255) / 256;
    chunk_merge_kernel<<<(unsigned)blocks, 256, 0, stream>>>(best, second, part, V, base, a0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "chunk merge launch");
    return MRF_OK;
}

int run_match(mrf_ctx *ctx, const mrf_dict *d, const void *fp, int64_t V, int32_t precision, int32_t top_k,
              int rescore, mrf_result *out, int64_t *idx_out, float *cc2_out, cudaStream_t stream, bool fused)
{
    const int mode = precision;
    const int K = top_k;
    // MRF_F32 over a stored dictionary takes the split form (fp16 and e4m3
    // planes); generated tiles the bf16 hi/lo split
    const bool split = mode == MRF_F32 && !fused;
    const int nb = split ? Cfg<kModeSplit>::kNB : mode == MRF_F32 ? Cfg<MRF_F32>::kNB : Cfg<MRF_BF16>::kNB;   // voxel blocks per CTA
    const int n_vu = (int)((V + 64 * nb - 1) / (64 * nb));
    const int64_t V_pad = (int64_t)n_vu * nb * 64;
    const int ebytes = mode == MRF_FP8E4M3 ? 1 : 2;
    const int n_tiles = (int)((d->entries + BN - 1) / BN);
    // voxel-unit groups whose operands (all hi/lo parts) fit about 40 MB of L2;
    // the dictionary streams once per group
    const size_t unit_bytes = (size_t)nb * 2 * 64 * d->ld * ebytes * (mode == MRF_F32 ? 2 : 1);
    const int g_max = std::max(1, std::min(n_vu, (int)((size_t)40 * 1024 * 1024 / unit_bytes)));
    const int n_groups = (n_vu + g_max - 1) / g_max;
    const int group_vu = (n_vu + n_groups - 1) / n_groups;   // balanced groups
    // chunks: make each group's units a multiple of the SM count where possible
    int n_chunks = ctx->sm_count / gcd_i(group_vu, ctx->sm_count);
    n_chunks = std::max(1, std::min(n_chunks, n_tiles));
    const int kbe = (mode == MRF_FP8E4M3 || split) ? 128 : 64;   // elements per K block (split: e4m3 blocks)
    const int k_blocks = (2 * d->n + kbe - 1) / kbe;   // K blocks holding at least one real element
    const int k_valid = 2 * d->n - (k_blocks - 1) * kbe;  // real elements in the last one (1..kbe)
    const int kstep = (mode == MRF_FP8E4M3 || split) ? 32 : 16;
    const int last_ksteps = (k_valid + kstep - 1) / kstep;
    // split form: fp16 K blocks of 64 elements and the k-steps of the last
    const int k_blocks16 = (2 * d->n + 63) / 64;
    const int last_ks16 = (2 * d->n - (k_blocks16 - 1) * 64 + 15) / 16;

    // Threshold pre-pass (K >= 8 on large dictionaries): the same matcher
    // over every kSample-th entry gives each voxel the K-th best CC^2 of that
    // subset, a lower bound on its K-th best over the whole dictionary. The
    // full pass starts every top-k list at that bound, so far fewer columns
    // reach the insertion; the merged result is the same.
    constexpr int kSample = 64;
    const int64_t D_s = (d->entries + kSample - 1) / kSample;
    const int n_tiles_s = (int)((D_s + BN - 1) / BN);
    const bool seeded = !fused && K >= 8 && n_tiles_s >= 4;   // generated tiles have no stored sample
    const int n_chunks_s = seeded ? std::max(1, std::min(n_tiles_s, ctx->sm_count / std::max(1, n_vu))) : 0;

    // scratch: A operands, row scales, partial lists, candidates, pre-pass lists and bounds
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    const size_t bA = (size_t)(2 * V_pad) * d->ld * ebytes;
    const size_t bA2 = mode == MRF_F32 ? bA : 0;
    const size_t bRS = mode == MRF_FP8E4M3 ? sizeof(float) * V_pad : 0;
    const size_t bP = sizeof(float2) * (size_t)V * n_chunks * K;
    const size_t bI = idx_out ? 0 : sizeof(int64_t) * (size_t)V * K;
    const size_t bC = cc2_out ? 0 : sizeof(float) * (size_t)V * K;
    const size_t bPs = seeded ? sizeof(float2) * (size_t)V * n_chunks_s * K : 0;
    const size_t bIs = seeded ? sizeof(int64_t) * (size_t)V * K : 0;
    const size_t bCs = seeded ? sizeof(float) * (size_t)V * K : 0;
    const size_t bL = K >= 8 ? sizeof(float) * (size_t)V : 0;
    const size_t total = al(bA) + al(bA2) + al(bRS) + al(bP) + al(bI) + al(bC) + al(bPs) + al(bIs) + al(bCs) + al(bL);
    int rc = budget_charge(ctx, total);
    if (rc) return rc;
    uint8_t *ws = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&ws, total, stream);
    if (e != cudaSuccess) { budget_release(ctx, total); return cuda_fail(e, "matcher scratch"); }
    uint8_t *pA = ws;
    uint8_t *pA2 = pA + al(bA);
    float *pRS = (float *)(pA2 + al(bA2));
    float2 *pP = (float2 *)((uint8_t *)pRS + al(bRS));
    int64_t *pI = idx_out ? idx_out : (int64_t *)((uint8_t *)pP + al(bP));
    float *pC = cc2_out ? cc2_out : (float *)((uint8_t *)pP + al(bP) + al(bI));
    uint8_t *pS = (uint8_t *)pP + al(bP) + al(bI) + al(bC);
    float2 *pPs = (float2 *)pS;
    int64_t *pIs = (int64_t *)(pS + al(bPs));
    float *pCs = (float *)(pS + al(bPs) + al(bIs));
    float *pL = bL ? (float *)(pS + al(bPs) + al(bIs) + al(bCs)) : nullptr;

    auto finish = [&](int code) {
        cudaFreeAsync(ws, stream);
        budget_release(ctx, total);
        return code;
    };

    // 1. voxel prep (split: the e4m3 value plane follows the residual plane in pA2)
    const size_t plane8 = (size_t)(2 * V_pad) * d->ld;
    if (split)
        voxel_prep_kernel<MRF_F32, true><<<(unsigned)V_pad, 256, 0, stream>>>((const float2 *)fp, V, d->n, d->ld, pA, pA2, pRS, plane8);
    else if (mode == MRF_F32)
        voxel_prep_kernel<MRF_F32><<<(unsigned)V_pad, 256, 0, stream>>>((const float2 *)fp, V, d->n, d->ld, pA, pA2, pRS, 0);
    else if (mode == MRF_BF16)
        voxel_prep_kernel<MRF_BF16><<<(unsigned)V_pad, 256, 0, stream>>>((const float2 *)fp, V, d->n, d->ld, pA, pA2, pRS, 0);
    else
        voxel_prep_kernel<MRF_FP8E4M3><<<(unsigned)V_pad, 256, 0, stream>>>((const float2 *)fp, V, d->n, d->ld, pA, pA2, pRS, 0);
    count_launch(ctx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return finish(cuda_fail(e, "voxel prep launch"));

    // 2. tensor-core pass. Split maps: a = fp16 rows, a2 / a3 = e4m3 residual /
    // value planes of the voxels; b = fp16 rows, b2 / b3 = e4m3 value /
    // residual planes of the dictionary (each plane D x ld bytes).
    MatchMaps mm;
    const size_t dplane8 = (size_t)d->entries * d->ld;
    if (split) {
        rc = make_map(&mm.a, pA, 2 * V_pad, d->ld, 2, BM);
        if (!rc) rc = make_map(&mm.a2, pA2, 2 * V_pad, d->ld, 1, BM);
        if (!rc) rc = make_map(&mm.a3, pA2 + plane8, 2 * V_pad, d->ld, 1, BM);
        if (!rc) rc = make_map(&mm.b, d->hi, d->entries, d->ld, 2, BN);
        if (!rc) rc = make_map(&mm.b2, d->lo, d->entries, d->ld, 1, BN);
        if (!rc) rc = make_map(&mm.b3, (const uint8_t *)d->lo + dplane8, d->entries, d->ld, 1, BN);
        if (rc) return finish(rc);
    } else {
        rc = make_map(&mm.a, pA, 2 * V_pad, d->ld, ebytes, BM);
        if (!rc && !fused) rc = make_map(&mm.b, d->hi, d->entries, d->ld, ebytes, BN);
        if (!rc && mode == MRF_F32) rc = make_map(&mm.a2, pA2, 2 * V_pad, d->ld, ebytes, BM);
        if (rc) return finish(rc);
        if (mode != MRF_F32) mm.a2 = mm.a;
        if (fused) mm.b = mm.a;   // unused: the kernel generates its B tiles
        mm.b2 = mm.b;
        mm.a3 = mm.a;
        mm.b3 = mm.b;
    }
    MatchParams p;
    p.D = d->entries;
    p.V = V;
    p.n_tiles = n_tiles;
    p.n_vu = n_vu;
    p.n_chunks = n_chunks;
    p.group_vu = group_vu;
    p.k_blocks = k_blocks;
    p.last_ksteps = last_ksteps;
    p.k_blocks16 = k_blocks16;
    p.last_ks16 = last_ks16;
    p.colscale = mode == MRF_BF16 ? nullptr : d->scale;
    p.col_stride = 1;
    p.thr0 = nullptr;
    p.thr0_stride = 0;
    p.thr_live = nullptr;
    p.part = pP;
    p.err = ctx->err_flag;
    p.s = d->seq->dev();
    p.g = d->grid.dev();
    p.n = d->n;
    if (fused) p.colscale = nullptr;

    const unsigned mblocks = (unsigned)((V + 3) / 4);
    auto merge = [&](const float2 *part, int chunks, const float *row_scale, int64_t *io, float *co) {
        switch (K) {
        case 1: merge_kernel<1><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        case 2: merge_kernel<2><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        case 4: merge_kernel<4><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        case 8: merge_kernel<8><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        case 16: merge_kernel<16><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        case 32: merge_kernel<32><<<mblocks, 128, 0, stream>>>(part, V, chunks, row_scale, io, co); break;
        }
        count_launch(ctx);
        return cudaGetLastError();
    };
    auto launch_all = [&](const MatchMaps &m, const MatchParams &pp) {
        std::lock_guard<std::mutex> lk(g_match_attr_mu);
        if (fused && mode == MRF_F32) return launch_match_mode<MRF_F32, true>(ctx, K, m, pp, stream);
        if (fused) return launch_match_mode<MRF_BF16, true>(ctx, K, m, pp, stream);
        if (mode == MRF_F32) return launch_match_mode<kModeSplit>(ctx, K, m, pp, stream);
        if (mode == MRF_BF16) return launch_match_mode<MRF_BF16>(ctx, K, m, pp, stream);
        return launch_match_mode<MRF_FP8E4M3>(ctx, K, m, pp, stream);
    };
    {
        // one timed region: pre-pass, its merge and the full pass
        ProfScope prof(ctx, kProfMatcher, stream);
        if (seeded) {
            // every kSample-th stored row of each plane
            MatchMaps ms = mm;
            rc = make_map(&ms.b, d->hi, D_s, d->ld, split ? 2 : ebytes, BN, kSample);
            if (!rc && split) rc = make_map(&ms.b2, d->lo, D_s, d->ld, 1, BN, kSample);
            if (!rc && split) rc = make_map(&ms.b3, (const uint8_t *)d->lo + dplane8, D_s, d->ld, 1, BN, kSample);
            if (rc) return finish(rc);
            if (!split) ms.b2 = ms.b3 = ms.b;
            MatchParams ps = p;
            ps.D = D_s;
            ps.n_tiles = n_tiles_s;
            ps.n_chunks = n_chunks_s;
            ps.group_vu = n_vu;
            ps.col_stride = kSample;
            ps.part = pPs;
            rc = launch_all(ms, ps);
            if (rc) return finish(rc);
            count_launch(ctx);
            // bounds in the kernel's units (no FP8 row scale)
            e = merge(pPs, n_chunks_s, nullptr, pIs, pCs);
            if (e != cudaSuccess) return finish(cuda_fail(e, "pre-pass merge launch"));
            p.thr0 = pCs + (K - 1);
            p.thr0_stride = K;
        }
        if (pL) {
            e = cudaMemsetAsync(pL, 0, bL, stream);
            if (e != cudaSuccess) return finish(cuda_fail(e, "bound scratch"));
            p.thr_live = pL;
        }
        rc = launch_all(mm, p);
    }
    if (rc) return finish(rc);

    // 3. merge chunk lists
    e = merge(pP, n_chunks, mode == MRF_FP8E4M3 ? pRS : nullptr, pI, pC);
    if (e != cudaSuccess) return finish(cuda_fail(e, "merge launch"));

    // 4. re-score / finalize
    if (out) {
        const SeqDev s = d->seq->dev();
        const GridDev g = d->grid.dev();
        RescoreSmooth sm;
        sm.h = d->smooth_h;
        for (int k = 0; k < 3; ++k) sm.w[k] = d->smooth_w[k];
        const int64_t per_block = 4 * (32 / (rescore ? K : 1));   // 4 warps of 32 / W voxels
        const unsigned rblocks = (unsigned)((V + per_block - 1) / per_block);
        if (s.xonly)
            rescore_kernel<true><<<rblocks, 128, 0, stream>>>(s, g, (const float2 *)fp, V, K, pI, pC, rescore, d->entries, sm, out, ctx->err_flag);
        else
            rescore_kernel<false><<<rblocks, 128, 0, stream>>>(s, g, (const float2 *)fp, V, K, pI, pC, rescore, d->entries, sm, out, ctx->err_flag);
        count_launch(ctx);
        e = cudaGetLastError();
        if (e != cudaSuccess) return finish(cuda_fail(e, "re-score launch"));
    }
    return finish(MRF_OK);
}
