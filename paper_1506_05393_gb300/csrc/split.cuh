// Storage and products of the MRF_F32 form of the tensor-core matcher.
//
// A real operand value v (|v| <= 1: a component of a unit-norm voxel, or a
// magnetisation component of a dictionary entry) is held as three numbers,
//     hi = fp16(v 2^sh)                      sh = 15 for entries, 12 for voxels
//     h8 = e4m3(v 2^8)
//     l8 = e4m3((v - hi 2^-sh) 2^19)         the fp16 residual, |.| <= 2^-11 |v|
// and a product x d is formed as
//     hi_x hi_d + l8_x h8_d + h8_x l8_d       at the scale 2^27 (12 + 15 = 19 + 8 = 8 + 19).
// The two e4m3 products carry the residuals (each at most 2^-11 of |x d|)
// with at most 2^-3 relative error, and the dropped residual product is below
// 2^-22 |x d|: per term at most about 2^-13 |x d|, rms about 2^-16 |x d|.
// One fp16 MMA of K = 16 takes as long as one e4m3 MMA of K = 32, so the
// three products cost two bf16 product times per element against three for
// the bf16 hi/lo split (hi.hi + hi.lo + lo.hi).
//
// The tensor core adds e4m3 products into a large accumulator at a reduced
// precision (measured on sm_103a: an f8f6f4 MMA added after the fp16 ones
// lost its 2^-11-relative contribution, added before them it was exact to
// FP32 rounding), so every tile accumulates its two e4m3 products over the
// whole K range first and its fp16 products after them.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

constexpr float kSplitHiD = 32768.0f;              // 2^15: fp16 scale of dictionary entries
constexpr float kSplitHiX = 4096.0f;               // 2^12: fp16 scale of voxels
constexpr float kSplitH8 = 256.0f;                 // 2^8: e4m3 scale of the values
constexpr float kSplitL8 = 524288.0f;              // 2^19: e4m3 scale of the fp16 residuals
constexpr float kSplitUnscale = 1.0f / 134217728.0f;   // 2^-27: one operand side of the product scale
constexpr float kSplitDecHi = 1.0f / 32768.0f;     // entry value = hi 2^-15 + l8 2^-19
constexpr float kSplitDecLo = 1.0f / 524288.0f;

// The three parts of a complex sample (vr, vi) at fp16 scale sh: fp16 pair
// (4 bytes), e4m3 pair of the values and e4m3 pair of the residuals (2 bytes each).
struct SplitPair {
    uint32_t hi;
    uint16_t h8, l8;
};

__device__ __forceinline__ SplitPair split_pair(float vr, float vi, float sh)
{
    const __half2 h = __floats2half2_rn(vr * sh, vi * sh);
    const float2 hf = __half22float2(h);
    const float inv = 1.0f / sh;                      // a power of two: exact
    // v - hi is exact in FP32 (hi is v rounded to 11 significant bits)
    const float rr = vr - hf.x * inv, ri = vi - hf.y * inv;
    SplitPair p;
    p.hi = *reinterpret_cast<const uint32_t *>(&h);
    p.h8 = (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(vr * kSplitH8, vi * kSplitH8), __NV_SATFINITE, __NV_E4M3);
    p.l8 = (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(rr * kSplitL8, ri * kSplitL8), __NV_SATFINITE, __NV_E4M3);
    return p;
}

// Entry value from its stored fp16 part and e4m3 residual.
__device__ __forceinline__ float split_decode(__half hi, __nv_fp8_storage_t l8)
{
    const __half_raw r = __nv_cvt_fp8_to_halfraw(l8, __NV_E4M3);
    return fmaf(__half2float(__half(r)), kSplitDecLo, __half2float(hi) * kSplitDecHi);
}
