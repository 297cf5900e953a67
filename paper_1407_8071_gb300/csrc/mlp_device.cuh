// mlp_device.cuh -- the learned proposal's network on the tensor cores.
//
// 51 inputs (5x5 patches of v and w around an observed lattice node, and y at
// the node) -> 128 -> 128 -> 4 (o_mu_v, o_mu_w, o_s_v, o_s_w), GELU in its
// tanh form.
// Operands are bfloat16, accumulation FP32 on the tensor cores (tcgen05): the
// inputs are padded to 64 columns and the 4 outputs to 8 (16 in the MMA).
// Parameter vector (FP32 master, the oracle's layout): W1 (128 x 51), b1 (128),
// W2 (128 x 128), b2 (128), W3 (4 x 128), b3 (4).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace pf {
namespace mlp {

constexpr int kIn = 51, kInPad = 64, kHid = 128, kOut = 4, kOutPad = 8;
constexpr int kParams = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;  // 23684
constexpr int kOffW1 = 0, kOffB1 = kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
constexpr float kClamp = 3.0f;

// BF16 weights in the layout the kernels stage into shared memory:
// W1p [128][64] (zero-padded columns), W2p [128][128], W3p [8][128] (rows 4..7 zero).
constexpr int kPackW1 = kHid * kInPad, kPackW2 = kHid * kHid, kPackW3 = kOutPad * kHid;
constexpr int kPackTotal = kPackW1 + kPackW2 + kPackW3;

// GELU in its tanh form (Hendrycks & Gimpel 2016),
//   g(x) = x (1 + tanh(u)) / 2,  u = k0 (x + k1 x^3),  k0 = sqrt(2/pi), k1 = 0.044715,
// which equals x / (1 + e^{-2u}) = x / (1 + 2^a) with a = x (c0 + c1 x^2),
// c0 = -2 k0 log2(e), c1 = c0 k1: one exp2 and one reciprocal on the MUFU
// unit and five FP32 operations, each of which rounds to nearest.  With exp2
// and the reciprocal within 2^-21 and 2^-22 of their results, the value is
// within 3.6e-7 (|x| + |g(x)|) of g(x): the argument's three roundings enter
// through r (1 - r) |a| ln 2 <= 0.23 (r = 1 / (1 + 2^a)), exp2's error through
// r (1 - r) <= 1/4, the reciprocal's and the two last roundings through r.
// Saturation is exact: 2^a overflows to +inf for large negative x (r = 0,
// g = -0) and flushes to 0 for large positive x (r = 1, g = x).
constexpr float kGeluC0 = -2.30220818519592285f;  // -2 sqrt(2/pi) log2(e)
constexpr float kGeluC1 = -0.102943241596221924f;  // kGeluC0 * 0.044715
constexpr float kGelu2K0 = 1.59576912160573081f;   // 2 sqrt(2/pi)
constexpr float kGelu3K1 = 0.134145f;              // 3 * 0.044715

__device__ __forceinline__ float rcp_apx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_apx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// g of two values at once on the packed FP32 pipes (each lane rounds as the
// scalar instruction would).
__device__ __forceinline__ float2 gelu_x2(float2 x)
{
    const float2 p = __ffma2_rn(__fmul2_rn(x, x), make_float2(kGeluC1, kGeluC1), make_float2(kGeluC0, kGeluC0));
    const float2 a = __fmul2_rn(x, p);
    const float2 d = __fadd2_rn(make_float2(ex2_apx(a.x), ex2_apx(a.y)), make_float2(1.0f, 1.0f));
    return __fmul2_rn(x, make_float2(rcp_apx(d.x), rcp_apx(d.y)));
}

// g'(x) = r + x r (1 - r) 2 k0 (1 + 3 k1 x^2), r = 1 / (1 + e^{-2u}) (the
// training kernels' GELU derivative; r (1 - r) is written so that it is 0,
// not NaN, where 2^a saturates).
__device__ __forceinline__ float gelu_grad(float x)
{
    const float x2 = x * x;
    const float r = rcp_apx(1.0f + ex2_apx(x * fmaf(kGeluC1, x2, kGeluC0)));
    return r + x * r * (1.0f - r) * (kGelu2K0 * fmaf(kGelu3K1, x2, 1.0f));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

}  // namespace mlp
}  // namespace pf
