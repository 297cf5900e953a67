// mlp_device.cuh -- the learned proposal's network on the tensor cores.
//
// 51 inputs (5x5 patches of v and w around an observed lattice node, and y at
// the node) -> 128 -> 128 -> 4 (o_mu_v, o_mu_w, o_s_v, o_s_w), exact GELU.
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

// GELU of the tensor-core kernels: x Phi(x) with Phi(x) = (1 + erf(x / sqrt 2)) / 2
// and erf from Abramowitz & Stegun 7.1.26 (Hastings' rational form,
// |error| <= 1.5e-7): 1 - erf(u) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-u^2},
// t = 1 / (1 + p u), u = |x| / sqrt 2; Phi(x) = 1 - tail / 2 for x >= 0 and
// tail / 2 below.  Far below the BF16 rounding of the activations it feeds.
// Every rounding is spelled out, so that the two-lane form below gives the
// same bits lane by lane.
constexpr float kInvSqrt2 = 0.70710678118654752f, kLog2e = 1.44269504088896341f, kAsP = 0.3275911f;
constexpr float kAs1 = 0.254829592f, kAs2 = -0.284496736f, kAs3 = 1.421413741f, kAs4 = -1.453152027f,
                kAs5 = 1.061405429f;

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

__device__ __forceinline__ float gelu_fast(float x)
{
    const float u = __fmul_rn(fabsf(x), kInvSqrt2);
    const float t = rcp_apx(__fmaf_rn(kAsP, u, 1.0f));
    float q = __fmaf_rn(t, kAs5, kAs4);
    q = __fmaf_rn(t, q, kAs3);
    q = __fmaf_rn(t, q, kAs2);
    q = __fmaf_rn(t, q, kAs1);
    q = __fmul_rn(q, t);
    const float e = ex2_apx(__fmul_rn(__fmul_rn(u, u), -kLog2e));
    const float tail = __fmul_rn(q, e);  // 1 - erf(|x| / sqrt 2) = 2 Phi(-|x|), without cancellation
    return __fmul_rn(__fmul_rn(0.5f, x), x >= 0.0f ? __fmaf_rn(tail, -1.0f, 2.0f) : tail);
}

// gelu_fast of two values at once on the packed FP32 pipes (lane by lane the
// same bits, about two thirds of the instructions).
__device__ __forceinline__ float2 gelu_fast_x2(float2 x)
{
    const float2 c = make_float2(kInvSqrt2, kInvSqrt2);
    const float2 u = __fmul2_rn(make_float2(fabsf(x.x), fabsf(x.y)), c);
    const float2 d = __ffma2_rn(make_float2(kAsP, kAsP), u, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_apx(d.x), rcp_apx(d.y));
    float2 q = __ffma2_rn(t, make_float2(kAs5, kAs5), make_float2(kAs4, kAs4));
    q = __ffma2_rn(t, q, make_float2(kAs3, kAs3));
    q = __ffma2_rn(t, q, make_float2(kAs2, kAs2));
    q = __ffma2_rn(t, q, make_float2(kAs1, kAs1));
    q = __fmul2_rn(q, t);
    const float2 a = __fmul2_rn(__fmul2_rn(u, u), make_float2(-kLog2e, -kLog2e));
    const float2 tail = __fmul2_rn(q, make_float2(ex2_apx(a.x), ex2_apx(a.y)));
    const float2 two = __ffma2_rn(tail, make_float2(-1.0f, -1.0f), make_float2(2.0f, 2.0f));
    const float2 sel = make_float2(x.x >= 0.0f ? two.x : tail.x, x.y >= 0.0f ? two.y : tail.y);
    return __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), x), sel);
}

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

}  // namespace mlp
}  // namespace pf
