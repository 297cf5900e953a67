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
__device__ __forceinline__ float gelu_fast(float x)
{
    const float u = fabsf(x) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, u, 1.0f)));
    float q = fmaf(t, 1.061405429f, -1.453152027f);
    q = fmaf(t, q, 1.421413741f);
    q = fmaf(t, q, -0.284496736f);
    q = fmaf(t, q, 0.254829592f);
    q *= t;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-u * u * 1.44269504088896341f));
    const float tail = q * e;  // 1 - erf(|x| / sqrt 2) = 2 Phi(-|x|), without cancellation
    return 0.5f * x * (x >= 0.0f ? 2.0f - tail : tail);
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
