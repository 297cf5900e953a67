// mlp_device.cuh -- the learned proposal's network on the tensor cores.
//
// 51 inputs (5x5 patches of v and w around an observed lattice node, and y at
// the node) -> 128 -> 128 -> 4 (o_mu_v, o_mu_w, o_s_v, o_s_w), exact GELU.
// Operands are bfloat16, accumulation FP32 (mma.sync m16n8k16 .bf16): the
// inputs are padded to 64 columns and the 4 outputs to one 8-wide tile.
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

// Shared-memory rows get a 16-byte pad so that the fragment loads of the 8
// row groups fall in different banks.
constexpr int kLdIn = kInPad + 8;    // bf16 elements per padded row of 64
constexpr int kLdHid = kHid + 8;     // ... of 128

// BF16 weights in the layout the kernels stage into shared memory:
// W1p [128][64] (zero-padded columns), W2p [128][128], W3p [8][128] (rows 4..7 zero).
constexpr int kPackW1 = kHid * kInPad, kPackW2 = kHid * kHid, kPackW3 = kOutPad * kHid;
constexpr int kPackTotal = kPackW1 + kPackW2 + kPackW3;

// GELU for the inference kernel: x Phi(x) with Phi(x) = (1 + erf(x / sqrt 2)) / 2
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

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D += A * B for one 16 x 8 tile, A 16 x 16 row-major, B 16 x 8 column-major
// (given as B^T rows), bfloat16 operands, FP32 accumulators.  Fragment
// ownership (PTX ISA, mma.m16n8k16): lane = 4 g + c;
//   A: a0 (g, 2c..2c+1), a1 (g+8, 2c..), a2 (g, 2c+8..), a3 (g+8, 2c+8..)
//   B: b0 (k 2c..2c+1, n g), b1 (k 2c+8.., n g)
//   D: d0,d1 (g, 2c..2c+1), d2,d3 (g+8, 2c..2c+1)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of rows [r0, r0+16), columns [k0, k0+16) of a row-major bf16
// matrix in shared memory with leading dimension ld (elements).
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16 *s, int ld, int r0, int k0, int lane)
{
    const int g = lane >> 2, c = lane & 3;
    const __nv_bfloat16 *p0 = s + (r0 + g) * ld + k0 + 2 * c;
    const __nv_bfloat16 *p1 = p0 + 8 * ld;
    a[0] = *reinterpret_cast<const uint32_t *>(p0);
    a[1] = *reinterpret_cast<const uint32_t *>(p1);
    a[2] = *reinterpret_cast<const uint32_t *>(p0 + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(p1 + 8);
}

// B fragment for output columns [n0, n0+8) and k in [k0, k0+16) from B^T
// stored row-major ([n][k], leading dimension ld).
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const __nv_bfloat16 *s, int ld, int n0, int k0, int lane)
{
    const int g = lane >> 2, c = lane & 3;
    const __nv_bfloat16 *p = s + (n0 + g) * ld + k0 + 2 * c;
    b[0] = *reinterpret_cast<const uint32_t *>(p);
    b[1] = *reinterpret_cast<const uint32_t *>(p + 8);
}

// One warp: acc[nt] (16 x 8 tiles nt = 0..NT-1 starting at column n0) +=
// A[16 rows from r0][K] * (B^T)[n0 + 8 nt][K].
template <int NT, int K>
__device__ __forceinline__ void warp_gemm(float (&acc)[NT][4], const __nv_bfloat16 *sA, int lda, int r0,
                                          const __nv_bfloat16 *sBt, int ldb, int n0, int lane)
{
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        load_a(a, sA, lda, r0, k0, lane);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            uint32_t b[2];
            load_b(b, sBt, ldb, n0 + 8 * nt, k0, lane);
            mma_bf16(acc[nt], a, b);
        }
    }
}

}  // namespace mlp
}  // namespace pf
