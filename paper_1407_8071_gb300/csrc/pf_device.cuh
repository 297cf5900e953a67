// pf_device.cuh -- device building blocks of the GB300 ensemble particle filter:
// the counter-based generator, Box-Muller normals, and the state-space models
// of arXiv:1407.8071 (Sec. 4.1 Lorenz 63; Sec. 5.1 FitzHugh-Nagumo lattice in
// the Rogers-McCulloch form; a linear-Gaussian model whose exact filter is the
// Kalman filter).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace pf {

enum : uint32_t {
    kStreamTruth = 0u,
    kStreamObs = 1u,
    kStreamInit = 2u,
    kStreamDyn = 3u,
    kStreamResample = 4u,
    kStreamProposal = 5u,
    kStreamMisc = 6u,       // also the particles' random stimulus of the paper's lattice variant
    kStreamStimTruth = 7u,  // the truth's random stimulus
};

enum ModelKind : int32_t { kLinearGaussian = 0, kLorenz63 = 1, kFhnLattice = 2, kFhnPaper = 3 };

// Both lattices: particle-major state, node pairs, stencil kernels.
__host__ __device__ __forceinline__ bool is_lattice(int32_t kind) { return kind == kFhnLattice || kind == kFhnPaper; }

constexpr int kMaxLgDim = 4;
constexpr int kMaxObsSmall = 8;  // observation indices passed by value for the small models

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the 4x32
// Philox bijection with the published multipliers; round r uses the key
// advanced r times by the Weyl increments (0.32 fixed point of the golden
// ratio's fraction and of sqrt(3) - 1).  The ten round keys are computed once
// on the host and passed as kernel parameters, so the rounds read them as
// constant operands.  One 32x32->64 multiply per product.
// ---------------------------------------------------------------------------
struct Key {
    uint32_t k0[10], k1[10];
};

inline Key make_key(uint64_t seed)
{
    Key k;
    uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const Key &key)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ key.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ key.k1[r],
                       (uint32_t)p0);
    }
    return c;
}

// Box & Muller (1958) on two 32-bit words.  u1 = ((a >> 8) + 1) 2^-24 in (0, 1]
// and u2 = (b >> 8) 2^-24 in [0, 1) are exact in binary32 and binary64;
// z0 = R cos(2 pi u2), z1 = R sin(2 pi u2), R = sqrt(-2 ln u1).
// FP32: the angle is taken as 2 pi (u2 - 1/2) in [-pi, pi) (u2 - 1/2 is exact;
// cos and sin change sign) so the hardware sine/cosine run on their accurate
// range (absolute error below 2^-21); R = v * rsqrt(v); v = -2 ln u1 from
// neg2_ln_u24 below.
template <typename Real>
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, Real &z0, Real &z1);

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// -2 ln(n 2^-24) for an integer n in [1, 2^24], in FP32 with a relative error
// of a few ulp everywhere (also as n -> 2^24, where v -> 0).  Range reduction:
// n = f 2^k with f in [sqrt(1/2), sqrt(2)) (k from the exponent of the exact
// binary32 n, moved by one when the significand is at or above sqrt(2)), then
// ln f = 2 artanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + ...), s = (f - 1)/(f + 1),
// |s| <= 3 - 2 sqrt(2) = 0.1716 (Abramowitz & Stegun 4.1.27); the first
// omitted term, 2 s^9 / 9, is below 3e-8 of ln f.  f - 1 is exact (Sterbenz),
// so s keeps its relative accuracy as f -> 1.  -2 ln u1 = -2 (k - 24) ln 2 - 2 ln f.
// Every rounding is spelled out (no contraction left to the compiler), so the
// two-lane form below gives the same bits lane by lane.
constexpr float kM2Ln2 = -1.38629436111989061883f;  // -2 ln 2
constexpr float kTwoPi = 6.28318530717958647692f;

__device__ __forceinline__ uint32_t ln_reduce(uint32_t n, uint32_t &k)
{
    const uint32_t bits = __float_as_uint(__uint2float_rn(n));
    k = (bits - 0x3F3504F3u) >> 23;  // 0x3F3504F3: binary32 sqrt(1/2)
    return bits - (k << 23);
}

__device__ __forceinline__ float neg2_ln_u24(uint32_t n)
{
    uint32_t k;
    const float f = __uint_as_float(ln_reduce(n, k));
    const float s = __fmul_rn(__fadd_rn(f, -1.0f), rcp_approx(__fadd_rn(f, 1.0f)));
    const float s2 = __fmul_rn(s, s);
    float c = __fmaf_rn(-4.0f / 7.0f, s2, -4.0f / 5.0f);  // -2 x the series' coefficients 2 / (2j + 1)
    c = __fmaf_rn(c, s2, -4.0f / 3.0f);
    const float m2lnf = __fmaf_rn(__fmul_rn(s, s2), c, __fmul_rn(-4.0f, s));
    return __fmaf_rn((float)((int32_t)k - 24), kM2Ln2, m2lnf);
}

template <>
__device__ __forceinline__ void box_muller<float>(uint32_t a, uint32_t b, float &z0, float &z1)
{
    const float v = neg2_ln_u24((a >> 8) + 1u);
    const float h = __fmaf_rn(__uint2float_rn(b >> 8), 0x1p-24f, -0.5f);
    const float R = v > 0.0f ? __fmul_rn(v, rsqrtf(v)) : 0.0f;
    float s, c;
    __sincosf(__fmul_rn(kTwoPi, h), &s, &c);
    z0 = __fmul_rn(-R, c);
    z1 = __fmul_rn(-R, s);
}

// Two lanes at once on the packed FP32 pipes (fma/mul/add.rn.f32x2: each
// lane rounds as the scalar instruction does): lane i is neg2_ln_u24(n_i) and
// box_muller<float>(a_i, b_i) bit for bit, for half the FP32 instructions.
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

__device__ __forceinline__ float2 neg2_ln_u24_x2(uint32_t n0, uint32_t n1)
{
    uint32_t k0, k1;
    const uint32_t r0 = ln_reduce(n0, k0), r1 = ln_reduce(n1, k1);
    const float2 f = make_float2(__uint_as_float(r0), __uint_as_float(r1));
    const float2 fp = __fadd2_rn(f, f2s(1.0f));
    const float2 s = __fmul2_rn(__fadd2_rn(f, f2s(-1.0f)), make_float2(rcp_approx(fp.x), rcp_approx(fp.y)));
    const float2 s2 = __fmul2_rn(s, s);
    float2 c = __ffma2_rn(f2s(-4.0f / 7.0f), s2, f2s(-4.0f / 5.0f));
    c = __ffma2_rn(c, s2, f2s(-4.0f / 3.0f));
    const float2 m2lnf = __ffma2_rn(__fmul2_rn(s, s2), c, __fmul2_rn(f2s(-4.0f), s));
    return __ffma2_rn(make_float2((float)((int32_t)k0 - 24), (float)((int32_t)k1 - 24)), f2s(kM2Ln2), m2lnf);
}

__device__ __forceinline__ void box_muller_x2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, float2 &z0,
                                              float2 &z1)
{
    const float2 v = neg2_ln_u24_x2((a0 >> 8) + 1u, (a1 >> 8) + 1u);
    const float2 h = __ffma2_rn(make_float2(__uint2float_rn(b0 >> 8), __uint2float_rn(b1 >> 8)), f2s(0x1p-24f),
                                f2s(-0.5f));
    const float2 rv = __fmul2_rn(v, make_float2(rsqrtf(v.x), rsqrtf(v.y)));
    const float2 nR = make_float2(v.x > 0.0f ? -rv.x : -0.0f, v.y > 0.0f ? -rv.y : -0.0f);
    const float2 ang = __fmul2_rn(f2s(kTwoPi), h);
    float s0, c0, s1, c1;
    __sincosf(ang.x, &s0, &c0);
    __sincosf(ang.y, &s1, &c1);
    z0 = __fmul2_rn(nR, make_float2(c0, c1));
    z1 = __fmul2_rn(nR, make_float2(s0, s1));
}

template <>
__device__ __forceinline__ void box_muller<double>(uint32_t a, uint32_t b, double &z0, double &z1)
{
    const double u1 = ((double)(a >> 8) + 1.0) * 0x1p-24;
    const double u2 = (double)(b >> 8) * 0x1p-24;
    const double R = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = R * c;
    z1 = R * s;
}

// Normals (4 per block) of counter (c0, c1, c2, stream<<24 | block).
template <typename Real>
__device__ __forceinline__ void normals4(const Key &key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t stream,
                                         uint32_t block, Real z[4])
{
    const uint4 r = philox4x32_10(make_uint4(c0, c1, c2, (stream << 24) | block), key);
    box_muller<Real>(r.x, r.y, z[0], z[1]);
    box_muller<Real>(r.z, r.w, z[2], z[3]);
}

// normals4<float> of two counters (c0a and c0b, the other words shared) in the
// two lanes of z: lane 0 is the first counter's normal, lane 1 the second's.
__device__ __forceinline__ void normals4_x2(const Key &key, uint32_t c0a, uint32_t c0b, uint32_t c1, uint32_t c2,
                                            uint32_t stream, uint32_t block, float2 z[4])
{
    const uint32_t w = (stream << 24) | block;
    const uint4 ra = philox4x32_10(make_uint4(c0a, c1, c2, w), key);
    const uint4 rb = philox4x32_10(make_uint4(c0b, c1, c2, w), key);
    box_muller_x2(ra.x, ra.y, rb.x, rb.y, z[0], z[1]);
    box_muller_x2(ra.z, ra.w, rb.z, rb.w, z[2], z[3]);
}

// ---------------------------------------------------------------------------
// Model parameters passed by value to the kernels.
// ---------------------------------------------------------------------------
struct ModelParams {
    int32_t kind;
    int32_t dx;
    int32_t J;
    int32_t K;             // Euler-Maruyama sub-steps per observation
    double dt;
    double sigma_dyn;
    double sigma0;
    double sigma_obs;
    double p[24];          // LG: A row-major (dx <= 4); L63: s, r, b; FHN: a, b, c1, c2, d, D, amp, steps, block;
                           // the paper's lattice: the 17 values of pf.h
    int32_t dy;
    int32_t obs_small[kMaxObsSmall];  // observation indices when dy <= kMaxObsSmall
    double x0_small[kMaxLgDim];       // prior mean for the small models
    // FP32 and integer copies made once on the host (FP64 is a narrow pipe on this
    // GPU, and converting a double to an integer runs on it):
    float fp[24];      // p
    int64_t ip[24];    // p truncated toward zero (the integer-valued parameters: step counts, sizes)
    float fdt;         // dt
    float fsq;         // sigma_dyn * sqrt(dt)
    float fhalf_prec;  // -1 / (2 sigma_obs^2)
    double dsq;        // sigma_dyn * sqrt(dt) in FP64 (truth records)
    double dhalf_prec; // -1 / (2 sigma_obs^2) in FP64
};

// Model constants in the precision of the state.
template <typename Real>
__device__ __forceinline__ Real par(const ModelParams &mp, int i)
{
    if constexpr (std::is_same<Real, float>::value) return mp.fp[i];
    else return mp.p[i];
}
template <typename Real>
__device__ __forceinline__ Real par_dt(const ModelParams &mp)
{
    if constexpr (std::is_same<Real, float>::value) return mp.fdt;
    else return mp.dt;
}
template <typename Real>
__device__ __forceinline__ Real par_sq(const ModelParams &mp)
{
    if constexpr (std::is_same<Real, float>::value) return mp.fsq;
    else return mp.dsq;
}
template <typename Real>
__device__ __forceinline__ Real par_half_prec(const ModelParams &mp)
{
    if constexpr (std::is_same<Real, float>::value) return mp.fhalf_prec;
    else return mp.dhalf_prec;
}

// Drift of the small models (thread per particle), in the state's precision.
template <int D, typename Real>
struct SmallModel {
    // f(x) for LG (drift -A x) or Lorenz 63 (Sec. 4.1; first component
    // -s (x1 - x2) as in eq. eqDiscreteLorenz-1).
    __device__ __forceinline__ static void drift(const ModelParams &mp, const Real x[D], Real f[D])
    {
        if (mp.kind == kLorenz63) {
            const Real s = par<Real>(mp, 0), r = par<Real>(mp, 1), b = par<Real>(mp, 2);
            f[0] = s * (x[1] - x[0]);
            f[1] = r * x[0] - x[1] - x[0] * x[2];
            f[2] = x[0] * x[1] - b * x[2];
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                Real s = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) s += par<Real>(mp, i * D + j) * x[j];
                f[i] = -s;
            }
        }
    }
};

// lcm(D, 4) / D sub-steps share lcm(D, 4) / 4 Philox blocks: normal number
// nu = k * D + v of an observation interval sits in block nu / 4, lane nu % 4.
template <int D>
struct NoisePacking {
    static constexpr int lcm = (D % 4 == 0) ? D : (D % 2 == 0) ? 2 * D : 4 * D;
    static constexpr int steps = lcm / D;   // sub-steps per group
    static constexpr int blocks = lcm / 4;  // Philox calls per group
};

// Propagates R particles of a small model over the K sub-steps of
// observation t (Alg. 1 step 2a; Euler-Maruyama), stream `stream`, counter
// words (c0[r], t, c2).  Several particles per thread give the scheduler
// independent generator chains to interleave.  Noise = false takes the
// noise-free Euler steps (z = 0) without drawing normals.
template <int D, int R, typename Real, bool Noise = true>
__device__ __forceinline__ void propagate_small_n(const ModelParams &mp, const Key &key, uint32_t stream,
                                                  const uint32_t c0[R], uint32_t t, uint32_t c2, Real x[R][D])
{
    using NP = NoisePacking<D>;
    const Real dt = par_dt<Real>(mp);
    const Real sq = par_sq<Real>(mp);
    const int K = mp.K;
    uint32_t block = 0;
    for (int k0 = 0; k0 < K; k0 += NP::steps) {
        Real z[R][4 * NP::blocks];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int b = 0; b < NP::blocks; ++b) {
                if (Noise) {
                    normals4<Real>(key, c0[r], t, c2, stream, block + b, z[r] + 4 * b);
                } else {  // the noise-free Euler prediction (auxiliary filter's look-ahead)
#pragma unroll
                    for (int i = 0; i < 4; ++i) z[r][4 * b + i] = (Real)0;
                }
            }
        block += NP::blocks;
#pragma unroll
        for (int s = 0; s < NP::steps; ++s) {
            if (k0 + s < K) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    Real f[D];
                    SmallModel<D, Real>::drift(mp, x[r], f);
#pragma unroll
                    for (int v = 0; v < D; ++v) x[r][v] = x[r][v] + dt * f[v] + sq * z[r][s * D + v];
                }
            }
        }
    }
}

// The same interval for two particles of a thread at once (counter words c0a
// and c0b), their states in the two lanes of x: the normals from
// normals4_x2, the drift and the Euler-Maruyama update on the packed FP32
// pipes with every rounding spelled out -- Lorenz 63 as s (x2 - x1),
// x1 (r - x3) - x2, x1 x2 - b x3; the linear-Gaussian drift as the dot product
// sum_j A_ij x_j in order j = 0, 1, ..; the update (x + dt f) + sq z, two
// fused multiply-adds.  Both particles of a thread take the same instructions.
template <int D, bool Noise = true>
__device__ __forceinline__ void propagate_small_x2(const ModelParams &mp, const Key &key, uint32_t stream,
                                                   uint32_t c0a, uint32_t c0b, uint32_t t, uint32_t c2, float2 x[D])
{
    using NP = NoisePacking<D>;
    const float2 DT = f2s(mp.fdt), NDT = f2s(-mp.fdt), SQ = f2s(mp.fsq), M1 = f2s(-1.0f);
    const bool lorenz = mp.kind == kLorenz63;
    const int K = mp.K;
    uint32_t block = 0;
    for (int k0 = 0; k0 < K; k0 += NP::steps) {
        float2 z[4 * NP::blocks];
#pragma unroll
        for (int b = 0; b < NP::blocks; ++b) {
            if (Noise) {
                normals4_x2(key, c0a, c0b, t, c2, stream, block + b, z + 4 * b);
            } else {  // the noise-free Euler prediction (auxiliary filter's look-ahead)
#pragma unroll
                for (int i = 0; i < 4; ++i) z[4 * b + i] = f2s(0.0f);
            }
        }
        block += NP::blocks;
#pragma unroll
        for (int s = 0; s < NP::steps; ++s) {
            if (k0 + s < K) {
                if (D == 3 && lorenz) {
                    const float2 f0 = __fmul2_rn(f2s(mp.fp[0]), __ffma2_rn(x[0], M1, x[1]));
                    const float2 f1 = __ffma2_rn(x[1], M1, __fmul2_rn(x[0], __ffma2_rn(x[2], M1, f2s(mp.fp[1]))));
                    const float2 fz = __ffma2_rn(f2s(-mp.fp[2]), x[2], __fmul2_rn(x[0], x[1]));
                    x[0] = __ffma2_rn(SQ, z[s * D], __ffma2_rn(DT, f0, x[0]));
                    x[1] = __ffma2_rn(SQ, z[s * D + 1], __ffma2_rn(DT, f1, x[1]));
                    x[2] = __ffma2_rn(SQ, z[s * D + 2], __ffma2_rn(DT, fz, x[2]));
                } else {  // dx' = -A x dt + sq dW
                    float2 ax[D];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        ax[i] = __fmul2_rn(f2s(mp.fp[i * D]), x[0]);
#pragma unroll
                        for (int j = 1; j < D; ++j) ax[i] = __ffma2_rn(f2s(mp.fp[i * D + j]), x[j], ax[i]);
                    }
#pragma unroll
                    for (int i = 0; i < D; ++i) x[i] = __ffma2_rn(SQ, z[s * D + i], __ffma2_rn(NDT, ax[i], x[i]));
                }
            }
        }
    }
}

template <int D, typename Real>
__device__ __forceinline__ void propagate_small(const ModelParams &mp, const Key &key, uint32_t stream, uint32_t c0,
                                                uint32_t t, uint32_t c2, Real x[D])
{
    Real xr[1][D];
#pragma unroll
    for (int v = 0; v < D; ++v) xr[0][v] = x[v];
    const uint32_t c[1] = {c0};
    propagate_small_n<D, 1, Real>(mp, key, stream, c, t, c2, xr);
#pragma unroll
    for (int v = 0; v < D; ++v) x[v] = xr[0][v];
}

// log g without its constant: -1/2 sum_j (y_j - x[idx_j])^2 / sigma_obs^2.
template <int D, typename Real>
__device__ __forceinline__ Real loglik_small(const ModelParams &mp, const float *y, const Real x[D])
{
    Real s = 0;
    for (int j = 0; j < mp.dy; ++j) {
        const int idx = mp.obs_small[j];
        Real xv = 0;
#pragma unroll
        for (int v = 0; v < D; ++v)
            if (v == idx) xv = x[v];
        const Real e = (Real)y[j] - xv;
        s += e * e;
    }
    return par_half_prec<Real>(mp) * s;
}

}  // namespace pf
