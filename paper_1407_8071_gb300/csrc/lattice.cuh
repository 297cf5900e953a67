// lattice.cuh -- per-node arithmetic of the FitzHugh-Nagumo lattice (Sec. 5.1,
// here in the Rogers-McCulloch form), shared by every kernel that takes a
// lattice sub-step so that they round identically.
#pragma once

#include "pf_device.cuh"

namespace pf {

// Drift of v and w at one node: c1 v (v - a)(1 - v) - c2 v w + D lap + I and
// b (v - d w).  In FP32 every rounding is spelled out (((c1 v)(v - a))(1 - v),
// then - (c2 v) w and + D lap as fused multiply-adds, then + I; and
// b (v - d w) with v - d w fused), so that the two-node forms below give the
// same bits lane by lane.
template <typename Real>
__device__ __forceinline__ Real fhn_drift_v(const ModelParams &mp, Real v, Real w, Real lap, Real I)
{
    const Real a = par<Real>(mp, 0), c1 = par<Real>(mp, 2), c2 = par<Real>(mp, 3), D = par<Real>(mp, 5);
    if constexpr (std::is_same<Real, float>::value) {
        const float cubic = __fmul_rn(__fmul_rn(__fmul_rn(c1, v), __fadd_rn(v, -a)), __fadd_rn(1.0f, -v));
        return __fadd_rn(__fmaf_rn(D, lap, __fmaf_rn(-__fmul_rn(c2, v), w, cubic)), I);
    } else {
        return c1 * v * (v - a) * ((Real)1 - v) - c2 * v * w + D * lap + I;
    }
}

template <typename Real>
__device__ __forceinline__ Real fhn_drift_w(const ModelParams &mp, Real v, Real w)
{
    const Real b = par<Real>(mp, 1), d = par<Real>(mp, 4);
    if constexpr (std::is_same<Real, float>::value) return __fmul_rn(b, __fmaf_rn(-d, w, v));
    else return b * (v - d * w);
}

// The FP32 drifts of two nodes at once on the packed FP32 pipes (lane i is
// fhn_drift_v / fhn_drift_w of node i, bit for bit).
__device__ __forceinline__ float2 fhn_drift_v_x2(const ModelParams &mp, float2 v, float2 w, float2 lap, float2 I)
{
    const float a = mp.fp[0], c1 = mp.fp[2], c2 = mp.fp[3], D = mp.fp[5];
    const float2 cubic = __fmul2_rn(__fmul2_rn(__fmul2_rn(f2s(c1), v), __fadd2_rn(v, f2s(-a))),
                                    __fadd2_rn(f2s(1.0f), make_float2(-v.x, -v.y)));
    const float2 c2v = __fmul2_rn(f2s(c2), v);
    return __fadd2_rn(__ffma2_rn(f2s(D), lap, __ffma2_rn(make_float2(-c2v.x, -c2v.y), w, cubic)), I);
}

__device__ __forceinline__ float2 fhn_drift_w_x2(const ModelParams &mp, float2 v, float2 w)
{
    return __fmul2_rn(f2s(mp.fp[1]), __ffma2_rn(f2s(-mp.fp[4]), w, v));
}

// Mirror reflection of a lattice coordinate k in [-2, J + 1] (zero flux at the
// edges): -1 -> 0, -2 -> 1, J -> J - 1, J + 1 -> J - 2.
__device__ __forceinline__ int mirror_index(int k, int J) { return k < 0 ? -k - 1 : (k >= J ? 2 * J - k - 1 : k); }

// Euler-Maruyama update written with explicit fused multiply-adds, so that
// every kernel that takes a lattice sub-step rounds it identically.
__device__ __forceinline__ float em_update(float x, float f, float z, float dt, float sq)
{
    return __fmaf_rn(sq, z, __fmaf_rn(dt, f, x));
}
__device__ __forceinline__ double em_update(double x, double f, double z, double dt, double sq)
{
    return fma(sq, z, fma(dt, f, x));
}

// Zero-flux Laplacian of a node pair from its own values and the four
// neighbour pairs (missing neighbours passed as the node itself).  In FP32:
// (up + dn) + (the row neighbours' sum), then - 4 v fused, as the two-node
// form rounds it.
template <typename Real>
__device__ __forceinline__ void pair_laplacian(Real v0, Real v1, Real up0, Real up1, Real dn0, Real dn1, Real left,
                                               Real right, Real &l0, Real &l1)
{
    if constexpr (std::is_same<Real, float>::value) {
        l0 = __fmaf_rn(-4.0f, v0, __fadd_rn(__fadd_rn(up0, dn0), __fadd_rn(left, v1)));
        l1 = __fmaf_rn(-4.0f, v1, __fadd_rn(__fadd_rn(up1, dn1), __fadd_rn(v0, right)));
    } else {
        l0 = ((up0 + dn0) + (left + v1)) - (Real)4 * v0;
        l1 = ((up1 + dn1) + (v0 + right)) - (Real)4 * v1;
    }
}

__device__ __forceinline__ float2 pair_laplacian_x2(float2 v, float2 up, float2 dn, float left, float right)
{
    const float2 ud = __fadd2_rn(up, dn), lr = __fadd2_rn(make_float2(left, v.x), make_float2(v.y, right));
    return __ffma2_rn(f2s(-4.0f), v, __fadd2_rn(ud, lr));
}

// Euler-Maruyama update of two values at once: em_update lane by lane.
__device__ __forceinline__ float2 em_update_x2(float2 x, float2 f, float2 z, float dt, float sq)
{
    return __ffma2_rn(f2s(sq), z, __ffma2_rn(f2s(dt), f, x));
}

// The four normals of one node pair's Philox block as (v, w) noise pairs:
// zv = (z[0], z[2]) and zw = (z[1], z[3]) of normals4<float>, bit for bit.
__device__ __forceinline__ void pair_normals_x2(const Key &key, uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t stream, uint32_t block, float2 &zv, float2 &zw)
{
    const uint4 r = philox4x32_10(make_uint4(c0, c1, c2, (stream << 24) | block), key);
    box_muller_x2(r.x, r.y, r.z, r.w, zv, zw);
}

}  // namespace pf
