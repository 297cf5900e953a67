// lattice.cuh -- per-node arithmetic of the FitzHugh-Nagumo lattice (Sec. 5.1,
// here in the Rogers-McCulloch form), shared by every kernel that takes a
// lattice sub-step so that they round identically.
#pragma once

#include "pf_device.cuh"

namespace pf {

// Drift of v and w at one node: c1 v (v - a)(1 - v) - c2 v w + D lap + I and
// b (v - d w).
template <typename Real>
__device__ __forceinline__ Real fhn_drift_v(const ModelParams &mp, Real v, Real w, Real lap, Real I)
{
    const Real a = par<Real>(mp, 0), c1 = par<Real>(mp, 2), c2 = par<Real>(mp, 3), D = par<Real>(mp, 5);
    return c1 * v * (v - a) * ((Real)1 - v) - c2 * v * w + D * lap + I;
}

template <typename Real>
__device__ __forceinline__ Real fhn_drift_w(const ModelParams &mp, Real v, Real w)
{
    const Real b = par<Real>(mp, 1), d = par<Real>(mp, 4);
    return b * (v - d * w);
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
// neighbour pairs (missing neighbours passed as the node itself).
template <typename Real>
__device__ __forceinline__ void pair_laplacian(Real v0, Real v1, Real up0, Real up1, Real dn0, Real dn1, Real left,
                                               Real right, Real &l0, Real &l1)
{
    l0 = ((up0 + dn0) + (left + v1)) - (Real)4 * v0;
    l1 = ((up1 + dn1) + (v0 + right)) - (Real)4 * v1;
}

}  // namespace pf
