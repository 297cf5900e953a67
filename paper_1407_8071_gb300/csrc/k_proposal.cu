// k_proposal.cu -- the learned proposal inside the lattice filter, and the
// recording of training tuples.
//
// With a network set, a step of the lattice filter is
//   k_propagate_fhn(4)    K - 1 ordinary sub-steps (Alg. 1 step 2a, transition)
//   network forward       tensor cores, input rows gathered from the state
//                         (k_proposal_tc.cu; k_build_rows when recording tuples)
//   k_last_step_fhn(4)    last sub-step: proposal at the observed nodes, the
//                         transition elsewhere; weight g p / q, and the weight
//                         the transition alone would have given
//   k_proposal_select     per filter: ESS of the proposal weights; below
//                         ess_frac N the step falls back to the transition
// then the usual resampling chain.  Every random number is the transition's
// own (same counters), so a network whose output is zero reproduces the
// bootstrap filter bit for bit.
#include <algorithm>
#include <cmath>

#include "lattice.cuh"
#include "mlp_device.cuh"
#include "pf.h"
#include "pf_internal.h"

namespace pf {

// Network input rows (BF16, 64 wide, zero-padded) for every (particle, observed
// node): the 5x5 patches of v and w around the node, mirrored at the edges,
// then y at the node.
__global__ void k_build_rows(ModelParams mp, const float *__restrict__ x, int64_t P, const int32_t *__restrict__ pfilt,
                             const int32_t *__restrict__ obs_idx, const float *__restrict__ obs, int32_t obs_stride,
                             __nv_bfloat16 *__restrict__ rows)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int dy = mp.dy;
    if (gid >= P * dy) return;
    const int64_t p = gid / dy;
    const int j = (int)(gid - p * dy);
    const int J = mp.J, nn = J * J, nd = obs_idx[j], ri = nd / J, ci = nd - ri * J;
    const float *xp = x + p * (int64_t)mp.dx;
    const float y = obs[(obs_stride ? (int64_t)pfilt[p] * obs_stride : 0) + j];
    __nv_bfloat16 *out = rows + gid * mlp::kInPad;
    int r = 0;
    for (int di = -2; di <= 2; ++di)
        for (int dj = -2; dj <= 2; ++dj, ++r) {
            const int k = mirror_index(ri + di, J) * J + mirror_index(ci + dj, J);
            out[r] = __float2bfloat16_rn(xp[k]);
            out[25 + r] = __float2bfloat16_rn(xp[nn + k]);
        }
    out[50] = __float2bfloat16_rn(y);
    for (int k = 51; k < mlp::kInPad; ++k) out[k] = __float2bfloat16_rn(0.0f);
}

// The last sub-step of an observation interval with the proposal at the
// observed nodes (Alg. 1 step 2a with an importance function).  Same thread
// layout as k_propagate_fhn.  For an observed node and component c:
//   m = x + dt f(x),  mu = m + h o_mu,  s = h e^{os},  os = clip(o_s, -3, 3),
//   x' = mu + s z,  log p - log q = os + ((x' - mu)/s)^2 / 2 - ((x' - m)/h)^2 / 2,
// where z is the transition's own normal; elsewhere x' = m + h z.  Writes x',
// the transition's candidate and m at the observed nodes, log g + sum(log p -
// log q) and the transition's log g.
__global__ void __launch_bounds__(1024, 2) k_last_step_fhn(ModelParams mp, Key key, const int32_t *pfilt,
                                                           const FilterDesc *filt, float *x, int64_t P,
                                                           const float *obs, int32_t obs_stride,
                                                           const int32_t *obs_slot, const int32_t *d_t, int32_t ppc,
                                                           const float *mlp_out, float *xboot, float *mp_obs,
                                                           float *logw, float *logw_boot)
{
    extern __shared__ unsigned char smem_raw[];
    const int J = mp.J, nn = J * J, pairs = nn / 2, half = J / 2, dy = mp.dy;
    float2 *sv = reinterpret_cast<float2 *>(smem_raw);  // [ppc][pairs]
    const int slot = (int)threadIdx.x / pairs;
    const int s = min(slot, ppc);
    const int q = threadIdx.x - min(slot, ppc - 1) * pairs;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(*d_t + 1);
    const int k = mp.K - 1;
    uint32_t c0 = 0, c2 = 0;
    float v[2] = {0.f, 0.f}, w[2] = {0.f, 0.f};
    const int n0 = 2 * q, row = n0 / J, col = n0 - row * J;
    int32_t m = 0;
    if (active) {
        m = pfilt[p];
        c0 = (uint32_t)(p - filt[m].off);
        c2 = (uint32_t)m;
        const float *xi = x + p * (int64_t)mp.dx;
        v[0] = xi[n0];
        v[1] = xi[n0 + 1];
        w[0] = xi[nn + n0];
        w[1] = xi[nn + n0 + 1];
        sv[s * pairs + q] = make_float2(v[0], v[1]);
    }
    __syncthreads();
    float part_prop = 0.0f, part_boot = 0.0f, lw = 0.0f;
    if (active) {
        const float dt = mp.fdt, h = mp.fsq;
        const float2 *buf = sv + s * pairs;
        const int qu = row > 0 ? q - half : q, qd = row < J - 1 ? q + half : q;
        const int ql = col > 0 ? q - 1 : q, qr = col + 2 < J ? q + 1 : q;
        const float2 up = buf[qu], dn = buf[qd], lf = buf[ql], rt = buf[qr];
        const float left = col > 0 ? lf.y : v[0], right = col + 2 < J ? rt.x : v[1];
        float lap[2];
        pair_laplacian<float>(v[0], v[1], up.x, up.y, dn.x, dn.y, left, right, lap[0], lap[1]);
        const int64_t n_base = (int64_t)(t - 1) * mp.K;
        const bool on = (n_base + k) < mp.ip[7];
        const int blk = (int)mp.ip[8];
        float z[4];
        normals4<float>(key, c0, t, c2, kStreamDyn, (uint32_t)k * (uint32_t)(mp.dx / 4) + (uint32_t)q, z);
        const float *y = obs + (obs_stride ? (int64_t)m * obs_stride : 0);
        float *xo = x + p * (int64_t)mp.dx;
        const float inv_h = 1.0f / h;
#pragma unroll 1
        for (int e = 0; e < 2; ++e) {
            const int node = n0 + e;
            const bool stim = on && row < blk && col + e < blk;
            const float I = stim ? par<float>(mp, 6) : 0.0f;
            const float fv = fhn_drift_v<float>(mp, v[e], w[e], lap[e], I), fw = fhn_drift_w<float>(mp, v[e], w[e]);
            const float mv = __fmaf_rn(dt, fv, v[e]), mw = __fmaf_rn(dt, fw, w[e]);
            const float zv = z[2 * e], zw = z[2 * e + 1];
            const float bv = __fmaf_rn(h, zv, mv), bw = __fmaf_rn(h, zw, mw);  // = em_update
            float nv = bv, nw = bw;
            const int j = obs_slot[node];
            if (j >= 0) {
                float o[4] = {0.f, 0.f, 0.f, 0.f};
                if (mlp_out) {
                    const float4 oo = reinterpret_cast<const float4 *>(mlp_out)[p * dy + j];
                    o[0] = oo.x; o[1] = oo.y; o[2] = oo.z; o[3] = oo.w;
                }
                const float mc[2] = {mv, mw}, zc[2] = {zv, zw};
                float xn[2];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const float os = fminf(fmaxf(o[2 + cc], -mlp::kClamp), mlp::kClamp);
                    const float mu = __fmaf_rn(h, o[cc], mc[cc]);
                    const float es = __expf(os);  // exactly 1 at os = 0
                    const float sd = h * es;
                    xn[cc] = __fmaf_rn(sd, zc[cc], mu);
                    // standardised residuals under p and q (the same products when o = 0,
                    // so a zero network adds exactly nothing)
                    const float t1 = (xn[cc] - mc[cc]) * inv_h, t2 = (xn[cc] - mu) * (inv_h / es);
                    lw += os + 0.5f * (t2 * t2 - t1 * t1);
                }
                nv = xn[0];
                nw = xn[1];
                const int64_t oj = (p * dy + j) * 2;
                xboot[oj] = bv;
                xboot[oj + 1] = bw;
                mp_obs[oj] = mv;
                mp_obs[oj + 1] = mw;
                const float ep = y[j] - nv, eb = y[j] - bv;
                part_prop += ep * ep;
                part_boot += eb * eb;
            }
            xo[node] = nv;
            xo[nn + node] = nw;
        }
    }
    // per-particle sums, one warp per particle slot, fixed order
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);
    const int nthreads = blockDim.x;
    red[threadIdx.x] = part_prop;
    red[nthreads + threadIdx.x] = part_boot;
    red[2 * nthreads + threadIdx.x] = lw;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sl = warp; sl < ppc; sl += nwarps) {
        const int64_t pp = (int64_t)blockIdx.x * ppc + sl;
        float a = 0.0f, b = 0.0f, c = 0.0f;
        for (int i = lane; i < pairs; i += 32) {
            a += red[sl * pairs + i];
            b += red[nthreads + sl * pairs + i];
            c += red[2 * nthreads + sl * pairs + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0 && pp < P) {
            logw[pp] = mp.fhalf_prec * a + c;
            logw_boot[pp] = mp.fhalf_prec * b;
        }
    }
}

// The same last sub-step with four nodes per thread (lattice sides divisible
// by 4), the layout of k_propagate_fhn4: float4 loads and stores of a quad's v
// and w, one shared-memory exchange, the two pairs' normals, the per-node
// arithmetic of k_last_step_fhn in the same order, and the per-pair partial sums
// reduced per particle in the pair kernel's order -- so the results are the
// pair kernel's bit for bit, with four CTAs or three per SM instead of two.
constexpr int kLast4MaxThreads = 512;

// Sub-step k_sub of the proposal's span (the last `span` sub-steps of the
// interval, sharing one network evaluation): the transition at unobserved
// nodes, the proposal at observed ones.  The span's sums of log p - log q are
// carried in lw_acc from its first sub-step (first) to its last (last), which
// adds log g and writes the step's log-weights; a span of one sub-step is the
// last-sub-step reading (first = last = 1), the only one whose transition
// candidates (xboot, logw_boot) serve a fallback.

template <int MinB>
__global__ void __launch_bounds__(kLast4MaxThreads, MinB)
    k_last_step_fhn4(ModelParams mp, Key key, const int32_t *pfilt, const FilterDesc *filt, float *x, int64_t P,
                     const float *obs, int32_t obs_stride, const int32_t *obs_slot, const int32_t *d_t, int32_t ppc,
                     const float *mlp_out, float *xboot, float *mp_obs, float *logw, float *logw_boot,
                     int32_t k_sub, int32_t first, int32_t last, float *lw_acc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int J = mp.J, nn = J * J, quads = nn / 4, pairs = nn / 2, qrow = J / 4, dy = mp.dy;
    float4 *sv = reinterpret_cast<float4 *>(smem_raw);  // [ppc][quads]
    const int slot = (int)threadIdx.x / quads;
    const int s = min(slot, ppc);
    const int q = threadIdx.x - min(slot, ppc - 1) * quads;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(*d_t + 1);
    const int k = k_sub;
    uint32_t c0 = 0, c2 = 0;
    float v[4] = {0.f, 0.f, 0.f, 0.f}, w[4] = {0.f, 0.f, 0.f, 0.f};
    const int n0 = 4 * q, row = n0 / J, col = n0 - row * J;
    int32_t m = 0;
    if (active) {
        m = pfilt[p];
        c0 = (uint32_t)(p - filt[m].off);
        c2 = (uint32_t)m;
        const float4 a = *reinterpret_cast<const float4 *>(x + p * (int64_t)mp.dx + n0);
        const float4 b = *reinterpret_cast<const float4 *>(x + p * (int64_t)mp.dx + nn + n0);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        w[0] = b.x; w[1] = b.y; w[2] = b.z; w[3] = b.w;
        sv[s * quads + q] = a;
    }
    __syncthreads();
    float part_prop[2] = {0.f, 0.f}, part_boot[2] = {0.f, 0.f}, lw[2] = {0.f, 0.f};
    if (active) {
        const float dt = mp.fdt, h = mp.fsq;
        const float4 *buf = sv + s * quads;
        const int qu = row > 0 ? q - qrow : q, qd = row < J - 1 ? q + qrow : q;
        const bool has_left = col > 0, has_right = col + 4 < J;
        const float4 up = buf[qu], dn = buf[qd];
        const float left = has_left ? buf[q - 1].w : v[0], right = has_right ? buf[q + 1].x : v[3];
        // the transition of both node pairs on the packed FP32 pipes (the scalar helpers' bits)
        const float2 lap2[2] = {
            pair_laplacian_x2(make_float2(v[0], v[1]), make_float2(up.x, up.y), make_float2(dn.x, dn.y), left, v[2]),
            pair_laplacian_x2(make_float2(v[2], v[3]), make_float2(up.z, up.w), make_float2(dn.z, dn.w), v[1], right)};
        const int64_t n_base = (int64_t)(t - 1) * mp.K;
        const bool on = (n_base + k) < mp.ip[7];
        const int blk = (int)mp.ip[8];
        const uint32_t bk = (uint32_t)k * (uint32_t)(mp.dx / 4) + 2u * (uint32_t)q;
        float2 zv2[2], zw2[2], mv2[2], mw2[2], bv2[2], bw2[2];
#pragma unroll
        for (int hp = 0; hp < 2; ++hp) {
            pair_normals_x2(key, c0, t, c2, kStreamDyn, bk + (uint32_t)hp, zv2[hp], zw2[hp]);
            const float amp = par<float>(mp, 6);
            const float2 I = make_float2((on && row < blk && col + 2 * hp < blk) ? amp : 0.0f,
                                         (on && row < blk && col + 2 * hp + 1 < blk) ? amp : 0.0f);
            const float2 vv = make_float2(v[2 * hp], v[2 * hp + 1]), ww = make_float2(w[2 * hp], w[2 * hp + 1]);
            const float2 fv = fhn_drift_v_x2(mp, vv, ww, lap2[hp], I), fw = fhn_drift_w_x2(mp, vv, ww);
            mv2[hp] = __ffma2_rn(f2s(dt), fv, vv);
            mw2[hp] = __ffma2_rn(f2s(dt), fw, ww);
            bv2[hp] = __ffma2_rn(f2s(h), zv2[hp], mv2[hp]);  // = em_update
            bw2[hp] = __ffma2_rn(f2s(h), zw2[hp], mw2[hp]);
        }
        const float *y = obs + (obs_stride ? (int64_t)m * obs_stride : 0);
        const float inv_h = 1.0f / h;
        float nvs[4], nws[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int node = n0 + e, hp = e >> 1;
            const bool hi = e & 1;
            const float mv = hi ? mv2[hp].y : mv2[hp].x, mw = hi ? mw2[hp].y : mw2[hp].x;
            const float zv = hi ? zv2[hp].y : zv2[hp].x, zw = hi ? zw2[hp].y : zw2[hp].x;
            const float bv = hi ? bv2[hp].y : bv2[hp].x, bw = hi ? bw2[hp].y : bw2[hp].x;
            float nv = bv, nw = bw;
            const int j = obs_slot[node];
            if (j >= 0) {
                float o[4] = {0.f, 0.f, 0.f, 0.f};
                if (mlp_out) {
                    const float4 oo = reinterpret_cast<const float4 *>(mlp_out)[p * dy + j];
                    o[0] = oo.x; o[1] = oo.y; o[2] = oo.z; o[3] = oo.w;
                }
                const float mc[2] = {mv, mw}, zc[2] = {zv, zw};
                float xn[2];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const float os = fminf(fmaxf(o[2 + cc], -mlp::kClamp), mlp::kClamp);
                    const float mu = __fmaf_rn(h, o[cc], mc[cc]);
                    const float es = __expf(os);
                    const float sd = h * es;
                    xn[cc] = __fmaf_rn(sd, zc[cc], mu);
                    const float t1 = (xn[cc] - mc[cc]) * inv_h, t2 = (xn[cc] - mu) * (inv_h / es);
                    lw[hp] += os + 0.5f * (t2 * t2 - t1 * t1);
                }
                nv = xn[0];
                nw = xn[1];
                const int64_t oj = (p * dy + j) * 2;
                xboot[oj] = bv;
                xboot[oj + 1] = bw;
                mp_obs[oj] = mv;
                mp_obs[oj + 1] = mw;
                const float ep = y[j] - nv, eb = y[j] - bv;
                part_prop[hp] += ep * ep;
                part_boot[hp] += eb * eb;
            }
            nvs[e] = nv;
            nws[e] = nw;
        }
        float *xo = x + p * (int64_t)mp.dx;
        *reinterpret_cast<float4 *>(xo + n0) = make_float4(nvs[0], nvs[1], nvs[2], nvs[3]);
        *reinterpret_cast<float4 *>(xo + nn + n0) = make_float4(nws[0], nws[1], nws[2], nws[3]);
    }
    // per-pair partials, then per particle in the pair kernel's order
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);  // [3][ppc][pairs]
    const int np = ppc * pairs;
    if (active) {
#pragma unroll
        for (int hp = 0; hp < 2; ++hp) {
            red[s * pairs + 2 * q + hp] = part_prop[hp];
            red[np + s * pairs + 2 * q + hp] = part_boot[hp];
            red[2 * np + s * pairs + 2 * q + hp] = lw[hp];
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sl = warp; sl < ppc; sl += nwarps) {
        const int64_t pp = (int64_t)blockIdx.x * ppc + sl;
        float a = 0.0f, b = 0.0f, c = 0.0f;
        for (int i = lane; i < pairs; i += 32) {
            a += red[sl * pairs + i];
            b += red[np + sl * pairs + i];
            c += red[2 * np + sl * pairs + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0 && pp < P) {
            // the sub-step's sum of log p - log q joins those of the span's earlier sub-steps
            const float cs = first ? c : lw_acc[pp] + c;
            if (last) {
                logw[pp] = mp.fhalf_prec * a + cs;
                logw_boot[pp] = mp.fhalf_prec * b;
            } else {
                lw_acc[pp] = cs;
            }
        }
    }
}

// Per filter: the ESS of the proposal weights; below ess_frac N the step takes
// the transition's candidates and weights instead (the bootstrap fallback).
// Also sets the filter's maximum log-weight for the resampling chain.
__global__ void __launch_bounds__(256) k_proposal_select(const FilterDesc *filt, ModelParams mp, float ess_frac,
                                                         int32_t use_proposal, float *logw, const float *logw_boot,
                                                         float *x, const float *xboot, const int32_t *obs_idx,
                                                         int32_t *fmax_key, double *fstats)
{
    __shared__ float shf[2][8];
    __shared__ double shd[2][8];
    __shared__ int fallback;
    const FilterDesc fd = filt[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    float mp_ = -INFINITY, mb = -INFINITY;
    for (int i = tid; i < fd.N; i += blockDim.x) {
        const float a = logw[fd.off + i], b = logw_boot[fd.off + i];
        if (a < INFINITY) mp_ = fmaxf(mp_, a);
        if (b < INFINITY) mb = fmaxf(mb, b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mp_ = fmaxf(mp_, __shfl_xor_sync(0xffffffffu, mp_, o));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if (lane == 0) {
        shf[0][wid] = mp_;
        shf[1][wid] = mb;
    }
    __syncthreads();
    mp_ = shf[0][0];
    mb = shf[1][0];
    for (int i = 1; i < nw; ++i) {
        mp_ = fmaxf(mp_, shf[0][i]);
        mb = fmaxf(mb, shf[1][i]);
    }
    if (use_proposal) {
        double s1 = 0.0, s2 = 0.0;  // few particles per thread: FP64 directly
        if (mp_ > -INFINITY)
            for (int i = tid; i < fd.N; i += blockDim.x) {
                const float l = logw[fd.off + i];
                const double wv = (l > -INFINITY && l < INFINITY) ? (double)expf(l - mp_) : 0.0;
                s1 += wv;
                s2 += wv * wv;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            shd[0][wid] = s1;
            shd[1][wid] = s2;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int i = 0; i < nw; ++i) {
                a += shd[0][i];
                b += shd[1][i];
            }
            const double ess = b > 0.0 ? a * a / b : 0.0;
            fallback = ess < (double)ess_frac * (double)fd.N;
        }
    } else if (tid == 0) {
        fallback = 1;  // recording without a network: the transition's step
    }
    __syncthreads();
    if (fallback)  // the observed nodes follow in k_proposal_fixup
        for (int i = tid; i < fd.N; i += blockDim.x) logw[fd.off + i] = logw_boot[fd.off + i];
    if (tid == 0) {
        const float mx = fallback ? mb : mp_;
        fmax_key[blockIdx.x] = mx > -INFINITY ? float_order_key(mx) : kNegInfKey;
        fstats[(int64_t)blockIdx.x * kFsCount + kFsFallback] = (use_proposal && fallback) ? 1.0 : 0.0;
    }
}

// The fallback's state: for particles of filters that took the transition's
// step, the observed nodes get the transition's candidates (grid-wide, one
// thread per (particle, observed node), so the copy is as parallel as the data).
__global__ void __launch_bounds__(256) k_proposal_fixup(const int32_t *__restrict__ pfilt, ModelParams mp, int64_t P,
                                                        const double *__restrict__ fstats, float *x,
                                                        const float *__restrict__ xboot,
                                                        const int32_t *__restrict__ obs_idx)
{
    const int dy = mp.dy;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * dy) return;
    const int64_t p = e / dy;
    if (fstats[(int64_t)pfilt[p] * kFsCount + kFsFallback] == 0.0) return;
    const int j = (int)(e - p * dy), nd = obs_idx[j], nn = mp.J * mp.J;
    x[p * mp.dx + nd] = xboot[e * 2];
    x[p * mp.dx + nn + nd] = xboot[e * 2 + 1];
}

// Training tuples from the resampled particles: for every kept particle i
// (filter-local index a multiple of `stride`) and observed node j, the
// network input of its ancestor and the standardised residual of its node
// (x_new - m) / h.  Slot (rec_base + (sel_off[m] + i / stride) dy + j).
__global__ void k_gather_tuples(ModelParams mp, const FilterDesc *filt, const int32_t *pfilt, const int32_t *anc,
                                const float *x_new, int64_t P, const int32_t *obs_idx,
                                const __nv_bfloat16 *rows, const float *mp_obs, int32_t stride,
                                const int64_t *sel_off, int64_t rec_base, int64_t cap, float *X, float *R)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int dy = mp.dy;
    if (gid >= P * dy) return;
    const int64_t p = gid / dy;
    const int j = (int)(gid - p * dy);
    const int32_t m = pfilt[p];
    const int64_t i = p - filt[m].off;
    if (i % stride) return;
    const int64_t k = rec_base + (sel_off[m] + i / stride) * dy + j;
    if (k >= cap) return;
    const int64_t src = filt[m].off + anc[p];
    const __nv_bfloat16 *row = rows + (src * dy + j) * mlp::kInPad;
    for (int c = 0; c < mlp::kIn; ++c) X[k * mlp::kIn + c] = __bfloat162float(row[c]);
    const int nn = mp.J * mp.J, nd = obs_idx[j];
    const float inv_h = 1.0f / mp.fsq;
    R[k * 2] = (x_new[p * mp.dx + nd] - mp_obs[(src * dy + j) * 2]) * inv_h;
    R[k * 2 + 1] = (x_new[p * mp.dx + nn + nd] - mp_obs[(src * dy + j) * 2 + 1]) * inv_h;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_propagate_split(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *x,
                                   const int32_t *gather, cudaStream_t s)
{
    const int pairs = c.mp.J * c.mp.J / 2;
    int n = 1;
    while ((n + 1) * pairs <= 1024 && n < 8) ++n;
    if (c.fhn_ppc > 0 && c.fhn_ppc < n) n = c.fhn_ppc;
    const int ppc = n;
    const int threads = (ppc * pairs + 31) / 32 * 32;
    const unsigned grid = (unsigned)((c.P + ppc - 1) / ppc);
    // K - L ordinary sub-steps (no weights yet), L = the proposal's span; recording builds its
    // network inputs at the same place (without a network the span's sub-steps are the transition's)
    const int L = c.prop_span;
    if (c.mp.K > L) {
        cudaError_t e = launch_fhn_substeps(c, d_obs, stride, xi, x, gather, c.mp.K - L, s);
        if (e != cudaSuccess) return e;
    } else if (xi != x || gather) {
        return cudaErrorInvalidValue;  // a span of the whole interval steps in place
    }
    const float *mo = nullptr;
    if (c.rec_X) {  // the recorded tuples need the rows themselves
        const int64_t R = c.P * c.mp.dy;
        k_build_rows<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(c.mp, x, c.P, c.pfilt, c.obs_idx, d_obs, stride,
                                                                 c.rows);
    }
    if (c.prop_on) {  // rows built inside the tensor-core forward
        cudaError_t e = launch_proposal_forward_tc(c.mp.J, c.mp.dx, c.mp.dy, x, c.P, c.pfilt, c.obs_idx, d_obs, stride,
                                                   c.wpack, c.theta, c.mlp_out, c.err, s);
        if (e != cudaSuccess) return e;
        mo = c.mlp_out;
    }
    if ((c.fhn_nodes != 2 || L > 1) && c.mp.J % 4 == 0) {  // four nodes per thread, as the sub-steps
        const int quads = c.mp.J * c.mp.J / 4;
        int n4 = 1;
        while ((n4 + 1) * quads <= kLast4MaxThreads && n4 < 8) ++n4;
        if (c.fhn_ppc > 0 && c.fhn_ppc < n4) n4 = c.fhn_ppc;
        const int threads4 = (n4 * quads + 31) / 32 * 32;
        const unsigned grid4 = (unsigned)((c.P + n4 - 1) / n4);
        const size_t smem4 = (size_t)3 * n4 * pairs * sizeof(float);  // >= the v-planes (n4 * J * J floats)
        for (int k = c.mp.K - L; k < c.mp.K; ++k) {
            const int32_t first = k == c.mp.K - L, last = k == c.mp.K - 1;
            if (c.fhn_quad_ctas == 4)
                k_last_step_fhn4<4><<<grid4, threads4, smem4, s>>>(c.mp, c.key, c.pfilt, c.filt, x, c.P, d_obs, stride,
                                                                   c.obs_slot, c.d_t, n4, mo, c.xboot, c.mp_obs,
                                                                   c.logw, c.logw_boot, k, first, last, c.lw_acc);
            else
                k_last_step_fhn4<3><<<grid4, threads4, smem4, s>>>(c.mp, c.key, c.pfilt, c.filt, x, c.P, d_obs, stride,
                                                                   c.obs_slot, c.d_t, n4, mo, c.xboot, c.mp_obs,
                                                                   c.logw, c.logw_boot, k, first, last, c.lw_acc);
        }
    } else {
        const size_t smem_last = std::max((size_t)ppc * pairs * sizeof(float2), (size_t)3 * threads * sizeof(float));
        k_last_step_fhn<<<grid, threads, smem_last, s>>>(c.mp, c.key, c.pfilt, c.filt, x, c.P, d_obs, stride,
                                                         c.obs_slot, c.d_t, ppc, mo, c.xboot, c.mp_obs, c.logw,
                                                         c.logw_boot);
    }
    // a fallback needs the transition's candidates from the same state: only for a span of one
    const float ess_frac = L == 1 ? c.prop_ess_frac : 0.0f;
    k_proposal_select<<<c.M, 256, 0, s>>>(c.filt, c.mp, ess_frac, c.prop_on ? 1 : 0, c.logw, c.logw_boot, x,
                                          c.xboot, c.obs_idx, c.fmax_key, c.fstats);
    const int64_t rows = c.P * c.mp.dy;
    k_proposal_fixup<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(c.pfilt, c.mp, c.P, c.fstats, x, c.xboot,
                                                                  c.obs_idx);
    return cudaGetLastError();
}

cudaError_t launch_gather_tuples(const Ctx &c, const float *x_new, cudaStream_t s)
{
    const int64_t n = c.P * c.mp.dy;
    k_gather_tuples<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.mp, c.filt, c.pfilt, c.anc, x_new, c.P, c.obs_idx,
                                                                 c.rows, c.mp_obs, c.rec_stride, c.rec_sel_off,
                                                                 c.rec_count, c.rec_cap, c.rec_X, c.rec_R);
    return cudaGetLastError();
}

}  // namespace pf
