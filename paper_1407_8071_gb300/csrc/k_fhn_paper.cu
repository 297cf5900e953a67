// k_fhn_paper.cu -- the paper's own stochastic FitzHugh-Nagumo lattice
// (Sec. 5.1, eqs. eqUd, eqVd, eqStimulusRegion-eqPsi_ijt; set-up of Sec. 5.2)
// on the GPU: per node U, V and S (sub-steps since the node's last random
// stimulus, capped at l0), Euler steps of
//   U <- U + dt (p3(U) - V + (1/D) sum_nbr U + m F_n + Psi) + sigma sqrt(dt) z,
//   V <- V + dt (b0 U + b1 V + b2),
// Psi = amplitude while S < l0, forcing pulses on the first columns, and the
// random stimulus before each sub-step: with probability eps one node of the
// stimulus region (nodes whose U, or a neighbour's U, lies in (u-, u+)),
// chosen uniformly, and its neighbours restart their S at 0.
//
// Layout as k_propagate_fhn: thread (slot s, pair q) carries nodes 2q, 2q+1
// of particle blockIdx.x * ppc + s; the U plane sits in shared memory as
// pairs (double-buffered, one barrier per sub-step).  A slot's leader draws
// the stimulus numbers; only when some particle of the CTA has an event do
// the threads count the region (shared atomics) and find the chosen node by
// a block-wide exclusive scan over the pair order (= row-major node order).
// Noise: normal 2 node of block k dx / 4 + q (the pair's U lanes 0 and 2; V
// takes no noise); stimulus numbers: Philox block (c0, t, c2, stim << 24 | k).
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "lattice.cuh"
#include "pf.h"
#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kMaxSlots = 8;

template <typename Real>
__device__ __forceinline__ Real fhnp_p3(const ModelParams &mp, Real u)
{
    return ((par<Real>(mp, 0) * u + par<Real>(mp, 1)) * u + par<Real>(mp, 2)) * u + par<Real>(mp, 3);
}

template <typename Real>
__device__ __forceinline__ bool in_band(const ModelParams &mp, Real u)
{
    return u > par<Real>(mp, 12) && u < par<Real>(mp, 13);
}

// Exclusive scan of one int per thread over the whole block (thread order);
// `warp_tot` holds 32 ints.  Every thread must call it.
__device__ int block_exclusive_scan(int v, int *warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int before = 0;
    for (int i = 0; i < w; ++i) before += warp_tot[i];
    (void)nw;
    return before + x - v;
}

}  // namespace

// MaxT / MinB: the filters' build for lattices whose particle fits 512 threads
// (J <= 32) is <512, 3> -- at most 40 registers, three CTAs per SM: with one
// Euler step per observation the kernel streams the state and needs the warps
// to hide its loads; larger lattices and the FP64 truth record use <1024, 1>.
template <typename Real, int MaxT = 1024, int MinB = 1>
__global__ void __launch_bounds__(MaxT, MinB)
    k_propagate_fhnp(ModelParams mp, Key key, uint32_t stream, uint32_t stim_stream, const int32_t *pfilt,
                     const FilterDesc *filt, const Real *x_in, Real *x_out, int64_t P,
                     float *logw, const float *obs, int32_t obs_stride, const int32_t *obs_slot, const int32_t *d_t,
                     int32_t fixed_c0, int32_t fixed_c2, int32_t t_direct, int32_t ppc, int32_t *fmax_key,
                     int32_t n_steps, AuxPtrs aux, int32_t noise)
{
    using Pair = typename std::conditional<std::is_same<Real, float>::value, float2, double2>::type;
    extern __shared__ unsigned char smem_raw[];
    __shared__ int sh_ev[2][kMaxSlots], sh_cnt[2][kMaxSlots], sh_target[2][kMaxSlots], sh_base[kMaxSlots];
    __shared__ uint32_t sh_r1[2][kMaxSlots];
    __shared__ int warp_tot[32];
    const int J = mp.J, nn = J * J, pairs = nn / 2, half = J / 2;
    Pair *sv = reinterpret_cast<Pair *>(smem_raw);  // [2][ppc][pairs]
    const int slot = (int)threadIdx.x / pairs;
    const int s = min(slot, ppc);                   // s == ppc: padding thread
    const int q = threadIdx.x - min(slot, ppc - 1) * pairs;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(d_t ? *d_t + 1 : t_direct);

    uint32_t c0 = 0, c2 = 0;
    Real u0 = 0, u1 = 0, v0 = 0, v1 = 0, s0 = 0, s1 = 0;
    const int n0 = 2 * q, row = n0 / J, col = n0 - row * J;
    if (active) {
        if (pfilt) {
            const int32_t m = pfilt[p];
            c0 = (uint32_t)(p - filt[m].off);
            c2 = (uint32_t)m;
        } else {
            c0 = (uint32_t)fixed_c0;
            c2 = (uint32_t)fixed_c2;
        }
        const int64_t row_in = aux.gather ? filt[pfilt[p]].off + aux.gather[p] : p;
        const Pair *xi = reinterpret_cast<const Pair *>(x_in + row_in * (int64_t)mp.dx + n0);  // n0, nn even
        const Pair a = xi[0], b = xi[nn / 2], c = xi[nn];
        u0 = a.x;
        u1 = a.y;
        v0 = b.x;
        v1 = b.y;
        s0 = c.x;
        s1 = c.y;
    }
    const Real dt = par_dt<Real>(mp), sq = par_sq<Real>(mp), coup = par<Real>(mp, 7);
    const Real b0 = par<Real>(mp, 4), b1 = par<Real>(mp, 5), b2 = par<Real>(mp, 6);
    const Real Ff = par<Real>(mp, 8), Fpsi = par<Real>(mp, 15), l0 = par<Real>(mp, 16);
    const int64_t period = mp.ip[9], width = mp.ip[10];
    const int fcols = (int)mp.ip[11];
    const uint32_t eps_thr = (uint32_t)mp.ip[14];
    const int64_t n_base = (int64_t)(t - 1) * mp.K;  // (n - 1) of sub-step k is n_base + k
    // (n_base + k) mod period, advanced per sub-step; 32-bit division when both fit
    int64_t phase = (n_base < 0x7FFFFFFF && period < 0x7FFFFFFF)
                        ? (int64_t)((uint32_t)n_base % (uint32_t)period) : n_base % period;
    const uint32_t blocks_per_step = (uint32_t)(mp.dx / 4);
    const bool has_up = row > 0, has_dn = row < J - 1, has_left = col > 0, has_right = col + 2 < J;
    const int qu = has_up ? q - half : q, qd = has_dn ? q + half : q;
    const int ql = has_left ? q - 1 : q, qr = has_right ? q + 1 : q;

    for (int k = 0; k < n_steps; ++k) {
        const int par_k = k & 1;
        Pair *buf = sv + (par_k * ppc + (active ? s : 0)) * pairs;
        if (active) {
            Pair mine;
            mine.x = u0;
            mine.y = u1;
            buf[q] = mine;
            if (q == 0) {  // the slot's stimulus numbers
                int ev = 0;
                uint32_t r1 = 0;
                if (noise) {
                    const uint4 r = philox4x32_10(make_uint4(c0, t, c2, (stim_stream << 24) | (uint32_t)k), key);
                    ev = (r.x >> 8) < eps_thr;
                    r1 = r.y;
                }
                sh_ev[par_k][s] = ev;
                sh_r1[par_k][s] = r1;
                sh_cnt[par_k][s] = 0;
                sh_target[par_k][s] = -1;
            }
        }
        __syncthreads();
        int any = 0;
        for (int i = 0; i < ppc; ++i) any |= sh_ev[par_k][i];
        Pair up, dn, lf, rt;
        if (active) {
            up = buf[qu];
            dn = buf[qd];
            lf = buf[ql];
            rt = buf[qr];
        }
        bool hit0 = false, hit1 = false;
        if (any) {  // uniform over the CTA
            int f0 = 0, f1 = 0;
            if (active && sh_ev[par_k][s]) {
                const Real left = has_left ? lf.y : u0, right = has_right ? rt.x : u1;
                f0 = in_band<Real>(mp, u0) || in_band<Real>(mp, u1) || (has_left && in_band<Real>(mp, left)) ||
                     (has_up && in_band<Real>(mp, up.x)) || (has_dn && in_band<Real>(mp, dn.x));
                f1 = in_band<Real>(mp, u1) || in_band<Real>(mp, u0) || (has_right && in_band<Real>(mp, right)) ||
                     (has_up && in_band<Real>(mp, up.y)) || (has_dn && in_band<Real>(mp, dn.y));
            }
            const int c = f0 + f1;
            if (c) atomicAdd(&sh_cnt[par_k][s], c);
            const int excl = block_exclusive_scan(c, warp_tot);
            if (active && q == 0) sh_base[s] = excl;
            __syncthreads();
            if (active && sh_ev[par_k][s] && c) {
                const int cnt = sh_cnt[par_k][s];
                const int rank = (int)(((uint64_t)(sh_r1[par_k][s] >> 8) * (uint64_t)cnt) >> 24);
                const int local = excl - sh_base[s];
                if (rank >= local && rank < local + c) {
                    const int node = (rank == local) ? (f0 ? n0 : n0 + 1) : n0 + 1;
                    sh_target[par_k][s] = node;
                }
            }
            __syncthreads();
            if (active) {
                const int tg = sh_target[par_k][s];
                if (tg >= 0) {
                    const int ti = tg / J, tj = tg - (tg / J) * J;
                    hit0 = (row == ti && (col == tj || col == tj - 1 || col == tj + 1)) ||
                           (col == tj && (row == ti - 1 || row == ti + 1));
                    hit1 = (row == ti && (col + 1 == tj || col + 1 == tj - 1 || col + 1 == tj + 1)) ||
                           (col + 1 == tj && (row == ti - 1 || row == ti + 1));
                }
            }
        }
        if (active) {
            s0 = hit0 ? (Real)0 : (s0 + (Real)1 < l0 ? s0 + (Real)1 : l0);
            s1 = hit1 ? (Real)0 : (s1 + (Real)1 < l0 ? s1 + (Real)1 : l0);
            Real z[4] = {(Real)0, (Real)0, (Real)0, (Real)0};
            if (noise) normals4<Real>(key, c0, t, c2, stream, (uint32_t)k * blocks_per_step + (uint32_t)q, z);
            // (1/D) times the sum over the existing von Neumann neighbours (Sec. 5.2's sets)
            Real nb0 = (has_up ? up.x : (Real)0) + (has_dn ? dn.x : (Real)0);
            nb0 = nb0 + (has_left ? lf.y : (Real)0) + u1;
            Real nb1 = (has_up ? up.y : (Real)0) + (has_dn ? dn.y : (Real)0);
            nb1 = nb1 + u0 + (has_right ? rt.x : (Real)0);
            const bool on = phase < width;
            const Real F0 = (on && col < fcols) ? Ff : (Real)0, F1 = (on && col + 1 < fcols) ? Ff : (Real)0;
            const Real P0 = s0 < l0 ? Fpsi : (Real)0, P1 = s1 < l0 ? Fpsi : (Real)0;
            const Real fu0 = fhnp_p3<Real>(mp, u0) - v0 + coup * nb0 + F0 + P0;
            const Real fu1 = fhnp_p3<Real>(mp, u1) - v1 + coup * nb1 + F1 + P1;
            const Real fv0 = b0 * u0 + b1 * v0 + b2, fv1 = b0 * u1 + b1 * v1 + b2;
            u0 = em_update(u0, fu0, z[0], dt, sq);
            u1 = em_update(u1, fu1, z[2], dt, sq);
            v0 = em_update(v0, fv0, (Real)0, dt, sq);
            v1 = em_update(v1, fv1, (Real)0, dt, sq);
        }
        if (++phase == period) phase = 0;
    }
    if (active && x_out) {
        Pair *xo = reinterpret_cast<Pair *>(x_out + p * (int64_t)mp.dx + n0);
        Pair a, b, c;
        a.x = u0, a.y = u1;
        b.x = v0, b.y = v1;
        c.x = s0, c.y = s1;
        xo[0] = a;
        xo[nn / 2] = b;
        xo[nn] = c;
    }
    if (!logw) return;
    // log-likelihood over the observed U nodes, per particle, fixed order (as the RM kernel)
    float part = 0.0f;
    if (active) {
        const int32_t m = pfilt ? pfilt[p] : 0;
        const float *y = obs + (obs_stride ? (int64_t)m * obs_stride : 0);
        const int j0 = obs_slot[n0], j1 = obs_slot[n0 + 1];
        if (j0 >= 0) { const float e = y[j0] - (float)u0; part += e * e; }
        if (j1 >= 0) { const float e = y[j1] - (float)u1; part += e * e; }
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);
    red[threadIdx.x] = part;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sl = warp; sl < ppc; sl += nwarps) {
        const int64_t pp = (int64_t)blockIdx.x * ppc + sl;
        float acc = 0.0f;
        for (int i = lane; i < pairs; i += 32) acc += red[sl * pairs + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && pp < P) {
            float l = mp.fhalf_prec * acc;
            if (aux.la_out) {
                aux.la_out[pp] = l;
                l = aux.lw_prev[pp] + l;
            } else if (aux.la_src) {
                l -= aux.la_src[filt[pfilt[pp]].off + aux.anc[pp]];
            }
            logw[pp] = l;
            if (l > -INFINITY && l < INFINITY) atomicMax(&fmax_key[pfilt[pp]], float_order_key(l));
        }
    }
}

// The same interval in FP32 with 4G consecutive nodes of a row per thread
// (lattice sides divisible by 4G): thread (slot s, unit q) carries nodes
// 4Gq..4Gq+4G-1, i.e. the pairs 2Gq..2Gq+2G-1 of k_propagate_fhnp, with their
// Philox blocks, the same per-node arithmetic in the same order, the same
// stimulus selection (row-major rank over the region) and the same
// per-particle sum over pair partials, so its results are the pair kernel's
// bits.  With one Euler step per observation a thread's fixed cost (indices,
// parameters, the filter lookup, the barriers) is spread over 4G nodes
// instead of two.  MinB: CTAs per SM the compiler must fit.  JT: the lattice
// side fixed at compile time (0: mp.J), so that the index divisions of a
// one-sub-step launch become shifts.
template <int MinB, int G, int JT = 0>
__global__ void __launch_bounds__(kFhnp4MaxThreads, MinB)
    k_propagate_fhnp4(ModelParams mp, Key key, uint32_t stream, uint32_t stim_stream, const int32_t *pfilt,
                      const FilterDesc *filt, const float *x_in, float *x_out, int64_t P, float *logw,
                      const float *obs, int32_t obs_stride, const int32_t *obs_slot, const int32_t *d_t, int32_t ppc,
                      int32_t *fmax_key, int32_t n_steps, AuxPtrs aux, int32_t noise)
{
    constexpr int NV = 4 * G;
    extern __shared__ unsigned char smem_raw[];
    __shared__ int sh_ev[2][kMaxSlots], sh_cnt[2][kMaxSlots], sh_target[2][kMaxSlots], sh_base[kMaxSlots];
    __shared__ uint32_t sh_r1[2][kMaxSlots];
    __shared__ int warp_tot[32];
    const int J = JT ? JT : mp.J, nn = J * J, units = nn / NV, pairs = nn / 2, urow = J / NV;
    float4 *sv = reinterpret_cast<float4 *>(smem_raw);  // [2][ppc][units][G]
    const int slot = (int)threadIdx.x / units;
    const int s = min(slot, ppc);  // s == ppc: padding thread
    const int q = threadIdx.x - min(slot, ppc - 1) * units;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(*d_t + 1);

    uint32_t c0 = 0, c2 = 0;
    float u[NV], v[NV], sc[NV];
#pragma unroll
    for (int e = 0; e < NV; ++e) u[e] = v[e] = sc[e] = 0.0f;
    const int n0 = NV * q, row = n0 / J, col = n0 - row * J;
    if (active) {
        const int32_t m = pfilt[p];
        c0 = (uint32_t)(p - filt[m].off);
        c2 = (uint32_t)m;
        const int64_t row_in = aux.gather ? filt[m].off + aux.gather[p] : p;
        const float *xi = x_in + row_in * (int64_t)mp.dx + n0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float4 a = *reinterpret_cast<const float4 *>(xi + 4 * g);
            const float4 b = *reinterpret_cast<const float4 *>(xi + nn + 4 * g);
            const float4 c = *reinterpret_cast<const float4 *>(xi + 2 * nn + 4 * g);
            u[4 * g] = a.x; u[4 * g + 1] = a.y; u[4 * g + 2] = a.z; u[4 * g + 3] = a.w;
            v[4 * g] = b.x; v[4 * g + 1] = b.y; v[4 * g + 2] = b.z; v[4 * g + 3] = b.w;
            sc[4 * g] = c.x; sc[4 * g + 1] = c.y; sc[4 * g + 2] = c.z; sc[4 * g + 3] = c.w;
        }
    }
    const float dt = par_dt<float>(mp), sq = par_sq<float>(mp), coup = par<float>(mp, 7);
    const float b0 = par<float>(mp, 4), b1 = par<float>(mp, 5), b2 = par<float>(mp, 6);
    const float Ff = par<float>(mp, 8), Fpsi = par<float>(mp, 15), l0 = par<float>(mp, 16);
    const int64_t period = mp.ip[9], width = mp.ip[10];
    const int fcols = (int)mp.ip[11];
    const uint32_t eps_thr = (uint32_t)mp.ip[14];
    const int64_t n_base = (int64_t)(t - 1) * mp.K;
    int64_t phase = (n_base < 0x7FFFFFFF && period < 0x7FFFFFFF)
                        ? (int64_t)((uint32_t)n_base % (uint32_t)period) : n_base % period;
    const uint32_t blocks_per_step = (uint32_t)(mp.dx / 4);
    const bool has_up = row > 0, has_dn = row < J - 1, has_left = col > 0, has_right = col + NV < J;
    const int qu = has_up ? q - urow : q, qd = has_dn ? q + urow : q;
    const int ql = has_left ? q - 1 : q, qr = has_right ? q + 1 : q;

    for (int k = 0; k < n_steps; ++k) {
        const int par_k = k & 1;
        float4 *buf = sv + (par_k * ppc + (active ? s : 0)) * units * G;
        if (active) {
#pragma unroll
            for (int g = 0; g < G; ++g) buf[q * G + g] = make_float4(u[4 * g], u[4 * g + 1], u[4 * g + 2], u[4 * g + 3]);
            if (q == 0) {  // the slot's stimulus numbers
                int ev = 0;
                uint32_t r1 = 0;
                if (noise) {
                    const uint4 r = philox4x32_10(make_uint4(c0, t, c2, (stim_stream << 24) | (uint32_t)k), key);
                    ev = (r.x >> 8) < eps_thr;
                    r1 = r.y;
                }
                sh_ev[par_k][s] = ev;
                sh_r1[par_k][s] = r1;
                sh_cnt[par_k][s] = 0;
                sh_target[par_k][s] = -1;
            }
        }
        __syncthreads();
        int any = 0;
        for (int i = 0; i < ppc; ++i) any |= sh_ev[par_k][i];
        // (1/D) times the sum over the existing von Neumann neighbours (Sec. 5.2's sets),
        // formed at once so that the neighbour values die here
        float nb[NV];
        if (active) {
            const float left = has_left ? buf[ql * G + G - 1].w : 0.0f, right = has_right ? buf[qr * G].x : 0.0f;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float4 up = buf[qu * G + g], dn = buf[qd * G + g];
                const float uu[4] = {up.x, up.y, up.z, up.w}, dd[4] = {dn.x, dn.y, dn.z, dn.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = 4 * g + i;
                    float a = (has_up ? uu[i] : 0.0f) + (has_dn ? dd[i] : 0.0f);
                    a = a + (e > 0 ? u[e - 1] : left);
                    nb[e] = a + (e < NV - 1 ? u[e + 1] : right);
                }
            }
        }
        uint32_t hit = 0;  // bit e: node e restarts its stimulus counter
        if (any) {         // uniform over the CTA (rare): the neighbours again from shared memory
            uint32_t f = 0;
            if (active && sh_ev[par_k][s]) {
                const float *bf = reinterpret_cast<const float *>(buf);
                const float left = has_left ? bf[ql * NV + NV - 1] : u[0];
                const float right = has_right ? bf[qr * NV] : u[NV - 1];
                for (int e = 0; e < NV; ++e) {
                    const bool in = in_band<float>(mp, u[e]) ||
                                    (e > 0 ? in_band<float>(mp, u[e - 1]) : (has_left && in_band<float>(mp, left))) ||
                                    (e < NV - 1 ? in_band<float>(mp, u[e + 1])
                                                : (has_right && in_band<float>(mp, right))) ||
                                    (has_up && in_band<float>(mp, bf[qu * NV + e])) ||
                                    (has_dn && in_band<float>(mp, bf[qd * NV + e]));
                    f |= (uint32_t)in << e;
                }
            }
            const int c = __popc(f);
            if (c) atomicAdd(&sh_cnt[par_k][s], c);
            const int excl = block_exclusive_scan(c, warp_tot);
            if (active && q == 0) sh_base[s] = excl;
            __syncthreads();
            if (active && sh_ev[par_k][s] && c) {
                const int cnt = sh_cnt[par_k][s];
                const int rank = (int)(((uint64_t)(sh_r1[par_k][s] >> 8) * (uint64_t)cnt) >> 24);
                const int local = excl - sh_base[s];
                if (rank >= local && rank < local + c) {
                    uint32_t rest = f;  // the (rank - local)-th set node, in row-major order
                    for (int i = local; i < rank; ++i) rest &= rest - 1;
                    sh_target[par_k][s] = n0 + __ffs(rest) - 1;
                }
            }
            __syncthreads();
            if (active) {
                const int tg = sh_target[par_k][s];
                if (tg >= 0) {
                    const int ti = tg / J, tj = tg - (tg / J) * J;
                    for (int e = 0; e < NV; ++e) {
                        const int ce = col + e;
                        const bool h = (row == ti && (ce == tj || ce == tj - 1 || ce == tj + 1)) ||
                                       (ce == tj && (row == ti - 1 || row == ti + 1));
                        hit |= (uint32_t)h << e;
                    }
                }
            }
        }
        if (active) {
            const bool on = phase < width;
#pragma unroll
            for (int h = 0; h < NV / 2; ++h) {  // pair h: nodes 2h, 2h + 1 and their Philox block
                float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (noise)
                    normals4<float>(key, c0, t, c2, stream,
                                    (uint32_t)k * blocks_per_step + (uint32_t)(NV / 2) * (uint32_t)q + (uint32_t)h, z);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int e = 2 * h + i;
                    sc[e] = ((hit >> e) & 1) ? 0.0f : (sc[e] + 1.0f < l0 ? sc[e] + 1.0f : l0);
                    const float F = (on && col + e < fcols) ? Ff : 0.0f, Ps = sc[e] < l0 ? Fpsi : 0.0f;
                    const float fu = fhnp_p3<float>(mp, u[e]) - v[e] + coup * nb[e] + F + Ps;
                    const float fv = b0 * u[e] + b1 * v[e] + b2;
                    u[e] = em_update(u[e], fu, z[2 * i], dt, sq);
                    v[e] = em_update(v[e], fv, 0.0f, dt, sq);
                }
            }
        }
        if (++phase == period) phase = 0;
    }
    if (active && x_out) {
        float *xo = x_out + p * (int64_t)mp.dx + n0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            *reinterpret_cast<float4 *>(xo + 4 * g) = make_float4(u[4 * g], u[4 * g + 1], u[4 * g + 2], u[4 * g + 3]);
            *reinterpret_cast<float4 *>(xo + nn + 4 * g) =
                make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
            *reinterpret_cast<float4 *>(xo + 2 * nn + 4 * g) =
                make_float4(sc[4 * g], sc[4 * g + 1], sc[4 * g + 2], sc[4 * g + 3]);
        }
    }
    if (!logw) return;
    float part[NV / 2];
#pragma unroll
    for (int h = 0; h < NV / 2; ++h) part[h] = 0.0f;
    if (active) {
        const float *y = obs + (obs_stride ? (int64_t)pfilt[p] * obs_stride : 0);
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const int j = obs_slot[n0 + e];
            if (j >= 0) {
                const float d = y[j] - u[e];
                part[e >> 1] += d * d;
            }
        }
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);  // [ppc][pairs], the pair kernel's order
    if (active)
#pragma unroll
        for (int h = 0; h < NV / 2; ++h) red[s * pairs + (NV / 2) * q + h] = part[h];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sl = warp; sl < ppc; sl += nwarps) {
        const int64_t pp = (int64_t)blockIdx.x * ppc + sl;
        float acc = 0.0f;
        for (int i = lane; i < pairs; i += 32) acc += red[sl * pairs + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && pp < P) {
            float l = mp.fhalf_prec * acc;
            if (aux.la_out) {
                aux.la_out[pp] = l;
                l = aux.lw_prev[pp] + l;
            } else if (aux.la_src) {
                l -= aux.la_src[filt[pfilt[pp]].off + aux.anc[pp]];
            }
            logw[pp] = l;
            if (l > -INFINITY && l < INFINITY) atomicMax(&fmax_key[pfilt[pp]], float_order_key(l));
        }
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_fhnp_interval(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                 int32_t n_steps, float *logw, int32_t *fmax, AuxPtrs aux, int32_t noise,
                                 cudaStream_t s)
{
    const int nodes = (c.fhn_nodes == 4 || c.fhn_nodes == 8) && c.mp.J % c.fhn_nodes == 0 ? c.fhn_nodes : 2;
    if (nodes > 2) {  // 4 or 8 nodes per thread
        const int units = c.mp.J * c.mp.J / nodes;
        int n = 1;
        while ((n + 1) * units <= kFhnp4MaxThreads && n < kMaxSlots) ++n;
        if (c.fhn_ppc > 0 && c.fhn_ppc < n) n = c.fhn_ppc;
        const int ppc = n, threads = (ppc * units + 31) / 32 * 32;
        const size_t planes = 2 * (size_t)ppc * c.mp.J * c.mp.J * sizeof(float);
        const size_t smem = planes > (size_t)threads * sizeof(float) ? planes : (size_t)threads * sizeof(float);
        const unsigned grid = (unsigned)((c.P + ppc - 1) / ppc);
        const bool more = c.fhn_quad_ctas >= (nodes == 4 ? 4 : 3);  // the build for more CTAs per SM
#define PF_FHNP4_ARGS                                                                                             \
    c.mp, c.key, kStreamDyn, kStreamMisc, c.pfilt, c.filt, xi, xo, c.P, logw, d_obs, stride, c.obs_slot, c.d_t, ppc, \
        fmax, n_steps, aux, noise
        if (c.mp.J == 32) {  // the paper's side (Sec. 5.2): compile-time indexing
            if (nodes == 4 && more)
                k_propagate_fhnp4<4, 1, 32><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
            else if (nodes == 4)
                k_propagate_fhnp4<3, 1, 32><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
            else if (more)
                k_propagate_fhnp4<3, 2, 32><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
            else
                k_propagate_fhnp4<2, 2, 32><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
        } else if (nodes == 4 && more)
            k_propagate_fhnp4<4, 1><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
        else if (nodes == 4)
            k_propagate_fhnp4<3, 1><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
        else if (more)
            k_propagate_fhnp4<3, 2><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
        else
            k_propagate_fhnp4<2, 2><<<grid, threads, smem, s>>>(PF_FHNP4_ARGS);
#undef PF_FHNP4_ARGS
        return cudaGetLastError();
    }
    const int pairs = c.mp.J * c.mp.J / 2;
    const bool small = pairs <= 512;  // a particle fits the 512-thread build
    const int cap = small ? 512 : 1024;
    int n = 1;
    while ((n + 1) * pairs <= cap && n < kMaxSlots) ++n;
    if (c.fhn_ppc > 0 && c.fhn_ppc < n) n = c.fhn_ppc;
    const int ppc = n, threads = (ppc * pairs + 31) / 32 * 32;
    const size_t planes = 2 * (size_t)ppc * c.mp.J * c.mp.J * sizeof(float), red = (size_t)threads * sizeof(float);
    const size_t smem = planes > red ? planes : red;
    const unsigned grid = (unsigned)((c.P + ppc - 1) / ppc);
    if (small)
        k_propagate_fhnp<float, 512, 3><<<grid, threads, smem, s>>>(c.mp, c.key, kStreamDyn, kStreamMisc, c.pfilt,
                                                                    c.filt, xi, xo, c.P, logw, d_obs, stride,
                                                                    c.obs_slot, c.d_t, 0, 0, 0, ppc, fmax, n_steps,
                                                                    aux, noise);
    else
        k_propagate_fhnp<float><<<grid, threads, smem, s>>>(c.mp, c.key, kStreamDyn, kStreamMisc, c.pfilt, c.filt, xi,
                                                            xo, c.P, logw, d_obs, stride, c.obs_slot, c.d_t, 0, 0, 0,
                                                            ppc, fmax, n_steps, aux, noise);
    return cudaGetLastError();
}

cudaError_t launch_fhnp_truth_step(const ModelParams &mp, Key key, int32_t record, int32_t t, const double *xi,
                                   double *xo, cudaStream_t s)
{
    const int pairs = mp.J * mp.J / 2, threads = (pairs + 31) / 32 * 32;
    const size_t planes = 2 * (size_t)mp.J * mp.J * sizeof(double), red = (size_t)threads * sizeof(float);
    k_propagate_fhnp<double><<<1, threads, planes > red ? planes : red, s>>>(
        mp, key, kStreamTruth, kStreamStimTruth, nullptr, nullptr, xi, xo, 1, nullptr, nullptr, 0, nullptr, nullptr, 0,
        record, t, 1, nullptr, mp.K, AuxPtrs{}, 1);
    return cudaGetLastError();
}

}  // namespace pf
