// k_filter.cu -- sm_103a kernels of the ensemble of independent bootstrap
// filters (arXiv:1407.8071, Algorithm 1 run M times, Definition 1 average).
//
// One observation step is
//   propagate+weight  (Alg. 1 step 2a)      k_propagate_small / k_propagate_fhn
//   tile maxima       (log-sum-exp, pass 1)  k_tile_max
//   weights           (FP64 sums, eq. eqGtN) k_weights
//   prefix + scatter  (step 2b, systematic)  k_scan_scatter
//   ancestors+gather  (step 2b)              k_ancestors_small / k_ancestors + k_gather_rows
//   estimates         (Def. 1)               k_filter_means / k_mean_rows, k_ensemble
// Particles of all filters are contiguous; tiles of <= kTile particles never
// span two filters, so per-filter reductions read only that filter's tiles
// and no kernel waits on another block.
#include <cfloat>
#include <cmath>

#include "pf.h"
#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kWarps = kResampleThreads / 32;

// ------------------------------------------------------------------ block primitives
__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Max over the block, returned to every thread.
__device__ float block_max_f(float v, float *sh)
{
    v = warp_max_f(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    float r = sh[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, sh[i]);
    return r;
}

// Sums of NV doubles over the block in a fixed order (deterministic), to every thread.
template <int NV>
__device__ void block_sum_d(double (&v)[NV], double *sh)
{
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum_d(v[j]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[w * NV + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i * NV + j];
        v[j] = r;
    }
}

// Exclusive prefix sum of one double per thread (exact for integer-valued
// doubles below 2^53, the only use); returns the exclusive prefix.
__device__ double block_exscan_d(double v, double *sh)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    double inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double n = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += n;
    }
    __syncthreads();
    if (l == 31) sh[w] = inc;
    __syncthreads();
    double base = 0.0;
    for (int i = 0; i < w; ++i) base += sh[i];
    return base + inc - v;
}

// Exclusive prefix max of one int per thread; returns the exclusive prefix
// (identity -1).
__device__ int block_exscan_max_i(int v, int *sh)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc = max(inc, n);
    }
    int ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (l == 0) ex = -1;
    __syncthreads();
    if (l == 31) sh[w] = inc;
    __syncthreads();
    int base = -1;
    for (int i = 0; i < w; ++i) base = max(base, sh[i]);
    return max(base, ex);
}

// ------------------------------------------------------------------ systematic resampling arithmetic
// t_i = RN(RN(i + u) * c), each operation rounded to nearest (no contraction).
__device__ __forceinline__ double t_of(int64_t i, double u, double c) { return __dmul_rn(__dadd_rn((double)i, u), c); }

// #{i in [0, N) : t_i < x}.  t_i is non-decreasing in i, so the set is a prefix;
// a real-valued estimate is corrected by a short walk, with bisection as the
// exact fallback.
__device__ int64_t count_below(double x, double u, double c, double inv_c, int64_t N)
{
    if (!(x > 0.0)) return 0;
    double est = ceil(x * inv_c - u);
    int64_t i = est <= 0.0 ? 0 : (est >= (double)N ? N : (int64_t)est);
    bool settled = false;
    for (int it = 0; it < 4; ++it) {
        if (i > 0 && t_of(i - 1, u, c) >= x) --i;
        else { settled = true; break; }
    }
    if (settled) {
        settled = false;
        for (int it = 0; it < 4; ++it) {
            if (i < N && t_of(i, u, c) < x) ++i;
            else { settled = true; break; }
        }
    }
    if (!settled) {
        int64_t lo = 0, hi = N;  // smallest i with t_i >= x, or N
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (t_of(mid, u, c) < x) lo = mid + 1; else hi = mid;
        }
        i = lo;
    }
    return i;
}

// Unnormalised weight of particle p: exp(l - max) in FP32 from the FP32
// log-weight (non-finite log-weights weigh 0; a degenerate filter weighs
// uniformly and is flagged), or the caller's FP64 weight.
__device__ __forceinline__ double weight_of(const ResampleArgs &a, int64_t p, float mx, bool degenerate)
{
    if (a.w_direct) return a.w_direct[p];
    if (degenerate) return 1.0;
    const float l = a.logw[p];
    return (l > -INFINITY && l < INFINITY) ? (double)expf(l - mx) : 0.0;
}

__device__ __forceinline__ double quantise(double w, int shift) { return floor(ldexp(w, shift)); }

}  // namespace

// ------------------------------------------------------------------ init (Alg. 1 step 1)
template <int D>
__global__ void __launch_bounds__(256) k_init_small(ModelParams mp, Key key, const TileDesc *tiles, float *x, int64_t P)
{
    const TileDesc td = tiles[blockIdx.x];
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const int64_t p = td.gstart + j;
        float z[4];
        normals4<float>(key, (uint32_t)(td.lstart + j), 0u, (uint32_t)td.m, kStreamInit, 0u, z);
#pragma unroll
        for (int v = 0; v < D; ++v) x[v * P + p] = (float)(mp.x0_small[v] + mp.sigma0 * (double)z[v]);
    }
}

// Lattice prior: thread per (particle, node pair); node pair q uses Philox block q
// (lanes: v(2q), w(2q), v(2q+1), w(2q+1)).
__global__ void __launch_bounds__(256) k_init_fhn(ModelParams mp, Key key, const int32_t *pfilt, const FilterDesc *filt,
                                                  const double *x0, float *x, int64_t P)
{
    const int nn = mp.J * mp.J, pairs = nn / 2;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= P * pairs) return;
    const int64_t p = gid / pairs;
    const int q = (int)(gid % pairs);
    const int32_t m = pfilt[p];
    const uint32_t i = (uint32_t)(p - filt[m].off);
    float z[4];
    normals4<float>(key, i, 0u, (uint32_t)m, kStreamInit, (uint32_t)q, z);
    float *xp = x + p * (int64_t)mp.dx;
    const int n0 = 2 * q, n1 = 2 * q + 1;
    xp[n0] = (float)(x0[n0] + mp.sigma0 * (double)z[0]);
    xp[nn + n0] = (float)(x0[nn + n0] + mp.sigma0 * (double)z[1]);
    xp[n1] = (float)(x0[n1] + mp.sigma0 * (double)z[2]);
    xp[nn + n1] = (float)(x0[nn + n1] + mp.sigma0 * (double)z[3]);
}

// ------------------------------------------------------------------ propagate + weight (Alg. 1 step 2a)
// Thread per particle, SoA state x[v * P + p] (coalesced), K Euler-Maruyama
// sub-steps in registers, then the FP32 log-likelihood.
template <int D>
__global__ void __launch_bounds__(256) k_propagate_small(ModelParams mp, Key key, const TileDesc *tiles,
                                                         const float *__restrict__ x_in, float *__restrict__ x_out,
                                                         int64_t P, float *logw, const float *obs, int32_t obs_stride,
                                                         const int32_t *d_t)
{
    const TileDesc td = tiles[blockIdx.x];
    const uint32_t t = (uint32_t)(*d_t + 1);
    const float *y = obs + (obs_stride ? (int64_t)td.m * obs_stride : 0);
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const int64_t p = td.gstart + j;
        float xs[D];
#pragma unroll
        for (int v = 0; v < D; ++v) xs[v] = x_in[v * P + p];
        propagate_small<D, float>(mp, key, kStreamDyn, (uint32_t)(td.lstart + j), t, (uint32_t)td.m, xs);
#pragma unroll
        for (int v = 0; v < D; ++v) x_out[v * P + p] = xs[v];
        logw[p] = loglik_small<D, float>(mp, y, xs);
    }
}

// Lattice propagation (Sec. 5.1, Rogers-McCulloch form): a CTA holds ppc
// particles; each thread owns two adjacent nodes (v, w in registers).  The
// v-plane goes through shared memory once per sub-step (double-buffered, one
// barrier per sub-step) for the zero-flux 5-point Laplacian.
template <typename Real>
__device__ __forceinline__ Real fhn_drift_v(const ModelParams &mp, Real v, Real w, Real lap, Real I)
{
    const Real a = (Real)mp.p[0], c1 = (Real)mp.p[2], c2 = (Real)mp.p[3], D = (Real)mp.p[5];
    return c1 * v * (v - a) * ((Real)1 - v) - c2 * v * w + D * lap + I;
}

template <typename Real>
__device__ __forceinline__ Real fhn_drift_w(const ModelParams &mp, Real v, Real w)
{
    const Real b = (Real)mp.p[1], d = (Real)mp.p[4];
    return b * (v - d * w);
}

// One observation interval of `count` lattice particles.  Real = float for
// the filters (state in FP32) and double for the truth record.
// Thread (slot s, pair q): particle p = first + s, nodes 2q and 2q+1 (same row).
template <typename Real>
__global__ void k_propagate_fhn(ModelParams mp, Key key, uint32_t stream, const int32_t *pfilt,
                                const FilterDesc *filt, const Real *__restrict__ x_in, Real *__restrict__ x_out,
                                int64_t P, float *logw, const float *obs, int32_t obs_stride,
                                const int32_t *obs_slot, const int32_t *d_t, int32_t fixed_c0, int32_t fixed_c2,
                                int32_t t_direct)
{
    extern __shared__ unsigned char smem_raw[];
    const int J = mp.J, nn = J * J, pairs = nn / 2;
    const int ppc = blockDim.x / pairs;
    Real *sv = reinterpret_cast<Real *>(smem_raw);  // [2][ppc][nn]
    const int s = threadIdx.x / pairs;
    const int q = threadIdx.x - s * pairs;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(d_t ? *d_t + 1 : t_direct);

    uint32_t c0 = 0, c2 = 0;
    const Real *xi = nullptr;
    Real *xo = nullptr;
    Real v0 = 0, v1 = 0, w0 = 0, w1 = 0;
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
        xi = x_in + p * (int64_t)mp.dx;
        xo = x_out + p * (int64_t)mp.dx;
        v0 = xi[n0];
        v1 = xi[n0 + 1];
        w0 = xi[nn + n0];
        w1 = xi[nn + n0 + 1];
    }
    const Real dt = (Real)mp.dt;
    const Real sq = (Real)(mp.sigma_dyn * sqrt(mp.dt));
    const Real amp = (Real)mp.p[6];
    const int64_t stim_steps = (int64_t)mp.p[7];
    const int blk = (int)mp.p[8];
    const bool stim_node0 = row < blk && col < blk, stim_node1 = row < blk && col + 1 < blk;
    const int64_t n_base = (int64_t)(t - 1) * mp.K;  // (n - 1) of sub-step k is n_base + k
    const uint32_t blocks_per_step = (uint32_t)(mp.dx / 4);
    const bool up = row > 0, down = row < J - 1, left = col > 0, right = col + 2 < J;
    const Real cnt0 = (Real)((int)up + (int)down + (int)left + 1);
    const Real cnt1 = (Real)((int)up + (int)down + (int)right + 1);

    for (int k = 0; k < mp.K; ++k) {
        Real *buf = sv + ((k & 1) * ppc + (active ? s : 0)) * nn;
        if (active) {
            buf[n0] = v0;
            buf[n0 + 1] = v1;
        }
        __syncthreads();
        if (active) {
            Real z[4];
            normals4<Real>(Key{key.k0, key.k1}, c0, t, c2, stream, (uint32_t)k * blocks_per_step + (uint32_t)q, z);
            Real l0 = v1, l1 = v0;
            if (up) { l0 += buf[n0 - J]; l1 += buf[n0 + 1 - J]; }
            if (down) { l0 += buf[n0 + J]; l1 += buf[n0 + 1 + J]; }
            if (left) l0 += buf[n0 - 1];
            if (right) l1 += buf[n0 + 2];
            l0 -= cnt0 * v0;
            l1 -= cnt1 * v1;
            const bool on = (n_base + k) < stim_steps;
            const Real I0 = (on && stim_node0) ? amp : (Real)0, I1 = (on && stim_node1) ? amp : (Real)0;
            const Real fv0 = fhn_drift_v<Real>(mp, v0, w0, l0, I0), fv1 = fhn_drift_v<Real>(mp, v1, w1, l1, I1);
            const Real fw0 = fhn_drift_w<Real>(mp, v0, w0), fw1 = fhn_drift_w<Real>(mp, v1, w1);
            v0 = v0 + dt * fv0 + sq * z[0];
            w0 = w0 + dt * fw0 + sq * z[1];
            v1 = v1 + dt * fv1 + sq * z[2];
            w1 = w1 + dt * fw1 + sq * z[3];
        }
    }
    if (active) {
        xo[n0] = v0;
        xo[n0 + 1] = v1;
        xo[nn + n0] = w0;
        xo[nn + n0 + 1] = w1;
    }
    if (!logw) return;
    // log-likelihood over the observed nodes, per particle, fixed order
    float part = 0.0f;
    if (active) {
        const int32_t m = pfilt ? pfilt[p] : 0;
        const float *y = obs + (obs_stride ? (int64_t)m * obs_stride : 0);
        const int j0 = obs_slot[n0], j1 = obs_slot[n0 + 1];
        if (j0 >= 0) { const float e = y[j0] - (float)v0; part += e * e; }
        if (j1 >= 0) { const float e = y[j1] - (float)v1; part += e * e; }
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);
    red[threadIdx.x] = part;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < ppc) {
        const int64_t pp = (int64_t)blockIdx.x * ppc + warp;
        float acc = 0.0f;
        for (int i = lane; i < pairs; i += 32) acc += red[warp * pairs + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && pp < P) logw[pp] = (float)(-0.5 / (mp.sigma_obs * mp.sigma_obs)) * acc;
    }
}

// ------------------------------------------------------------------ resampling chain
// Pass 1: maximum log-weight of each tile.
__global__ void __launch_bounds__(kResampleThreads) k_tile_max(ResampleArgs a)
{
    __shared__ float sh[kWarps];
    const TileDesc td = a.tiles[blockIdx.x];
    float mx = -INFINITY;
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const float l = a.logw[td.gstart + j];
        if (l < INFINITY) mx = fmaxf(mx, l);  // NaN and +inf never win
    }
    mx = block_max_f(mx, sh);
    if (threadIdx.x == 0) a.tile_max[blockIdx.x] = mx;
}

// Pass 2: filter maximum, then per tile the FP64 sums of w, w^2 and of the
// quantised weights q = floor(w 2^shift); clears the ancestor markers.
__global__ void __launch_bounds__(kResampleThreads) k_weights(ResampleArgs a)
{
    __shared__ double shd[kWarps * 3];
    __shared__ float shf[kWarps];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = a.filt[td.m];
    float mx = -INFINITY;
    if (!a.w_direct) {
        for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) mx = fmaxf(mx, a.tile_max[fd.tile_begin + j]);
        mx = block_max_f(mx, shf);
    }
    const bool degenerate = !a.w_direct && !(mx > -INFINITY);
    double s[3] = {0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const int64_t p = td.gstart + j;
        const double w = weight_of(a, p, mx, degenerate);
        s[0] += w;
        s[1] += w * w;
        s[2] += quantise(w, fd.shift);
        a.B[p] = -1;
    }
    block_sum_d<3>(s, shd);
    if (threadIdx.x == 0) {
        double *ts = a.tile_sums + (int64_t)blockIdx.x * kTsCount;
        ts[kTsW] = s[0];
        ts[kTsW2] = s[1];
        ts[kTsQ] = s[2];
        if (td.lstart == 0) {
            a.fstats[(int64_t)td.m * kFsCount + kFsMax] = degenerate ? 0.0 : (double)mx;
            a.fstats[(int64_t)td.m * kFsCount + kFsDegenerate] = degenerate ? 1.0 : 0.0;
            if (degenerate) {
                atomicOr(&a.err[0], kErrDegenerate);
                atomicCAS(&a.err[1], -1, td.m);
            }
        }
    }
}

// Pass 3: exact FP64 prefix of q (tile offset + block scan), the counts
// #{i : t_i < C_k}, and the start markers B[lo_k] = k of every particle with
// offspring (plus the tail marker of the last particle with q > 0).  The
// first tile of each filter also writes the filter's log Z, ESS, log G.
__global__ void __launch_bounds__(kResampleThreads) k_scan_scatter(ResampleArgs a)
{
    __shared__ double shd[kWarps * 4];
    __shared__ double shs[kWarps];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = a.filt[td.m];
    const int ti = blockIdx.x - fd.tile_begin;
    // filter totals and the prefix before this tile, in a fixed order
    double s[4] = {0.0, 0.0, 0.0, 0.0};  // Q_all, Q_before, W, W2
    for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) {
        const double *ts = a.tile_sums + (int64_t)(fd.tile_begin + j) * kTsCount;
        s[0] += ts[kTsQ];
        if (j < ti) s[1] += ts[kTsQ];
        s[2] += ts[kTsW];
        s[3] += ts[kTsW2];
    }
    block_sum_d<4>(s, shd);
    const float mx = a.w_direct ? 0.0f : (float)a.fstats[(int64_t)td.m * kFsCount + kFsMax];
    const bool degenerate = !a.w_direct && a.fstats[(int64_t)td.m * kFsCount + kFsDegenerate] != 0.0;
    double Ctot = s[0];
    const int32_t t = a.d_t ? *a.d_t + 1 : 0;
    const double u = a.u_direct ? a.u_direct[td.m] : resample_uniform(a.key, td.m, t);
    const int64_t N = fd.N;
    const double c = __ddiv_rn(Ctot, (double)N);
    const double inv_c = 1.0 / c;

    if (threadIdx.x == 0 && ti == 0) {
        double *fs = a.fstats + (int64_t)td.m * kFsCount;
        const double logS = log(s[2]);
        const double logZ = (double)mx + logS;
        fs[kFsLogZ] = logZ;
        fs[kFsEss] = s[2] * s[2] / s[3];
        if (a.d_t) fs[kFsLogG] = (t == 1 ? 0.0 : fs[kFsLogG]) + logZ - log((double)N) + a.log_const;
        fs[kFsCtot] = Ctot;
        fs[kFsU] = u;
        fs[kFsC] = c;
    }
    // blocked items: thread j owns tile positions [j * kItems, (j + 1) * kItems)
    const int j0 = threadIdx.x * kItems;
    double q[kItems];
    double tsum = 0.0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int j = j0 + r;
        q[r] = 0.0;
        if (j < td.len) q[r] = quantise(weight_of(a, td.gstart + j, mx, degenerate), fd.shift);
        tsum += q[r];
    }
    double Cprev = s[1] + block_exscan_d(tsum, shs);  // C_{k-1} before my first item
    int64_t cnt_prev = count_below(Cprev, u, c, inv_c, N);
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int j = j0 + r;
        if (j >= td.len) break;
        const int64_t k = td.lstart + j;
        const double Ck = Cprev + q[r];
        a.C[td.gstart + j] = Ck;
        if (q[r] > 0.0) {
            const int64_t cnt = count_below(Ck, u, c, inv_c, N);
            if (cnt > cnt_prev) a.B[fd.off + cnt_prev] = (int32_t)k;
            if (Ck == Ctot && cnt < N) a.B[fd.off + cnt] = (int32_t)k;  // tail of the last q > 0
            cnt_prev = cnt;
        }
        Cprev = Ck;
    }
}

// Ancestor of the tile's first output index by bisection over the filter's C.
__device__ __forceinline__ int32_t search_ancestor(const double *C, int64_t N, double Ctot, double tq)
{
    // min{k : C_k > tq}, or, when tq >= Ctot, min{k : C_k >= Ctot}
    const bool tail = !(tq < Ctot);
    int64_t lo = 0, hi = N - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const bool right = tail ? (C[mid] >= Ctot) : (C[mid] > tq);
        if (right) hi = mid; else lo = mid + 1;
    }
    return (int32_t)lo;
}

// Pass 4 (ancestors only): a_i = max(first ancestor of the tile, max of the
// markers B[i0..i]).
__device__ __forceinline__ void tile_ancestors(const ResampleArgs &a, const TileDesc &td, const FilterDesc &fd,
                                               int32_t (&anc)[kItems], int *shi)
{
    const double *fs = a.fstats + (int64_t)td.m * kFsCount;
    const double Ctot = fs[kFsCtot], u = fs[kFsU], c = fs[kFsC];
    const int32_t a0 = search_ancestor(a.C + fd.off, fd.N, Ctot, t_of(td.lstart, u, c));
    const int j0 = threadIdx.x * kItems;
    int b[kItems];
    int tmax = -1;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int j = j0 + r;
        b[r] = (j < td.len) ? a.B[td.gstart + j] : -1;
        tmax = max(tmax, b[r]);
    }
    int run = max(a0, block_exscan_max_i(tmax, shi));
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        run = max(run, b[r]);
        anc[r] = run;
    }
}

// Small models: ancestors, gather of the SoA state and per-tile FP64 sums of
// every variable of the resampled particles.
template <int D>
__global__ void __launch_bounds__(kResampleThreads) k_ancestors_small(ResampleArgs a, const float *__restrict__ x_in,
                                                                      float *__restrict__ x_out, int64_t P,
                                                                      double *tile_est)
{
    __shared__ int shi[kWarps];
    __shared__ double shd[kWarps * D];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = a.filt[td.m];
    int32_t anc[kItems];
    tile_ancestors(a, td, fd, anc, shi);
    const int j0 = threadIdx.x * kItems;
    double s[D];
#pragma unroll
    for (int v = 0; v < D; ++v) s[v] = 0.0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int j = j0 + r;
        if (j < td.len) {
            const int64_t p = td.gstart + j;
            a.anc[p] = anc[r];
            const int64_t src = fd.off + anc[r];
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const float xv = x_in[v * P + src];
                x_out[v * P + p] = xv;
                s[v] += (double)xv;
            }
        }
    }
    if (tile_est) {
        block_sum_d<D>(s, shd);
        if (threadIdx.x == 0)
#pragma unroll
            for (int v = 0; v < D; ++v) tile_est[(int64_t)blockIdx.x * D + v] = s[v];
    }
}

// Ancestors only (lattice models and the stateless entry point).
__global__ void __launch_bounds__(kResampleThreads) k_ancestors(ResampleArgs a)
{
    __shared__ int shi[kWarps];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = a.filt[td.m];
    int32_t anc[kItems];
    tile_ancestors(a, td, fd, anc, shi);
    const int j0 = threadIdx.x * kItems;
#pragma unroll
    for (int r = 0; r < kItems; ++r)
        if (j0 + r < td.len) a.anc[td.gstart + j0 + r] = anc[r];
}

// Lattice gather: whole particle rows x_out[p] = x_in[off + anc[p]] (float4).
__global__ void __launch_bounds__(256) k_gather_rows(const int32_t *__restrict__ anc, const int32_t *__restrict__ pfilt,
                                                     const FilterDesc *filt, const float4 *__restrict__ x_in,
                                                     float4 *__restrict__ x_out, int row4)
{
    const int64_t p = blockIdx.x;
    const int64_t src = filt[pfilt[p]].off + anc[p];
    const float4 *a = x_in + src * row4;
    float4 *b = x_out + p * row4;
    for (int i = threadIdx.x; i < row4; i += blockDim.x) b[i] = a[i];
}

// Lattice estimates: est[m][v] = (1/N_m) sum_i x[off + i][v], FP64, i ascending.
__global__ void __launch_bounds__(256) k_mean_rows(const FilterDesc *filt, const float *__restrict__ x, int dx,
                                                   double *est)
{
    const int m = blockIdx.y;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= dx) return;
    const FilterDesc fd = filt[m];
    const float *base = x + fd.off * (int64_t)dx + v;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 4 <= fd.N; i += 4) {
        s0 += (double)base[(int64_t)i * dx];
        s1 += (double)base[(int64_t)(i + 1) * dx];
        s2 += (double)base[(int64_t)(i + 2) * dx];
        s3 += (double)base[(int64_t)(i + 3) * dx];
    }
    for (; i < fd.N; ++i) s0 += (double)base[(int64_t)i * dx];
    est[(int64_t)m * dx + v] = ((s0 + s1) + (s2 + s3)) / (double)fd.N;
}

// Small models: est[m][v] = (1/N_m) sum over the filter's tiles, fixed order.
__global__ void k_filter_means(const FilterDesc *filt, const double *tile_est, int dx, double *est, int32_t M)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)M * dx) return;
    const int m = (int)(gid / dx), v = (int)(gid % dx);
    const FilterDesc fd = filt[m];
    double s = 0.0;
    for (int j = 0; j < fd.tile_count; ++j) s += tile_est[(int64_t)(fd.tile_begin + j) * dx + v];
    est[gid] = s / (double)fd.N;
}

// Definition 1: ens[v] = (1/M) sum_m est[m][v] (FP64, m ascending); advances
// the step counter.
__global__ void k_ensemble(const double *est, int dx, int32_t M, double *ens, int32_t *d_t)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < dx) {
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += est[(int64_t)m * dx + v];
        ens[v] = s / (double)M;
    }
    if (v == 0 && d_t) *d_t += 1;
}

// ------------------------------------------------------------------ synthetic record (FP64)
template <int D>
__global__ void k_simulate_small(ModelParams mp, Key key, int32_t T, int32_t record, int32_t init_random,
                                 double *xs, float *ys)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double x[D];
    if (init_random) {
        double z[4];
        normals4<double>(key, 0u, 0u, (uint32_t)record, kStreamMisc, 0u, z);
#pragma unroll
        for (int v = 0; v < D; ++v) x[v] = mp.x0_small[v] + mp.sigma0 * z[v];
    } else {
#pragma unroll
        for (int v = 0; v < D; ++v) x[v] = mp.x0_small[v];
    }
#pragma unroll
    for (int v = 0; v < D; ++v) xs[v] = x[v];
    for (int t = 1; t <= T; ++t) {
        propagate_small<D, double>(mp, key, kStreamTruth, 0u, (uint32_t)t, (uint32_t)record, x);
#pragma unroll
        for (int v = 0; v < D; ++v) xs[(int64_t)t * D + v] = x[v];
        double z[4];
        for (int j = 0; j < mp.dy; ++j) {
            if ((j & 3) == 0) normals4<double>(key, 0u, (uint32_t)t, (uint32_t)record, kStreamObs, (uint32_t)(j >> 2), z);
            double xv = 0.0;
#pragma unroll
            for (int v = 0; v < D; ++v)
                if (v == mp.obs_small[j]) xv = x[v];
            ys[(int64_t)(t - 1) * mp.dy + j] = (float)(xv + mp.sigma_obs * z[j & 3]);
        }
    }
}

__global__ void k_fhn_truth_init(ModelParams mp, Key key, int32_t record, int32_t init_random, const double *x0,
                                 double *x)
{
    const int nn = mp.J * mp.J, pairs = nn / 2;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= pairs) return;
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    if (init_random) normals4<double>(key, 0u, 0u, (uint32_t)record, kStreamMisc, (uint32_t)q, z);
    const int n0 = 2 * q, n1 = n0 + 1;
    x[n0] = x0[n0] + mp.sigma0 * z[0];
    x[nn + n0] = x0[nn + n0] + mp.sigma0 * z[1];
    x[n1] = x0[n1] + mp.sigma0 * z[2];
    x[nn + n1] = x0[nn + n1] + mp.sigma0 * z[3];
}

__global__ void k_observe(ModelParams mp, Key key, const int32_t *obs_idx, int32_t t, int32_t record,
                          const double *x, float *y)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= mp.dy) return;
    double z[4];
    normals4<double>(key, 0u, (uint32_t)t, (uint32_t)record, kStreamObs, (uint32_t)(j >> 2), z);
    y[j] = (float)(x[obs_idx[j]] + mp.sigma_obs * z[j & 3]);
}

// ------------------------------------------------------------------ generator components
__global__ void k_rng_philox(int64_t n, const uint4 *ctr, uint32_t k0, uint32_t k1, uint4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_rng_normals(int64_t n, const uint4 *ctr, Key key, float4 *z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(ctr[i], key.k0, key.k1);
    float a, b, c, d;
    box_muller<float>(r.x, r.y, a, b);
    box_muller<float>(r.z, r.w, c, d);
    z[i] = make_float4(a, b, c, d);
}

// ------------------------------------------------------------------ launchers
namespace {

int fhn_threads(const ModelParams &mp, int *ppc)
{
    const int pairs = mp.J * mp.J / 2;
    int n = 1;
    while ((n + 1) * pairs <= 1024 && n < 8) ++n;
    *ppc = n;
    return n * pairs;
}

size_t fhn_smem(const ModelParams &mp, int threads, int ppc, size_t real_bytes)
{
    const size_t planes = 2 * (size_t)ppc * mp.J * mp.J * real_bytes;
    const size_t red = (size_t)threads * sizeof(float);
    return planes > red ? planes : red;
}

template <int D>
cudaError_t init_small(const Ctx &c, cudaStream_t s)
{
    k_init_small<D><<<c.n_tiles, 256, 0, s>>>(c.mp, c.key, c.tiles, c.x[c.cur], c.P);
    return cudaGetLastError();
}

template <int D>
cudaError_t propagate_small_launch(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                   cudaStream_t s)
{
    k_propagate_small<D><<<c.n_tiles, 256, 0, s>>>(c.mp, c.key, c.tiles, xi, xo, c.P, c.logw, d_obs, stride, c.d_t);
    return cudaGetLastError();
}

ResampleArgs ctx_args(const Ctx &c)
{
    ResampleArgs a{};
    a.tiles = c.tiles;
    a.filt = c.filt;
    a.logw = c.logw;
    a.w_direct = nullptr;
    a.u_direct = nullptr;
    a.key = c.key;
    a.d_t = c.d_t;
    a.tile_max = c.tile_max;
    a.tile_sums = c.tile_sums;
    a.fstats = c.fstats;
    a.C = c.C;
    a.B = c.B;
    a.anc = c.anc;
    a.err = c.err;
    a.log_const = -0.5 * c.mp.dy * log(2.0 * M_PI * c.mp.sigma_obs * c.mp.sigma_obs);
    return a;
}

}  // namespace

cudaError_t launch_init(const Ctx &c, cudaStream_t s)
{
    if (c.mp.kind == kFhnLattice) {
        const int64_t work = c.P * (c.mp.J * c.mp.J / 2);
        k_init_fhn<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(c.mp, c.key, c.pfilt, c.filt, c.x0, c.x[c.cur], c.P);
        return cudaGetLastError();
    }
    switch (c.mp.dx) {
    case 1: return init_small<1>(c, s);
    case 2: return init_small<2>(c, s);
    case 3: return init_small<3>(c, s);
    case 4: return init_small<4>(c, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_propagate(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                             cudaStream_t s)
{
    if (c.mp.kind == kFhnLattice) {
        int ppc;
        const int threads = fhn_threads(c.mp, &ppc);
        const size_t smem = fhn_smem(c.mp, threads, ppc, sizeof(float));
        const unsigned grid = (unsigned)((c.P + ppc - 1) / ppc);
        k_propagate_fhn<float><<<grid, threads, smem, s>>>(c.mp, c.key, kStreamDyn, c.pfilt, c.filt, xi, xo, c.P,
                                                           c.logw, d_obs, stride, c.obs_slot, c.d_t, 0, 0, 0);
        return cudaGetLastError();
    }
    switch (c.mp.dx) {
    case 1: return propagate_small_launch<1>(c, d_obs, stride, xi, xo, s);
    case 2: return propagate_small_launch<2>(c, d_obs, stride, xi, xo, s);
    case 3: return propagate_small_launch<3>(c, d_obs, stride, xi, xo, s);
    case 4: return propagate_small_launch<4>(c, d_obs, stride, xi, xo, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resample(const Ctx &c, const float *xi, float *xo, cudaStream_t s)
{
    const ResampleArgs a = ctx_args(c);
    k_tile_max<<<c.n_tiles, kResampleThreads, 0, s>>>(a);
    k_weights<<<c.n_tiles, kResampleThreads, 0, s>>>(a);
    k_scan_scatter<<<c.n_tiles, kResampleThreads, 0, s>>>(a);
    const int dx = c.mp.dx;
    if (c.mp.kind == kFhnLattice) {
        k_ancestors<<<c.n_tiles, kResampleThreads, 0, s>>>(a);
        k_gather_rows<<<(unsigned)c.P, 256, 0, s>>>(c.anc, c.pfilt, c.filt, reinterpret_cast<const float4 *>(xi),
                                                   reinterpret_cast<float4 *>(xo), dx / 4);
        dim3 g((dx + 255) / 256, c.M);
        k_mean_rows<<<g, 256, 0, s>>>(c.filt, xo, dx, c.est);
    } else {
        switch (dx) {
        case 1: k_ancestors_small<1><<<c.n_tiles, kResampleThreads, 0, s>>>(a, xi, xo, c.P, c.tile_est); break;
        case 2: k_ancestors_small<2><<<c.n_tiles, kResampleThreads, 0, s>>>(a, xi, xo, c.P, c.tile_est); break;
        case 3: k_ancestors_small<3><<<c.n_tiles, kResampleThreads, 0, s>>>(a, xi, xo, c.P, c.tile_est); break;
        case 4: k_ancestors_small<4><<<c.n_tiles, kResampleThreads, 0, s>>>(a, xi, xo, c.P, c.tile_est); break;
        default: return cudaErrorInvalidValue;
        }
        const int64_t n = (int64_t)c.M * dx;
        k_filter_means<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.filt, c.tile_est, dx, c.est, c.M);
    }
    k_ensemble<<<(dx + 255) / 256, 256, 0, s>>>(c.est, dx, c.M, c.ens, c.d_t);
    return cudaGetLastError();
}

cudaError_t launch_systematic(int32_t M, int32_t n_tiles, const ResampleArgs &a, cudaStream_t s)
{
    (void)M;
    k_weights<<<n_tiles, kResampleThreads, 0, s>>>(a);
    k_scan_scatter<<<n_tiles, kResampleThreads, 0, s>>>(a);
    k_ancestors<<<n_tiles, kResampleThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rng_philox(int64_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_rng_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, reinterpret_cast<const uint4 *>(ctr), k0, k1,
                                                             reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_rng_normals(int64_t n, const uint32_t *ctr, uint64_t seed, float *z, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_rng_normals<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, reinterpret_cast<const uint4 *>(ctr),
                                                              make_key(seed), reinterpret_cast<float4 *>(z));
    return cudaGetLastError();
}

cudaError_t launch_simulate(const ModelParams &mp, const double *d_x0, const int32_t *d_obs_idx, Key key, int32_t T,
                            int32_t record, int32_t init_random, double *d_x, float *d_y, cudaStream_t s)
{
    if (mp.kind != kFhnLattice) {
        switch (mp.dx) {
        case 1: k_simulate_small<1><<<1, 32, 0, s>>>(mp, key, T, record, init_random, d_x, d_y); break;
        case 2: k_simulate_small<2><<<1, 32, 0, s>>>(mp, key, T, record, init_random, d_x, d_y); break;
        case 3: k_simulate_small<3><<<1, 32, 0, s>>>(mp, key, T, record, init_random, d_x, d_y); break;
        case 4: k_simulate_small<4><<<1, 32, 0, s>>>(mp, key, T, record, init_random, d_x, d_y); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int pairs = mp.J * mp.J / 2;
    k_fhn_truth_init<<<(pairs + 255) / 256, 256, 0, s>>>(mp, key, record, init_random, d_x0, d_x);
    const size_t smem = fhn_smem(mp, pairs, 1, sizeof(double));
    for (int32_t t = 1; t <= T; ++t) {
        const double *xi = d_x + (int64_t)(t - 1) * mp.dx;
        double *xo = d_x + (int64_t)t * mp.dx;
        k_propagate_fhn<double><<<1, pairs, smem, s>>>(mp, key, kStreamTruth, nullptr, nullptr, xi, xo, 1, nullptr,
                                                       nullptr, 0, nullptr, nullptr, 0, record, t);
        if (d_y)
            k_observe<<<(mp.dy + 255) / 256, 256, 0, s>>>(mp, key, d_obs_idx, t, record, xo,
                                                          d_y + (int64_t)(t - 1) * mp.dy);
    }
    return cudaGetLastError();
}

}  // namespace pf
