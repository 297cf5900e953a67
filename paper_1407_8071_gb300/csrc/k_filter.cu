// k_filter.cu -- sm_103a kernels of the ensemble of independent bootstrap
// filters (arXiv:1407.8071, Algorithm 1 run M times, Definition 1 average).
//
// One observation step is
//   propagate+weight  (Alg. 1 step 2a)      k_propagate_small / k_propagate_fhn(4) (+ per-filter max log-weight)
//   resampling        (step 2b, systematic; FP64 sums, eq. eqGtN)
//     filters of several tiles:  k_weights -> k_scan_scatter -> k_ancestors_small (gather, per-filter
//                                means) / k_ancestors
//     filters of one tile:       k_resample_whole (one launch per size class) -> k_whole_finish
//   lattice gather + estimates   k_gather_mean_rows(4) (Def. 1 per filter)
//   M-average         (Def. 1)               k_ensemble
// Particles of all filters are contiguous; tiles of <= kTile particles never
// span two filters, so per-filter reductions read only that filter's tiles
// and no kernel waits on another block.
//
// FP64 is a narrow pipe on this GPU (about 1/64 of the FP32 rate), so it is
// used only where the precision contract needs it -- the per-filter sums of
// the normaliser and of the estimates, and the average over filters -- and
// there only above the tile level: inside a tile, sums are compensated FP32
// pairs (Knuth's two-sum, about 48 significant bits), converted to FP64 once
// per tile.  Systematic resampling is exact integer arithmetic (64-bit
// prefix, 128-bit comparisons).  The per-filter means of the small models are
// finished by the last tile of each filter (completion counter, no waiting), in
// a fixed order.
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "pf.h"
#include "pf_internal.h"
#include "lattice.cuh"

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

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Compensated FP32 pair (hi + lo) and Knuth's two-sum: the pair holds a sum
// to about 2^-48 relative accuracy with FP32 instructions only.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, float b)
{
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return FF{s, __fadd_rn(a.lo, e)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF r = ff_add(a, b.hi);
    r.lo = __fadd_rn(r.lo, b.lo);
    return r;
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Sums of NV compensated pairs over the block in a fixed order; every thread
// receives the FP64 results.  Every thread leaves its pairs in shared memory;
// warp j (j < NV, strided over the block's warps) then adds column j -- each
// lane the values lane, lane + 32, ... in order, then an xor tree over the
// lanes -- so the shuffle tree runs once per sum instead of once per warp.
// `sf` holds 2 NV blockDim.x floats, `sd` NV doubles.
template <int NV>
__device__ void block_sum_ff(FF (&v)[NV], double (&out)[NV], float *sf, double *sd)
{
    const int n = blockDim.x, nw = n >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // the scratch may still be read by a previous use
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        sf[(2 * j) * n + threadIdx.x] = v[j].hi;
        sf[(2 * j + 1) * n + threadIdx.x] = v[j].lo;
    }
    __syncthreads();
    for (int j = w; j < NV; j += nw) {
        FF acc{0.0f, 0.0f};
        for (int i = l; i < n; i += 32) acc = ff_add(acc, FF{sf[(2 * j) * n + i], sf[(2 * j + 1) * n + i]});
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const FF other{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
            acc = ff_add(acc, other);
        }
        if (l == 0) sd[j] = ff_to_double(acc);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = sd[j];
}

// The same with one scratch area `shm` of 2 NV blockDim.x floats followed by NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum_ff(FF (&v)[NV], double (&out)[NV], void *shm)
{
    float *sf = reinterpret_cast<float *>(shm);
    block_sum_ff<NV>(v, out, sf, reinterpret_cast<double *>(sf + 2 * NV * blockDim.x));
}

// FP64 sums over the block of NV per-thread values, in a fixed order
// (deterministic): warp j < NV sums column j.  `sh` holds blockDim.x * NV + NV
// doubles.  Every thread receives the sums.
template <int NV>
__device__ void block_sum_dd(double (&v)[NV], double *sh)
{
    const int n = blockDim.x, tid = threadIdx.x;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j * n + tid] = v[j];
    __syncthreads();
    const int w = tid >> 5, l = tid & 31;
    for (int j = w; j < NV; j += (n >> 5)) {
        double acc = 0.0;
        for (int i = l; i < n; i += 32) acc += sh[j * n + i];
        acc = warp_sum_d(acc);
        if (l == 0) sh[NV * n + j] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = sh[NV * n + j];
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ uint64_t block_sum_u64(uint64_t v, uint64_t *sh)
{
    v = warp_sum_u64(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    uint64_t r = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;
}

// Two block sums of uint64 at once (one pair of barriers); `sh` holds 2 kWarps.
__device__ void block_sum_u64x2(uint64_t &a, uint64_t &b, uint64_t *sh)
{
    a = warp_sum_u64(a);
    b = warp_sum_u64(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) {
        sh[w] = a;
        sh[kWarps + w] = b;
    }
    __syncthreads();
    a = b = 0;
    for (int i = 0; i < nw; ++i) {
        a += sh[i];
        b += sh[kWarps + i];
    }
}

// Exclusive prefix sum of one uint64 per thread.
__device__ uint64_t block_exscan_u64(uint64_t v, uint64_t *sh)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t n = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += n;
    }
    __syncthreads();
    if (l == 31) sh[w] = inc;
    __syncthreads();
    uint64_t base = 0;
    for (int i = 0; i < w; ++i) base += sh[i];
    return base + inc - v;
}

// Exclusive prefix max of one int per thread (identity -1).
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

// ------------------------------------------------------------------ exact systematic resampling
// q = floor(w 2^shift) of a weight in [0, 1], exactly, from the float's bits
// (weights of 1 or more count as 1; NaN and non-positive weights as 0).
__device__ __forceinline__ uint64_t quant_f32(float w, int shift)
{
    if (!(w > 0.0f)) return 0;
    if (w >= 1.0f) return 1ull << shift;
    const uint32_t b = __float_as_uint(w);
    int e = (int)((b >> 23) & 0xFF);
    uint64_t m = b & 0x7FFFFFu;
    if (e == 0) e = 1; else m |= 0x800000u;  // w = m 2^(e - 150)
    const int sh = e - 150 + shift;
    if (sh >= 0) return m << sh;
    return (-sh) >= 64 ? 0 : (m >> (-sh));
}

__device__ __forceinline__ uint64_t quant_f64(double w, int shift)
{
    if (!(w > 0.0)) return 0;
    if (w >= 1.0) return 1ull << shift;
    const uint64_t b = (uint64_t)__double_as_longlong(w);
    int e = (int)((b >> 52) & 0x7FF);
    uint64_t m = b & ((1ull << 52) - 1);
    if (e == 0) e = 1; else m |= 1ull << 52;  // w = m 2^(e - 1075)
    const int sh = e - 1075 + shift;          // < 0 since w < 1 and shift <= 52
    return (-sh) >= 64 ? 0 : (m >> (-sh));
}

struct U128 {
    uint64_t hi, lo;
};

__device__ __forceinline__ U128 mul64(uint64_t a, uint64_t b) { return U128{__umul64hi(a, b), a * b}; }

struct Grid {
    uint64_t Ctot;  // C_{N-1}
    uint32_t U;     // u = U 2^-32
    int64_t N;
    float ratio;    // N / Ctot in FP32: only the starting point of the exact division below
    U128 UC;        // U Ctot
};

// A 64-bit unsigned value as FP32 from its two 32-bit halves: 64-bit integer
// conversions run on the narrow FP64 pipe of this GPU, 32-bit ones do not.
__device__ __forceinline__ float u64_to_f32(uint64_t v)
{
    return __fmaf_rn(__uint2float_rn((uint32_t)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

__device__ __forceinline__ Grid make_grid(uint64_t Ctot, uint32_t U, int64_t N)
{
    Grid g;
    g.Ctot = Ctot ? Ctot : 1;
    g.U = U;
    g.N = N;
    g.ratio = __int2float_rn((int32_t)N) / u64_to_f32(g.Ctot);
    g.UC = mul64((uint64_t)U, g.Ctot);
    return g;
}

// #{i in [0, N) : t_i < x}, t_i = (i + U 2^-32) Ctot / N, in exact integer
// arithmetic (x <= Ctot < 2^53, N <= 2^24).  With x N = Q Ctot + R,
// 0 <= R < Ctot, the grid points below x are i = 0 .. Q - 1, and i = Q when
// R / Ctot > U 2^-32, i.e. R 2^32 > U Ctot (128-bit products); so the count is
// Q + [R 2^32 > U Ctot], at most N.  Q starts from an FP32 estimate (relative
// error about 3e-7, so within a few units of Q for N <= 2^24) and is corrected
// exactly: R = x N - Q Ctot is formed modulo 2^64, which is exact while
// |R| < 2^63 (here |R| < 8 Ctot), and moved into [0, Ctot) by whole steps.
// The division x N = Q Ctot + R of a prefix value, kept as the prefix grows.
struct Counter {
    int64_t Q;
    uint64_t R;  // 0 <= R < Ctot
};

__device__ __forceinline__ Counter counter_at(uint64_t x, const Grid &g)
{
    const float qf = fminf(floorf(u64_to_f32(x) * g.ratio), (float)g.N);
    int64_t Q = qf > 0.0f ? (int64_t)__float2int_rz(qf) : 0;
    const int64_t C = (int64_t)g.Ctot;
    int64_t R = (int64_t)(x * (uint64_t)g.N - (uint64_t)Q * g.Ctot);
    while (R < 0) {
        --Q;
        R += C;
    }
    while (R >= C) {
        ++Q;
        R -= C;
    }
    return Counter{Q, (uint64_t)R};
}

// #{i : t_i < x} from x's division: Q + [R 2^32 > U Ctot], at most N.
__device__ __forceinline__ int64_t counter_value(const Counter &c, const Grid &g)
{
    const uint64_t lhi = c.R >> 32, llo = c.R << 32;
    const int64_t n = c.Q + ((lhi > g.UC.hi || (lhi == g.UC.hi && llo > g.UC.lo)) ? 1 : 0);
    return n < g.N ? n : g.N;
}

// The prefix grew by q to x: R grows by q N (< 2^53, since q <= 2^(52 - L) and
// N <= 2^L), which moves Q by its expected offspring count -- whole steps while
// that is small, the division afresh otherwise.
__device__ __forceinline__ void counter_add(Counter &c, uint64_t q, uint64_t x, const Grid &g)
{
    uint64_t R = c.R + q * (uint64_t)g.N;
    if (R < 8 * g.Ctot) {
        while (R >= g.Ctot) {
            R -= g.Ctot;
            ++c.Q;
        }
        c.R = R;
    } else {
        c = counter_at(x, g);
    }
}

// Unnormalised FP32 weight exp(l - max) from the FP32 log-weight; non-finite
// log-weights weigh 0; a degenerate filter weighs uniformly.
__device__ __forceinline__ float weight_f32(float l, float mx, bool degenerate)
{
    if (degenerate) return 1.0f;
    return (l > -INFINITY && l < INFINITY) ? expf(l - mx) : 0.0f;
}

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
    if (mp.kind == kFhnPaper) {  // the stimulus counters start exact
        xp[2 * nn + n0] = (float)x0[2 * nn + n0];
        xp[2 * nn + n1] = (float)x0[2 * nn + n1];
    }
}

// ------------------------------------------------------------------ propagate + weight (Alg. 1 step 2a)
// One CTA of kSubTile / 2 threads per sub-tile of <= kSubTile particles
// (filter aligned, so the grid has many small blocks and little
// wave-quantisation loss); thread i carries particles i and i + kSubTile / 2
// of its sub-tile (two independent generator chains to interleave).  SoA
// state x[v * P + p] (coalesced), K Euler-Maruyama sub-steps in registers,
// then the FP32 log-likelihood; the sub-tile's maximum of it joins the
// filter's maximum by one atomicMax (the first pass of the log-sum-exp).  A
// thread past the sub-tile's end repeats its last particle and stores nothing.
// x_in and x_out may be one buffer (the step propagates in place): a thread
// reads its particles before it writes them, and no other thread touches them;
// the same holds for the lattice kernels below, per particle row.
constexpr int kPropThreads = kSubTile / 2;

// Mode 0: the bootstrap filter.  Mode 1: the auxiliary filter's look-ahead
// (noise-free Euler prediction mu, nothing stored but la_out = log g(y | mu)
// and logw = lw_prev + la_out).  Mode 2: its second stage (logw = log g(y | x)
// - la_src[off + anc]).  Mode 3: carried weights (adaptive resampling):
// logw = lw_prev + log g(y | x).  At least ten CTAs per SM: the compiler
// keeps the two packed chains in 88 registers (11 CTAs, 22 warps per SM);
// held to 64 registers for 16 CTAs the Lorenz interval ran 2 % slower, and to
// 72 or 79 for 14 or 12 CTAs 1 % slower.
template <int D, int Mode>
__global__ void __launch_bounds__(kPropThreads, 10)
    k_propagate_small(ModelParams mp, Key key, const TileDesc *__restrict__ subs, const float *x_in,
                      float *x_out, int64_t P, float *logw, int32_t *fmax_key, const float *obs,
                      int32_t obs_stride, const int32_t *d_t, AuxPtrs aux)
{
    __shared__ float sh[kPropThreads / 32];
    const TileDesc st = subs[blockIdx.x];
    const uint32_t t = (uint32_t)(*d_t + 1);
    const float *y = obs + (obs_stride ? (int64_t)st.m * obs_stride : 0);
    int j[2];
    uint32_t c0[2];
    float xs[2][D];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        j[r] = min((int)threadIdx.x + r * kPropThreads, st.len - 1);
        c0[r] = (uint32_t)(st.lstart + j[r]);
        // with a folded gather the particle starts from its ancestor's variables
        const int64_t src = aux.gather ? (st.gstart - st.lstart) + aux.gather[st.gstart + j[r]] : st.gstart + j[r];
#pragma unroll
        for (int v = 0; v < D; ++v) xs[r][v] = x_in[v * P + src];
    }
    {
        float2 x2[D];
#pragma unroll
        for (int v = 0; v < D; ++v) x2[v] = make_float2(xs[0][v], xs[1][v]);
        propagate_small_x2<D, Mode != 1>(mp, key, kStreamDyn, c0[0], c0[1], t, (uint32_t)st.m, x2);
#pragma unroll
        for (int v = 0; v < D; ++v) xs[0][v] = x2[v].x, xs[1][v] = x2[v].y;
    }
    float l = -INFINITY;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if ((int)threadIdx.x + r * kPropThreads < st.len) {
            const int64_t p = st.gstart + j[r];
            if (Mode != 1) {
#pragma unroll
                for (int v = 0; v < D; ++v) x_out[v * P + p] = xs[r][v];
            }
            float lr = loglik_small<D, float>(mp, y, xs[r]);
            if (Mode == 1) {
                aux.la_out[p] = lr;
                lr = aux.lw_prev[p] + lr;
            } else if (Mode == 3) {
                lr = aux.lw_prev[p] + lr;
            } else if (Mode == 2) {
                lr -= aux.la_src[(st.gstart - st.lstart) + aux.anc[p]];
            }
            logw[p] = lr;
            l = fmaxf(l, lr < INFINITY ? lr : -INFINITY);  // NaN never wins
        }
    }
    const float mx = block_max_f(l, sh);
    if (threadIdx.x == 0 && mx > -INFINITY) atomicMax(&fmax_key[st.m], float_order_key(mx));
}

// One observation interval of lattice particles.  Real = float for the
// filters (state in FP32) and double for the truth record.  Thread (slot s,
// pair q): particle p = blockIdx.x * ppc + s, nodes 2q and 2q+1 (same row);
// threads past ppc * pairs (warp padding) hold no particle.  The v-plane sits
// in shared memory as one (v[2q], v[2q+1]) pair per thread, so every
// neighbour read is a conflict-free 2-word load; a missing neighbour (zero
// flux) reads the node itself, which turns sum_existing(v_n) - count v into
// sum_4(v_n) - 4 v.
template <typename Real, bool Noise = true>
__global__ void __launch_bounds__(1024, 2)
    k_propagate_fhn(ModelParams mp, Key key, uint32_t stream, const int32_t *pfilt, const FilterDesc *filt,
                    const Real *x_in, Real *x_out, int64_t P, float *logw, const float *obs,
                    int32_t obs_stride, const int32_t *obs_slot, const int32_t *d_t, int32_t fixed_c0,
                    int32_t fixed_c2, int32_t t_direct, int32_t ppc, int32_t *fmax_key, int32_t n_steps,
                    AuxPtrs aux, int32_t noise)
{
    using Pair = typename std::conditional<std::is_same<Real, float>::value, float2, double2>::type;
    extern __shared__ unsigned char smem_raw[];
    (void)noise;  // the template parameter Noise decides
    const int J = mp.J, nn = J * J, pairs = nn / 2, half = J / 2;
    Pair *sv = reinterpret_cast<Pair *>(smem_raw);  // [2][ppc][pairs]
    const int slot = (int)threadIdx.x / pairs;
    const int s = min(slot, ppc);                  // s == ppc: padding thread
    const int q = threadIdx.x - min(slot, ppc - 1) * pairs;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(d_t ? *d_t + 1 : t_direct);

    uint32_t c0 = 0, c2 = 0;
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
        const int64_t row_in = aux.gather ? filt[pfilt[p]].off + aux.gather[p] : p;
        const Real *xi = x_in + row_in * (int64_t)mp.dx;
        v0 = xi[n0];
        v1 = xi[n0 + 1];
        w0 = xi[nn + n0];
        w1 = xi[nn + n0 + 1];
    }
    const Real dt = par_dt<Real>(mp);
    const Real sq = par_sq<Real>(mp);
    const Real amp = par<Real>(mp, 6);
    const int64_t stim_steps = mp.ip[7];
    const int blk = (int)mp.ip[8];
    const bool stim_node0 = row < blk && col < blk, stim_node1 = row < blk && col + 1 < blk;
    const int64_t n_base = (int64_t)(t - 1) * mp.K;  // (n - 1) of sub-step k is n_base + k
    const uint32_t blocks_per_step = (uint32_t)(mp.dx / 4);
    // neighbour pairs (the own pair where the lattice ends)
    const int qu = row > 0 ? q - half : q, qd = row < J - 1 ? q + half : q;
    const int ql = col > 0 ? q - 1 : q, qr = col + 2 < J ? q + 1 : q;
    const bool has_left = col > 0, has_right = col + 2 < J;

    for (int k = 0; k < n_steps; ++k) {
        Pair *buf = sv + ((k & 1) * ppc + (active ? s : 0)) * pairs;
        if (active) {
            Pair mine;
            mine.x = v0;
            mine.y = v1;
            buf[q] = mine;
        }
        __syncthreads();
        if (active) {
            const Pair up = buf[qu], dn = buf[qd], lf = buf[ql], rt = buf[qr];
            const Real left = has_left ? lf.y : v0, right = has_right ? rt.x : v1;
            const bool on = (n_base + k) < stim_steps;
            const Real I0 = (on && stim_node0) ? amp : (Real)0, I1 = (on && stim_node1) ? amp : (Real)0;
            const uint32_t bk = (uint32_t)k * blocks_per_step + (uint32_t)q;
            if constexpr (std::is_same<Real, float>::value) {  // both nodes on the packed FP32 pipes
                float2 zv = f2s(0.0f), zw = f2s(0.0f);
                if (Noise) pair_normals_x2(key, c0, t, c2, stream, bk, zv, zw);
                const float2 vv = make_float2(v0, v1), ww = make_float2(w0, w1);
                const float2 lap = pair_laplacian_x2(vv, make_float2(up.x, up.y), make_float2(dn.x, dn.y), left, right);
                const float2 fv = fhn_drift_v_x2(mp, vv, ww, lap, make_float2(I0, I1)), fw = fhn_drift_w_x2(mp, vv, ww);
                const float2 vn = em_update_x2(vv, fv, zv, dt, sq), wn = em_update_x2(ww, fw, zw, dt, sq);
                v0 = vn.x, v1 = vn.y, w0 = wn.x, w1 = wn.y;
            } else {
                Real z[4];
                if (Noise) {
                    normals4<Real>(key, c0, t, c2, stream, bk, z);
                } else {
                    z[0] = z[1] = z[2] = z[3] = (Real)0;
                }
                Real l0, l1;
                pair_laplacian<Real>(v0, v1, up.x, up.y, dn.x, dn.y, left, right, l0, l1);
                const Real fv0 = fhn_drift_v<Real>(mp, v0, w0, l0, I0), fv1 = fhn_drift_v<Real>(mp, v1, w1, l1, I1);
                const Real fw0 = fhn_drift_w<Real>(mp, v0, w0), fw1 = fhn_drift_w<Real>(mp, v1, w1);
                v0 = em_update(v0, fv0, z[0], dt, sq);
                w0 = em_update(w0, fw0, z[1], dt, sq);
                v1 = em_update(v1, fv1, z[2], dt, sq);
                w1 = em_update(w1, fw1, z[3], dt, sq);
            }
        }
    }
    if (active && x_out) {
        Real *xo = x_out + p * (int64_t)mp.dx;
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sl = warp; sl < ppc; sl += nwarps) {  // one warp per particle slot, fixed order
        const int64_t pp = (int64_t)blockIdx.x * ppc + sl;
        float acc = 0.0f;
        for (int i = lane; i < pairs; i += 32) acc += red[sl * pairs + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && pp < P) {
            float l = mp.fhalf_prec * acc;
            if (aux.la_out) {  // auxiliary look-ahead
                aux.la_out[pp] = l;
                l = aux.lw_prev[pp] + l;
            } else if (aux.la_src) {  // auxiliary second stage
                l -= aux.la_src[filt[pfilt[pp]].off + aux.anc[pp]];
            }
            logw[pp] = l;
            if (l > -INFINITY && l < INFINITY) atomicMax(&fmax_key[pfilt[pp]], float_order_key(l));
        }
    }
}

// The same interval with four nodes per thread (lattice sides divisible by
// 4): thread (slot s, quad q) carries nodes 4q..4q+3 of one row, i.e. the two
// pairs 2q and 2q+1 of k_propagate_fhn, with their Philox blocks, the same
// per-node arithmetic (two pair_laplacian calls, the same drift and update
// calls) and the same per-particle reduction over pairs, so its results are
// bit-identical to the pair kernel's.  One barrier and four shared-memory
// loads serve four nodes (up/down as float4, left/right as scalars), and the
// two generator chains interleave.  At most fhn4_max_threads(4 G) threads per
// CTA.
//
// MinB: CTAs the compiler must fit per SM -- four nodes per thread: 2 (63
// registers) or 4 (32, with a little spilling); eight: 2 or 3 (48 registers
// within the 416-thread bound) -- the autotuner times both of each.  G float4 groups per
// thread: G = 1 the four-node kernel, G = 2 eight consecutive nodes of a row
// (sides divisible by 8), the same per-pair arithmetic, Philox blocks and
// reduction order in both, so every width gives the pair kernel's bits.  The
// G groups of a thread sit side by side in shared memory: with G = 2 lanes
// read float4s 32 bytes apart (two-way bank conflicts), yet the conflict-free
// [G][units] order measured slower for its runtime-stride addressing.
template <bool Noise = true, int MinB = 3, int G = 1>
__global__ void __launch_bounds__(fhn4_max_threads(4 * G), MinB)
    k_propagate_fhn4(ModelParams mp, Key key, const int32_t *pfilt, const FilterDesc *filt,
                     const float *x_in, float *x_out, int64_t P, float *logw,
                     const float *obs, int32_t obs_stride, const int32_t *obs_slot, const int32_t *d_t, int32_t ppc,
                     int32_t *fmax_key, int32_t n_steps, AuxPtrs aux, int32_t noise)
{
    constexpr int NV = 4 * G;  // nodes per thread
    extern __shared__ unsigned char smem_raw[];
    (void)noise;  // the template parameter Noise decides
    const int J = mp.J, nn = J * J, units = nn / NV, pairs = nn / 2, urow = J / NV;
    float4 *sv = reinterpret_cast<float4 *>(smem_raw);  // [2][ppc][units][G]
    const int slot = (int)threadIdx.x / units;
    const int s = min(slot, ppc);                   // s == ppc: padding thread
    const int q = threadIdx.x - min(slot, ppc - 1) * units;
    const int64_t p = (int64_t)blockIdx.x * ppc + s;
    const bool active = (s < ppc) && (p < P);
    const uint32_t t = (uint32_t)(*d_t + 1);

    uint32_t c0 = 0, c2 = 0;
    float v[NV], w[NV];
#pragma unroll
    for (int e = 0; e < NV; ++e) v[e] = w[e] = 0.0f;
    const int n0 = NV * q, row = n0 / J, col = n0 - row * J;
    if (active) {
        const int32_t m = pfilt[p];
        c0 = (uint32_t)(p - filt[m].off);
        c2 = (uint32_t)m;
        const int64_t row_in = aux.gather ? filt[m].off + aux.gather[p] : p;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float4 a = *reinterpret_cast<const float4 *>(x_in + row_in * (int64_t)mp.dx + n0 + 4 * g);
            const float4 b = *reinterpret_cast<const float4 *>(x_in + row_in * (int64_t)mp.dx + nn + n0 + 4 * g);
            v[4 * g] = a.x; v[4 * g + 1] = a.y; v[4 * g + 2] = a.z; v[4 * g + 3] = a.w;
            w[4 * g] = b.x; w[4 * g + 1] = b.y; w[4 * g + 2] = b.z; w[4 * g + 3] = b.w;
        }
    }
    const float dt = mp.fdt, sq = mp.fsq, amp = mp.fp[6];
    const int64_t stim_steps = mp.ip[7];
    const int blk = (int)mp.ip[8];
    const int64_t n_base = (int64_t)(t - 1) * mp.K;
    const uint32_t blocks_per_step = (uint32_t)(mp.dx / 4);
    const int qu = row > 0 ? q - urow : q, qd = row < J - 1 ? q + urow : q;
    const bool has_left = col > 0, has_right = col + NV < J;
    const int ql = has_left ? q - 1 : q, qr = has_right ? q + 1 : q;

    for (int k = 0; k < n_steps; ++k) {
        float4 *buf = sv + ((k & 1) * ppc + (active ? s : 0)) * units * G;
        if (active)
#pragma unroll
            for (int g = 0; g < G; ++g) buf[q * G + g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
        __syncthreads();
        if (active) {
            float2 zv[NV / 2], zw[NV / 2];  // pair h: the (v, w) noise of its two nodes
            const uint32_t bk = (uint32_t)k * blocks_per_step + (uint32_t)(NV / 2) * (uint32_t)q;  // pair n0 / 2
            if (Noise) {
#pragma unroll
                for (int h = 0; h < NV / 2; ++h) pair_normals_x2(key, c0, t, c2, kStreamDyn, bk + h, zv[h], zw[h]);
            } else {
#pragma unroll
                for (int h = 0; h < NV / 2; ++h) zv[h] = zw[h] = f2s(0.0f);
            }
            float4 up[G], dn[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                up[g] = buf[qu * G + g];
                dn[g] = buf[qd * G + g];
            }
            const float left = has_left ? buf[ql * G + G - 1].w : v[0];
            const float right = has_right ? buf[qr * G].x : v[NV - 1];
            float2 l[NV / 2];  // every pair's Laplacian from the values before this sub-step
#pragma unroll
            for (int h = 0; h < NV / 2; ++h) {  // pair h: nodes 2h, 2h + 1
                const float4 &u4 = up[h >> 1], &d4 = dn[h >> 1];
                const float2 u2 = (h & 1) ? make_float2(u4.z, u4.w) : make_float2(u4.x, u4.y);
                const float2 d2 = (h & 1) ? make_float2(d4.z, d4.w) : make_float2(d4.x, d4.y);
                const float lf = h == 0 ? left : v[2 * h - 1], rt = h == NV / 2 - 1 ? right : v[2 * h + 2];
                l[h] = pair_laplacian_x2(make_float2(v[2 * h], v[2 * h + 1]), u2, d2, lf, rt);
            }
            const bool on = (n_base + k) < stim_steps;
#pragma unroll
            for (int h = 0; h < NV / 2; ++h) {
                const float2 I = make_float2((on && row < blk && col + 2 * h < blk) ? amp : 0.0f,
                                             (on && row < blk && col + 2 * h + 1 < blk) ? amp : 0.0f);
                const float2 vv = make_float2(v[2 * h], v[2 * h + 1]), ww = make_float2(w[2 * h], w[2 * h + 1]);
                const float2 fv = fhn_drift_v_x2(mp, vv, ww, l[h], I), fw = fhn_drift_w_x2(mp, vv, ww);
                const float2 vn = em_update_x2(vv, fv, zv[h], dt, sq), wn = em_update_x2(ww, fw, zw[h], dt, sq);
                v[2 * h] = vn.x, v[2 * h + 1] = vn.y;
                w[2 * h] = wn.x, w[2 * h + 1] = wn.y;
            }
        }
    }
    if (active && x_out) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            *reinterpret_cast<float4 *>(x_out + p * (int64_t)mp.dx + n0 + 4 * g) =
                make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
            *reinterpret_cast<float4 *>(x_out + p * (int64_t)mp.dx + nn + n0 + 4 * g) =
                make_float4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
    }
    if (!logw) return;
    // per pair, as the pair kernel forms it, then its fixed-order sum over pairs
    float part[NV / 2];
#pragma unroll
    for (int h = 0; h < NV / 2; ++h) part[h] = 0.0f;
    if (active) {
        const int32_t m = pfilt[p];
        const float *y = obs + (obs_stride ? (int64_t)m * obs_stride : 0);
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const int j = obs_slot[n0 + e];
            if (j >= 0) {
                const float d = y[j] - v[e];
                part[e >> 1] += d * d;
            }
        }
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);  // [ppc][pairs]
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
            float lv = mp.fhalf_prec * acc;
            if (aux.la_out) {
                aux.la_out[pp] = lv;
                lv = aux.lw_prev[pp] + lv;
            } else if (aux.la_src) {
                lv -= aux.la_src[filt[pfilt[pp]].off + aux.anc[pp]];
            }
            logw[pp] = lv;
            if (lv > -INFINITY && lv < INFINITY) atomicMax(&fmax_key[pfilt[pp]], float_order_key(lv));
        }
    }
}

// ------------------------------------------------------------------ resampling chain
// The filter fields a tile kernel needs, from the tile descriptor alone.
__device__ __forceinline__ FilterDesc filter_of(const TileDesc &td)
{
    FilterDesc fd{};
    fd.off = td.gstart - td.lstart;
    fd.N = td.N;
    fd.tile_begin = td.tile_begin;
    fd.tile_count = td.tile_count;
    fd.shift = td.shift;
    return fd;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t value)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = value;
}

// The per-filter maximum log-weight from scratch (after pf_set_logw): one
// atomicMax per tile, into keys the caller reset to -inf.
__global__ void __launch_bounds__(kResampleThreads) k_refresh_max(const TileDesc *tiles, const float *logw,
                                                                  int32_t *fmax_key)
{
    __shared__ float sh[kWarps];
    const TileDesc td = tiles[blockIdx.x];
    float mx = -INFINITY;
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const float l = logw[td.gstart + j];
        if (l < INFINITY) mx = fmaxf(mx, l);  // NaN and +inf never win
    }
    mx = block_max_f(mx, sh);
    if (threadIdx.x == 0 && mx > -INFINITY) atomicMax(&fmax_key[td.m], float_order_key(mx));
}

// Pass 2: the filter maximum, then per tile sum w and sum w^2 (compensated
// FP32 pairs, FP64 per tile) and the exact sum of q = floor(w 2^shift);
// stores each q for the scan and clears the ancestor markers.  (Recomputing q
// in the scan instead, and clearing the markers in the ancestor kernel, was
// measured slower: 175 against 136 us for the Lorenz sweep's resampling.)
// Each thread holds IT particles of the tile (strided: coalesced loads).
template <bool Direct, int IT>
__global__ void __launch_bounds__(kResampleThreads) k_weights(ResampleArgs a)
{
    __shared__ double shd[kResampleThreads * 2 + 2];
    __shared__ uint64_t shu[kWarps];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = filter_of(td);
    float mx = 0.0f;
    bool degenerate = false;
    if (!Direct) {
        const float m = float_from_order_key(a.fmax_key[td.m]);
        degenerate = !(m > -INFINITY);
        mx = degenerate ? 0.0f : m;
    }
    double s[2];
    uint64_t qs = 0;
    if (Direct) {
        s[0] = s[1] = 0.0;
        for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
            const int64_t p = td.gstart + j;
            const double w = a.w_direct[p];
            s[0] += w;
            s[1] += w * w;
            qs += quant_f64(w, fd.shift);
            a.B[p] = -1;
        }
        block_sum_dd<2>(s, shd);
    } else {
        FF f[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
        float l[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = threadIdx.x + r * (int)blockDim.x;
            l[r] = j < td.len ? a.logw[td.gstart + j] : -INFINITY;
        }
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = threadIdx.x + r * (int)blockDim.x;
            if (j < td.len) {
                const float w = weight_f32(l[r], mx, degenerate);
                f[0] = ff_add(f[0], w);
                f[1] = ff_add(f[1], __fmul_rn(w, w));
                const uint64_t qv = quant_f32(w, fd.shift);
                qs += qv;
                a.C[td.gstart + j] = qv;  // the scan reads them back
                a.B[td.gstart + j] = -1;
            }
        }
        block_sum_ff<2>(f, s, shd);
    }
    qs = block_sum_u64(qs, shu);
    if (threadIdx.x == 0) {
        double *ts = a.tile_sums + (int64_t)blockIdx.x * kTsCount;
        ts[kTsW] = s[0];
        ts[kTsW2] = s[1];
        a.tile_q[blockIdx.x] = qs;
        if (td.lstart == 0) {
            a.fstats[(int64_t)td.m * kFsCount + kFsMax] = (double)mx;
            a.fstats[(int64_t)td.m * kFsCount + kFsDegenerate] = degenerate ? 1.0 : 0.0;
            if (degenerate) {
                atomicOr(&a.err[0], kErrDegenerate);
                atomicCAS(&a.err[1], -1, td.m);
            }
        }
    }
}

// Pass 3: the exact prefix C of the quantised weights q (tile offset + block
// scan), the counts
// #{i : t_i < C_k}, and the start markers B[lo_k] = k of every particle with
// offspring.  The first tile of each filter also writes the filter's log Z,
// ESS and log G (eq. eqGtN) and its (C_tot, U).  Each thread holds IT
// consecutive particles of the tile.
template <bool Direct, bool Adaptive, int IT>
__global__ void __launch_bounds__(kResampleThreads) k_scan_scatter(ResampleArgs a)
{
    __shared__ double shd[kResampleThreads * 2 + 2];
    __shared__ uint64_t shu[kWarps * 3];
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = filter_of(td);
    const int ti = blockIdx.x - fd.tile_begin;
    if (Adaptive) {
        // every tile of the filter forms the same FP64 sums in the same order: the same decision
        double s[2] = {0.0, 0.0};
        for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) {
            const double *ts = a.tile_sums + (int64_t)(fd.tile_begin + j) * kTsCount;
            s[0] += ts[kTsW];
            s[1] += ts[kTsW2];
        }
        block_sum_dd<2>(s, shd);
        const bool degenerate = a.fstats[(int64_t)td.m * kFsCount + kFsDegenerate] != 0.0;
        const bool resample = degenerate || s[0] * s[0] / s[1] < a.ess_threshold * (double)fd.N;
        if (!resample) {  // identity ancestors: a marker at every particle, the tile starts at itself
            for (int j = threadIdx.x; j < td.len; j += blockDim.x) a.B[td.gstart + j] = td.lstart + j;
            if (threadIdx.x == 0) a.tile_anc0[blockIdx.x] = td.lstart;
            if (ti == 0 && threadIdx.x == 0) {
                double *fs = a.fstats + (int64_t)td.m * kFsCount;
                const double logZ = fs[kFsMax] + log(s[0]);
                fs[kFsLogZ] = logZ;
                fs[kFsEss] = s[0] * s[0] / s[1];
                fs[kFsLogG] += logZ - fs[kFsLse2] + a.log_const;
                fs[kFsLse2] = logZ;
                fs[kFsResampled] = 0.0;
                a.fmax_key[td.m] = kNegInfKey;
            }
            return;
        }
    }
    __shared__ uint32_t shU;
    const int32_t t = a.d_t ? *a.d_t + 1 : 0;
    if (threadIdx.x == 0) {  // the filter's uniform, once per CTA (published by the barriers below)
        if (Direct) shU = (uint32_t)fmin(floor(a.u_direct[td.m] * 4294967296.0), 4294967295.0);
        else shU = philox4x32_10(make_uint4(0u, (uint32_t)t, (uint32_t)td.m, kStreamResample << 24), a.key).x;
    }
    uint64_t q_all = 0, q_before = 0;
    for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) {
        const uint64_t v = a.tile_q[fd.tile_begin + j];
        q_all += v;
        if (j < ti) q_before += v;
    }
    block_sum_u64x2(q_all, q_before, shu);
    const uint64_t Ctot = q_all, Cbefore = q_before;
    const uint32_t U = shU;
    const Grid g = make_grid(Ctot, U, (int64_t)fd.N);

    if (ti == 0) {  // filter scalars (FP64)
        double s[2] = {0.0, 0.0};
        for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) {
            const double *ts = a.tile_sums + (int64_t)(fd.tile_begin + j) * kTsCount;
            s[0] += ts[kTsW];
            s[1] += ts[kTsW2];
        }
        block_sum_dd<2>(s, shd);
        if (threadIdx.x == 0) {
            double *fs = a.fstats + (int64_t)td.m * kFsCount;
            const double logZ = fs[kFsMax] + log(s[0]);
            fs[kFsLogZ] = logZ;
            fs[kFsEss] = s[0] * s[0] / s[1];
            if (Adaptive) {  // the carried weights' log sum, log N after a resampling
                fs[kFsLogG] += logZ - fs[kFsLse2] + a.log_const;
                fs[kFsLse2] = log((double)fd.N);
                fs[kFsResampled] = 1.0;
            } else if (a.d_t) {
                fs[kFsLogG] = (t == 1 ? 0.0 : fs[kFsLogG]) + logZ - log((double)fd.N) + a.log_const;
            }
            a.fint[(int64_t)td.m * 2] = Ctot;
            a.fint[(int64_t)td.m * 2 + 1] = U;
        }
    }
    // blocked items: thread j owns tile positions [j IT, (j + 1) IT)
    const int j0 = threadIdx.x * IT;
    uint64_t q[IT];
    if (Direct) {
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = j0 + r;
            q[r] = j < td.len ? quant_f64(a.w_direct[td.gstart + j], fd.shift) : 0;
        }
    } else if (j0 + IT <= td.len && ((td.gstart + j0) & 1) == 0) {  // q from k_weights, 16-byte loads
#pragma unroll
        for (int r = 0; r < IT; r += 2) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(a.C + td.gstart + j0 + r);
            q[r] = v.x, q[r + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < IT; ++r) q[r] = j0 + r < td.len ? a.C[td.gstart + j0 + r] : 0;
    }
    uint64_t tsum = 0;
#pragma unroll
    for (int r = 0; r < IT; ++r) tsum += q[r];
    // the prefix C_k stays in registers: nothing after the counts reads it
    uint64_t Cprev = Cbefore + block_exscan_u64(tsum, shu + 2 * kWarps);  // C_{k-1} before my first item
    Counter cn = counter_at(Cprev, g);
    int64_t cnt_prev = counter_value(cn, g);
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        const int j = j0 + r;
        if (j >= td.len) break;
        const uint64_t Ck = Cprev + q[r];
        if (q[r] > 0) {
            counter_add(cn, q[r], Ck, g);
            const int64_t cnt = counter_value(cn, g);
            if (cnt > cnt_prev) {
                a.B[fd.off + cnt_prev] = td.lstart + j;
                // the outputs [cnt_prev, cnt) descend from this particle: it is the first
                // ancestor of every output tile that starts in that range (one writer each)
                for (int64_t o = (cnt_prev + kTile - 1) / kTile * kTile; o < cnt; o += kTile)
                    a.tile_anc0[fd.tile_begin + o / kTile] = td.lstart + j;
            }
            cnt_prev = cnt;
        }
        Cprev = Ck;
    }
}

// a_i = max(first ancestor of the tile, max of the markers B[i0..i]); the
// first ancestor comes from the scan (the particle whose offspring range
// holds the tile's first output).
template <int IT>
__device__ __forceinline__ void tile_ancestors(const ResampleArgs &a, const TileDesc &td, int32_t (&anc)[IT], int *shi)
{
    static_assert(IT % 4 == 0, "whole int4 groups of markers per thread");
    const int32_t a0 = a.tile_anc0[blockIdx.x];
    const int j0 = threadIdx.x * IT;
    int b[IT];
    const int32_t *B = a.B + td.gstart + j0;
    if (j0 + IT <= td.len && ((td.gstart + j0) & 3) == 0) {
#pragma unroll
        for (int r = 0; r < IT; r += 4) {
            const int4 v = *reinterpret_cast<const int4 *>(B + r);
            b[r] = v.x, b[r + 1] = v.y, b[r + 2] = v.z, b[r + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            b[r] = -1;
            if (j0 + r < td.len) b[r] = B[r];
        }
    }
    int tmax = -1;
#pragma unroll
    for (int r = 0; r < IT; ++r) tmax = max(tmax, b[r]);
    int run = max(a0, block_exscan_max_i(tmax, shi));
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        run = max(run, b[r]);
        anc[r] = run;
    }
}

// A thread's IT consecutive outputs p0 .. p0 + IT - 1 (the first `left` of
// them exist): their ancestor indices, the gathered SoA state
// x_out[v][p] = x_in[v][off + anc] (not stored when x_out is null: the gather
// is folded into the next propagation) and the running compensated sums of
// what was gathered, item by item.  Whole aligned groups store as int4 / float4.
template <int D, int IT>
__device__ __forceinline__ void gather_items(int32_t *anc_out, int64_t off, int64_t p0, int left,
                                             const int32_t (&anc)[IT], const float *__restrict__ x_in,
                                             float *__restrict__ x_out, int64_t P, FF (&f)[D])
{
    static_assert(IT % 4 == 0, "whole int4 / float4 groups per thread and variable");
#pragma unroll
    for (int v = 0; v < D; ++v) f[v] = FF{0.0f, 0.0f};
    if (!x_out) {  // a folded gather: only the sums of the ancestors' variables
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            if (r < left) {
                anc_out[p0 + r] = anc[r];
#pragma unroll
                for (int v = 0; v < D; ++v) f[v] = ff_add(f[v], x_in[v * P + off + anc[r]]);
            }
        }
        return;
    }
    if (left >= IT && ((p0 | P) & 3) == 0) {
#pragma unroll
        for (int r = 0; r < IT; r += 4)
            *reinterpret_cast<int4 *>(anc_out + p0 + r) = make_int4(anc[r], anc[r + 1], anc[r + 2], anc[r + 3]);
#pragma unroll
        for (int v = 0; v < D; ++v) {
            const float *xi = x_in + v * P + off;
#pragma unroll
            for (int r = 0; r < IT; r += 4) {
                float4 g;
                g.x = xi[anc[r]];
                g.y = xi[anc[r + 1]];
                g.z = xi[anc[r + 2]];
                g.w = xi[anc[r + 3]];
                *reinterpret_cast<float4 *>(x_out + v * P + p0 + r) = g;
                f[v] = ff_add(ff_add(ff_add(ff_add(f[v], g.x), g.y), g.z), g.w);
            }
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        if (r < left) {
            const int64_t p = p0 + r;
            anc_out[p] = anc[r];
            const int64_t src = off + anc[r];
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const float xv = x_in[v * P + src];
                x_out[v * P + p] = xv;
                f[v] = ff_add(f[v], xv);
            }
        }
    }
}

// Ancestors, and for the small models (D > 0) the gather of the SoA state
// and per-tile sums of every variable of the resampled particles (compensated
// FP32 pairs, FP64 per tile).  The last tile
// of a filter to finish (atomic completion counter after a memory fence;
// nothing waits) turns the filter's tile sums into est[m], the per-filter
// estimates of Definition 1, in a fixed order.  The filter's first tile
// resets its maximum log-weight key for the next step (every tile of the scan
// has read it by now).
template <int D, int IT, bool ResetMax>
__global__ void __launch_bounds__(kResampleThreads) k_ancestors_small(ResampleArgs a, const float *__restrict__ x_in,
                                                                      float *__restrict__ x_out, int64_t P,
                                                                      double *tile_est, double *est)
{
    constexpr int DS = D > 0 ? D : 1;
    __shared__ int shi[kWarps];
    __shared__ double shd[kResampleThreads * DS + 2 * DS * 32];
    __shared__ int last;
    const TileDesc td = a.tiles[blockIdx.x];
    const FilterDesc fd = filter_of(td);
    if (ResetMax && td.lstart == 0 && threadIdx.x == 0) a.fmax_key[td.m] = kNegInfKey;
    int32_t anc[IT];
    tile_ancestors<IT>(a, td, anc, shi);
    const int j0 = threadIdx.x * IT;
    if constexpr (D == 0) {
        (void)x_in, (void)x_out, (void)P, (void)tile_est, (void)est, (void)fd;
#pragma unroll
        for (int r = 0; r < IT; ++r)
            if (j0 + r < td.len) a.anc[td.gstart + j0 + r] = anc[r];
        return;
    } else {
        FF f[D];
        gather_items<D, IT>(a.anc, fd.off, td.gstart + j0, td.len - j0, anc, x_in, x_out, P, f);
        double s[D];
        block_sum_ff<D>(f, s, shd);
        if (fd.tile_count == 1) {  // the tile is the filter
            if (threadIdx.x < D) est[(int64_t)td.m * D + threadIdx.x] = s[threadIdx.x] / (double)fd.N;
            return;
        }
        if (threadIdx.x == 0) {
#pragma unroll
            for (int v = 0; v < D; ++v) tile_est[(int64_t)blockIdx.x * D + v] = s[v];
            __threadfence();
            last = (atomicAdd(&a.done[td.m], 1) == fd.tile_count - 1);
        }
        __syncthreads();
        if (!last) return;
        // the filter's estimate: tiles strided over the threads, then a fixed tree
        double part[D];
#pragma unroll
        for (int v = 0; v < D; ++v) part[v] = 0.0;
        for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x)
#pragma unroll
            for (int v = 0; v < D; ++v) part[v] += __ldcg(&tile_est[(int64_t)(fd.tile_begin + j) * D + v]);
        block_sum_dd<D>(part, shd);
        if (threadIdx.x < D) est[(int64_t)td.m * D + threadIdx.x] = part[threadIdx.x] / (double)fd.N;
        if (threadIdx.x == 0) a.done[td.m] = 0;
    }
}

// A whole filter of at most kTile particles per CTA: the resampling step of
// that filter in one kernel, with the quantised weights, the prefix and the
// start markers in shared memory instead of global scratch.  The same
// arithmetic as k_weights -> k_scan_scatter -> k_ancestors_small (or
// k_ancestors when D = 0): FP32 weights and compensated FP32 sums, the FP64
// normaliser, the exact q = floor(w 2^shift), the exact prefix C_k and the
// counts #{i : t_i < C_k} (Algorithm 1 step 2b, systematic form), the
// ancestor max-scan, then (D > 0) the gather of the SoA state and the
// per-filter means.  The results are those of the tile chain bit for bit.
// CTA b handles tile tile0 + b, which must be the filter's only tile.
template <int D, int IT>
__global__ void __launch_bounds__(kTile / IT, 8) k_resample_whole(ResampleArgs a, int32_t tile0,
                                                                     const float *__restrict__ x_in,
                                                                     float *__restrict__ x_out, int64_t P, double *est)
{
    __shared__ uint64_t shq[kTile];
    __shared__ int32_t shB[kTile];
    __shared__ double shd[4];  // block_sum_ff results; its scratch is shB, then shq
    __shared__ uint64_t shu[kWarps * 2];
    __shared__ int shi[kWarps];
    const int tix = tile0 + blockIdx.x;
    const TileDesc td = a.tiles[tix];
    const FilterDesc fd = filter_of(td);
    const float m0 = float_from_order_key(a.fmax_key[td.m]);
    const bool degenerate = !(m0 > -INFINITY);
    const float mx = degenerate ? 0.0f : m0;

    // weights, their sums and the quantised weights (strided: coalesced loads)
    FF f[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    uint64_t qs = 0;
    {
        float l[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = threadIdx.x + r * (int)blockDim.x;
            l[r] = j < td.len ? a.logw[td.gstart + j] : -INFINITY;
        }
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = threadIdx.x + r * (int)blockDim.x;
            if (j < td.len) {
                const float w = weight_f32(l[r], mx, degenerate);
                f[0] = ff_add(f[0], w);
                f[1] = ff_add(f[1], __fmul_rn(w, w));
                const uint64_t qv = quant_f32(w, fd.shift);
                qs += qv;
                shq[j] = qv;
            }
        }
    }
    double s[2];
    static_assert(2 * 2 * kResampleThreads * sizeof(float) <= sizeof(shB), "scratch of the weight sums");
    block_sum_ff<2>(f, s, reinterpret_cast<float *>(shB), shd);
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) shB[j] = -1;
    const uint64_t Ctot = block_sum_u64(qs, shu);  // its barriers also publish shq and shB
    const int32_t t = a.d_t ? *a.d_t + 1 : 0;
    const uint32_t U = philox4x32_10(make_uint4(0u, (uint32_t)t, (uint32_t)td.m, kStreamResample << 24), a.key).x;
    const Grid g = make_grid(Ctot, U, (int64_t)fd.N);
    if (threadIdx.x == 0) {  // the FP64 scalars follow in k_whole_finish, a thread per filter
        double *fs = a.fstats + (int64_t)td.m * kFsCount;
        fs[kFsMax] = (double)mx;
        fs[kFsDegenerate] = degenerate ? 1.0 : 0.0;
        if (degenerate) {
            atomicOr(&a.err[0], kErrDegenerate);
            atomicCAS(&a.err[1], -1, td.m);
        }
        fs[kFsS0] = s[0];
        fs[kFsS1] = s[1];
        a.fint[(int64_t)td.m * 2] = Ctot;
        a.fint[(int64_t)td.m * 2 + 1] = U;
        a.fmax_key[td.m] = kNegInfKey;
    }

    // exact prefix (blocked items), counts and start markers
    const int j0 = threadIdx.x * IT;
    {
        uint64_t q[IT];
        uint64_t tsum = 0;
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            q[r] = j0 + r < td.len ? shq[j0 + r] : 0;
            tsum += q[r];
        }
        uint64_t Cprev = block_exscan_u64(tsum, shu + kWarps);
        Counter cn = counter_at(Cprev, g);
        int64_t cnt_prev = counter_value(cn, g);
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = j0 + r;
            if (j >= td.len) break;
            const uint64_t Ck = Cprev + q[r];
            if (q[r] > 0) {
                counter_add(cn, q[r], Ck, g);
                const int64_t cnt = counter_value(cn, g);
                if (cnt > cnt_prev) shB[cnt_prev] = j;
                cnt_prev = cnt;
            }
            Cprev = Ck;
        }
    }
    __syncthreads();

    // ancestors: running max of the markers (output 0 always has one)
    int b[IT];
    int tmax = -1;
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        b[r] = j0 + r < td.len ? shB[j0 + r] : -1;
        tmax = max(tmax, b[r]);
    }
    int run = block_exscan_max_i(tmax, shi);
    if constexpr (D == 0) {
        (void)x_in, (void)x_out, (void)P, (void)est;
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            run = max(run, b[r]);
            if (j0 + r < td.len) a.anc[td.gstart + j0 + r] = run;
        }
    } else {
        constexpr int DD = D;
        int32_t anc[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            run = max(run, b[r]);
            anc[r] = run;
        }
        FF fx[DD];
        gather_items<DD, IT>(a.anc, fd.off, td.gstart + j0, td.len - j0, anc, x_in, x_out, P, fx);
        double sx[DD];
        static_assert(2 * DD * kResampleThreads * sizeof(float) <= sizeof(shq), "scratch of the state sums");
        block_sum_ff<DD>(fx, sx, reinterpret_cast<float *>(shq), shd);  // q is no longer needed
        if (threadIdx.x < DD) est[(int64_t)td.m * DD + threadIdx.x] = sx[threadIdx.x];  // divided by N later
    }
}

// Warp-level forms of the block primitives above (every lane gets the result).
__device__ __forceinline__ FF warp_sum_ff(FF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
}

__device__ __forceinline__ uint64_t warp_exscan_u64(uint64_t v, int lane)
{
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    return inc - v;
}

__device__ __forceinline__ int warp_exscan_max_i(int v, int lane)
{
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, n);
    }
    const int ex = __shfl_up_sync(0xffffffffu, inc, 1);
    return lane == 0 ? -1 : ex;
}

// Filters of at most 32 kWarpItems particles: one warp per filter, kWarpFilters
// filters per CTA, every reduction and scan in warp shuffles (no block
// barrier).  The same arithmetic as k_resample_whole: FP32 weights, the
// compensated sums (a lane's items in order, then an xor tree), the exact
// q = floor(w 2^shift), prefix C_k and counts, the ancestor max-scan, the
// gather and the sums of the gathered state; the FP64 scalars follow in
// k_whole_finish.  Warp w of CTA b takes one-tile filter tile0 + 4 b + w.
constexpr int kWarpItems = 8;
constexpr int kWarpFilters = 4;
constexpr int kWarpFilterMax = 32 * kWarpItems;

template <int D>
__global__ void __launch_bounds__(32 * kWarpFilters, 8) k_resample_warp(ResampleArgs a, int32_t tile0, int32_t n,
                                                                     const float *__restrict__ x_in,
                                                                     float *__restrict__ x_out, int64_t P, double *est)
{
    constexpr int IT = kWarpItems;
    __shared__ uint64_t shq_all[kWarpFilters][kWarpFilterMax];
    __shared__ int32_t shB_all[kWarpFilters][kWarpFilterMax];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fi = blockIdx.x * kWarpFilters + w;
    if (fi >= n) return;  // the whole warp leaves together
    uint64_t *shq = shq_all[w];
    int32_t *shB = shB_all[w];
    const TileDesc td = a.tiles[tile0 + fi];
    const FilterDesc fd = filter_of(td);
    const float m0 = float_from_order_key(a.fmax_key[td.m]);
    const bool degenerate = !(m0 > -INFINITY);
    const float mx = degenerate ? 0.0f : m0;

    // weights, their sums and the quantised weights (strided: coalesced loads)
    FF f0{0.0f, 0.0f}, f1{0.0f, 0.0f};
    uint64_t qs = 0;
    {
        float l[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = lane + 32 * r;
            l[r] = j < td.len ? a.logw[td.gstart + j] : -INFINITY;
        }
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = lane + 32 * r;
            shB[j] = -1;
            if (j < td.len) {
                const float wt = weight_f32(l[r], mx, degenerate);
                f0 = ff_add(f0, wt);
                f1 = ff_add(f1, __fmul_rn(wt, wt));
                const uint64_t qv = quant_f32(wt, fd.shift);
                qs += qv;
                shq[j] = qv;
            }
        }
    }
    f0 = warp_sum_ff(f0);
    f1 = warp_sum_ff(f1);
    const uint64_t Ctot = warp_sum_u64(qs);
    const int32_t t = a.d_t ? *a.d_t + 1 : 0;
    const uint32_t U = philox4x32_10(make_uint4(0u, (uint32_t)t, (uint32_t)td.m, kStreamResample << 24), a.key).x;
    const Grid g = make_grid(Ctot, U, (int64_t)fd.N);
    if (lane == 0) {
        double *fs = a.fstats + (int64_t)td.m * kFsCount;
        fs[kFsMax] = (double)mx;
        fs[kFsDegenerate] = degenerate ? 1.0 : 0.0;
        if (degenerate) {
            atomicOr(&a.err[0], kErrDegenerate);
            atomicCAS(&a.err[1], -1, td.m);
        }
        fs[kFsS0] = ff_to_double(f0);
        fs[kFsS1] = ff_to_double(f1);
        a.fint[(int64_t)td.m * 2] = Ctot;
        a.fint[(int64_t)td.m * 2 + 1] = U;
        a.fmax_key[td.m] = kNegInfKey;
    }
    __syncwarp();

    // exact prefix (blocked items), counts and start markers
    const int j0 = lane * IT;
    {
        uint64_t q[IT];
        uint64_t tsum = 0;
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            q[r] = j0 + r < td.len ? shq[j0 + r] : 0;
            tsum += q[r];
        }
        uint64_t Cprev = warp_exscan_u64(tsum, lane);
        Counter cn = counter_at(Cprev, g);
        int64_t cnt_prev = counter_value(cn, g);
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            const int j = j0 + r;
            if (j >= td.len) break;
            const uint64_t Ck = Cprev + q[r];
            if (q[r] > 0) {
                counter_add(cn, q[r], Ck, g);
                const int64_t cnt = counter_value(cn, g);
                if (cnt > cnt_prev) shB[cnt_prev] = j;
                cnt_prev = cnt;
            }
            Cprev = Ck;
        }
    }
    __syncwarp();

    // ancestors: running max of the markers (output 0 always has one)
    int b[IT];
    int tmax = -1;
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        b[r] = j0 + r < td.len ? shB[j0 + r] : -1;
        tmax = max(tmax, b[r]);
    }
    int run = warp_exscan_max_i(tmax, lane);
    if constexpr (D == 0) {
        (void)x_in, (void)x_out, (void)P, (void)est;
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            run = max(run, b[r]);
            if (j0 + r < td.len) a.anc[td.gstart + j0 + r] = run;
        }
    } else {
        int32_t anc[IT];
#pragma unroll
        for (int r = 0; r < IT; ++r) {
            run = max(run, b[r]);
            anc[r] = run;
        }
        FF fx[D];
        gather_items<D, IT>(a.anc, fd.off, td.gstart + j0, td.len - j0, anc, x_in, x_out, P, fx);
#pragma unroll
        for (int v = 0; v < D; ++v) {
            const FF sv = warp_sum_ff(fx[v]);
            if (lane == 0) est[(int64_t)td.m * D + v] = ff_to_double(sv);  // divided by N later
        }
    }
}

// The FP64 scalars of the one-tile filters, a thread per filter: log Z, ESS,
// log G (eq. eqGtN) and the per-filter means from the sums k_resample_whole
// left (the expressions of k_scan_scatter and k_ancestors_small, so the
// results are those of the tile chain).  Thirty-two filters share each FP64
// instruction here instead of one thread per CTA issuing them alone: FP64 is
// a narrow pipe on this GPU.
__global__ void __launch_bounds__(32) k_whole_finish(const TileDesc *__restrict__ tiles, int32_t tile0, int32_t n,
                                                      int dx, double *fstats, double *est, const int32_t *d_t,
                                                      double log_const)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TileDesc td = tiles[tile0 + i];
    double *fs = fstats + (int64_t)td.m * kFsCount;
    const double s0 = fs[kFsS0], s1 = fs[kFsS1];
    const double logZ = fs[kFsMax] + log(s0);
    fs[kFsLogZ] = logZ;
    fs[kFsEss] = s0 * s0 / s1;
    if (d_t) {
        const int32_t t = *d_t + 1;
        fs[kFsLogG] = (t == 1 ? 0.0 : fs[kFsLogG]) + logZ - log((double)td.N) + log_const;
    }
    for (int v = 0; v < dx; ++v) est[(int64_t)td.m * dx + v] /= (double)td.N;
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

// Per-filter means of every variable of the resampled lattice particles
// (estimator after eq. eqGtN): CTA (chunk of <= kMeanChunk particles of one
// filter, variable block).  Each thread sums its variable over the chunk in
// a compensated FP32 pair (coalesced over the block's variables), writes the
// FP64 partial, and the last CTA of the filter's chunks (completion counter,
// reset by that CTA) adds the partials in chunk order in FP64: deterministic,
// and parallel over particles, so one filter of many particles is as fast as
// many small ones.
__device__ __forceinline__ float aux_weight(float l, float mx)
{
    return (mx > -INFINITY && l > -INFINITY && l < INFINITY) ? expf(l - mx) : 0.0f;  // NaN weighs nothing
}

__global__ void __launch_bounds__(256) k_mean_rows(const FilterDesc *filt, const TileDesc *__restrict__ chunks,
                                                   const float *__restrict__ x, int dx, double *part, int32_t *cnt,
                                                   double *est, const float *__restrict__ lw2,
                                                   const int32_t *__restrict__ fmax2, const double *fstats)
{
    __shared__ int last;
    const TileDesc ch = chunks[blockIdx.x];
    const FilterDesc fd = filt[ch.m];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    // auxiliary filter: weighted by exp(lw2 - max), divided by the filter's sum of those weights
    const float mx = lw2 ? float_from_order_key(fmax2[ch.m]) : 0.0f;
    const double denom = lw2 ? fstats[(int64_t)ch.m * kFsCount + kFsSumW] : (double)fd.N;
    double mine = 0.0;
    if (v < dx) {
        const float *base = x + ch.gstart * (int64_t)dx + v;
        FF acc{0.0f, 0.0f};
        int i = 0;
        for (; i + 8 <= ch.len; i += 8) {  // eight loads in flight, then the ordered adds
            float r[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = base[(int64_t)(i + k) * dx];
            if (lw2) {
#pragma unroll
                for (int k = 0; k < 8; ++k) r[k] *= aux_weight(lw2[ch.gstart + i + k], mx);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = ff_add(acc, r[k]);
        }
        for (; i < ch.len; ++i)
            acc = ff_add(acc, base[(int64_t)i * dx] * (lw2 ? aux_weight(lw2[ch.gstart + i], mx) : 1.0f));
        mine = ff_to_double(acc);
    }
    if (fd.mc_count == 1) {  // the whole filter in this chunk (uniform over the CTA)
        if (v < dx) est[(int64_t)ch.m * dx + v] = mine / denom;
        return;
    }
    if (v < dx) part[(int64_t)blockIdx.x * dx + v] = mine;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *c = cnt + (int64_t)ch.m * gridDim.y + blockIdx.y;
        last = (atomicAdd(c, 1) == fd.mc_count - 1);
        if (last) *c = 0;  // every other chunk of this filter and block has counted
    }
    __syncthreads();
    if (last && v < dx) {
        __threadfence();
        double s = 0.0;
        for (int k = 0; k < fd.mc_count; ++k) s += __ldcg(&part[(int64_t)(fd.mc_begin + k) * dx + v]);
        est[(int64_t)ch.m * dx + v] = s / denom;
    }
}

// Second stage of the auxiliary particle filter, per filter: from the
// second-stage log-weights lw2 and their maximum (order keys), sum w and
// sum w^2 (ESS), log sum w (log G_t gains lse2_t - lse2_{t-1}: the first-stage
// factor sum W lambda with W normalised, times the mean second-stage weight),
// and for the small models the weighted means of the D variables.  Tile
// partials in compensated FP32 pairs, FP64 across tiles, combined in tile order
// by the filter's last tile (completion counter kept at 0 between steps).
// The lattice gather fused with the per-filter means: CTA (chunk of <=
// kMeanChunk particles of one filter, variable block) copies the ancestors'
// rows x_out[p] = x_in[off + anc[p]] variable by variable (coalesced over the
// block's variables) and sums what it copied, in the order and with the
// arithmetic of k_mean_rows (unweighted), so the estimates are identical and
// the resampled state is not read a second time.  With x_out null the rows
// are only summed: the gather itself is left to the next propagation, which
// loads each particle's ancestor row directly (the same values, so the same
// estimates).
__global__ void __launch_bounds__(256) k_gather_mean_rows(const FilterDesc *filt, const TileDesc *__restrict__ chunks,
                                                          const int32_t *__restrict__ anc,
                                                          const float *__restrict__ x_in, float *__restrict__ x_out,
                                                          int dx, double *part, int32_t *cnt, double *est)
{
    __shared__ int last;
    const TileDesc ch = chunks[blockIdx.x];
    const FilterDesc fd = filt[ch.m];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    double mine = 0.0;
    if (v < dx) {
        const int32_t *a = anc + ch.gstart;
        float *dst = x_out ? x_out + ch.gstart * (int64_t)dx + v : nullptr;
        const float *src = x_in + fd.off * (int64_t)dx + v;
        FF acc{0.0f, 0.0f};
        int i = 0;
        const bool store = x_out != nullptr;
        for (; i + 8 <= ch.len; i += 8) {  // eight rows in flight, then the ordered adds
            float r[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = src[(int64_t)a[i + k] * dx];
            if (store) {
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[(int64_t)(i + k) * dx] = r[k];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = ff_add(acc, r[k]);
        }
        for (; i < ch.len; ++i) {
            const float r = src[(int64_t)a[i] * dx];
            if (store) dst[(int64_t)i * dx] = r;
            acc = ff_add(acc, r);
        }
        mine = ff_to_double(acc);
    }
    const double denom = (double)fd.N;
    if (fd.mc_count == 1) {
        if (v < dx) est[(int64_t)ch.m * dx + v] = mine / denom;
        return;
    }
    if (v < dx) part[(int64_t)blockIdx.x * dx + v] = mine;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *c = cnt + (int64_t)ch.m * gridDim.y + blockIdx.y;
        last = (atomicAdd(c, 1) == fd.mc_count - 1);
        if (last) *c = 0;
    }
    __syncthreads();
    if (last && v < dx) {
        __threadfence();
        double s = 0.0;
        for (int k = 0; k < fd.mc_count; ++k) s += __ldcg(&part[(int64_t)(fd.mc_begin + k) * dx + v]);
        est[(int64_t)ch.m * dx + v] = s / denom;
    }
}

// k_gather_mean_rows with four consecutive variables per thread (dx % 4 ==
// 0, rows 16-byte aligned): float4 loads of the ancestors' rows (eight rows
// in flight, 128 bytes per thread), each variable's compensated sum over the
// chunk's outputs in the same order, so the copies and the estimates are
// k_gather_mean_rows' own.
__global__ void __launch_bounds__(256, 4) k_gather_mean_rows4(const FilterDesc *filt, const TileDesc *__restrict__ chunks,
                                                           const int32_t *__restrict__ anc,
                                                           const float *__restrict__ x_in, float *__restrict__ x_out,
                                                           int dx, double *part, int32_t *cnt, double *est)
{
    __shared__ int last;
    const TileDesc ch = chunks[blockIdx.x];
    const FilterDesc fd = filt[ch.m];
    const int v4 = blockIdx.y * blockDim.x + threadIdx.x, dx4 = dx >> 2;
    double mine[4] = {0.0, 0.0, 0.0, 0.0};
    if (v4 < dx4) {
        const int32_t *a = anc + ch.gstart;
        const float4 *src = reinterpret_cast<const float4 *>(x_in + fd.off * (int64_t)dx) + v4;
        float4 *dst = x_out ? reinterpret_cast<float4 *>(x_out + ch.gstart * (int64_t)dx) + v4 : nullptr;
        FF acc[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
        int i = 0;
        for (; i + 8 <= ch.len; i += 8) {
            float4 r[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = src[(int64_t)a[i + k] * dx4];
            if (dst) {
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[(int64_t)(i + k) * dx4] = r[k];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc[0] = ff_add(acc[0], r[k].x);
                acc[1] = ff_add(acc[1], r[k].y);
                acc[2] = ff_add(acc[2], r[k].z);
                acc[3] = ff_add(acc[3], r[k].w);
            }
        }
        for (; i < ch.len; ++i) {
            const float4 r = src[(int64_t)a[i] * dx4];
            if (dst) dst[(int64_t)i * dx4] = r;
            acc[0] = ff_add(acc[0], r.x);
            acc[1] = ff_add(acc[1], r.y);
            acc[2] = ff_add(acc[2], r.z);
            acc[3] = ff_add(acc[3], r.w);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) mine[e] = ff_to_double(acc[e]);
    }
    const double denom = (double)fd.N;
    if (fd.mc_count == 1) {
        if (v4 < dx4)
#pragma unroll
            for (int e = 0; e < 4; ++e) est[(int64_t)ch.m * dx + 4 * v4 + e] = mine[e] / denom;
        return;
    }
    if (v4 < dx4)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[(int64_t)blockIdx.x * dx + 4 * v4 + e] = mine[e];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *c = cnt + (int64_t)ch.m * gridDim.y + blockIdx.y;
        last = (atomicAdd(c, 1) == fd.mc_count - 1);
        if (last) *c = 0;
    }
    __syncthreads();
    if (last && v4 < dx4) {
        __threadfence();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int v = 4 * v4 + e;
            double sum = 0.0;
            for (int k = 0; k < fd.mc_count; ++k) sum += __ldcg(&part[(int64_t)(fd.mc_begin + k) * dx + v]);
            est[(int64_t)ch.m * dx + v] = sum / denom;
        }
    }
}

// k_mean_rows with four consecutive variables per thread (dx % 4 == 0, rows
// 16-byte aligned): float4 loads, four times the bytes in flight per
// instruction; each variable's compensated sum runs over the chunk's particles
// in the same order, so the estimates are k_mean_rows' own.
__global__ void __launch_bounds__(256) k_mean_rows4(const FilterDesc *filt, const TileDesc *__restrict__ chunks,
                                                    const float *__restrict__ x, int dx, double *part, int32_t *cnt,
                                                    double *est, const float *__restrict__ lw2,
                                                    const int32_t *__restrict__ fmax2, const double *fstats)
{
    __shared__ int last;
    const TileDesc ch = chunks[blockIdx.x];
    const FilterDesc fd = filt[ch.m];
    const int v4 = blockIdx.y * blockDim.x + threadIdx.x, dx4 = dx >> 2;
    const float mx = lw2 ? float_from_order_key(fmax2[ch.m]) : 0.0f;
    const double denom = lw2 ? fstats[(int64_t)ch.m * kFsCount + kFsSumW] : (double)fd.N;
    double mine[4] = {0.0, 0.0, 0.0, 0.0};
    if (v4 < dx4) {
        const float4 *base = reinterpret_cast<const float4 *>(x + ch.gstart * (int64_t)dx) + v4;
        FF acc[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
        int i = 0;
        for (; i + 16 <= ch.len; i += 16) {  // sixteen rows in flight, then the ordered adds
            float4 r[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) r[k] = base[(int64_t)(i + k) * dx4];
            if (lw2) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float wk = aux_weight(lw2[ch.gstart + i + k], mx);
                    r[k].x *= wk, r[k].y *= wk, r[k].z *= wk, r[k].w *= wk;
                }
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                acc[0] = ff_add(acc[0], r[k].x);
                acc[1] = ff_add(acc[1], r[k].y);
                acc[2] = ff_add(acc[2], r[k].z);
                acc[3] = ff_add(acc[3], r[k].w);
            }
        }
        for (; i < ch.len; ++i) {
            float4 r = base[(int64_t)i * dx4];
            const float wk = lw2 ? aux_weight(lw2[ch.gstart + i], mx) : 1.0f;
            acc[0] = ff_add(acc[0], r.x * wk);
            acc[1] = ff_add(acc[1], r.y * wk);
            acc[2] = ff_add(acc[2], r.z * wk);
            acc[3] = ff_add(acc[3], r.w * wk);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) mine[e] = ff_to_double(acc[e]);
    }
    if (fd.mc_count == 1) {  // the whole filter in this chunk (uniform over the CTA)
        if (v4 < dx4)
#pragma unroll
            for (int e = 0; e < 4; ++e) est[(int64_t)ch.m * dx + 4 * v4 + e] = mine[e] / denom;
        return;
    }
    if (v4 < dx4)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[(int64_t)blockIdx.x * dx + 4 * v4 + e] = mine[e];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *c = cnt + (int64_t)ch.m * gridDim.y + blockIdx.y;
        last = (atomicAdd(c, 1) == fd.mc_count - 1);
        if (last) *c = 0;  // every other chunk of this filter and block has counted
    }
    __syncthreads();
    if (last && v4 < dx4) {
        __threadfence();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            double sum = 0.0;
            for (int k = 0; k < fd.mc_count; ++k) sum += __ldcg(&part[(int64_t)(fd.mc_begin + k) * dx + 4 * v4 + e]);
            est[(int64_t)ch.m * dx + 4 * v4 + e] = sum / denom;
        }
    }
}

// Threads per CTA of the four-variable row kernels: the warp multiple in
// [128, 256] that wastes the fewest threads on the last column block (the
// smallest on a tie: more CTAs in flight).  At least 64 threads keep the
// column blocks within the ceil(dx / 256) completion counters per filter.
static int rows4_threads(int dx4)
{
    int best = 128;
    for (int th = 128; th <= 256; th += 32)
        if ((dx4 + th - 1) / th * th < (dx4 + best - 1) / best * best) best = th;
    return best;
}

// The ancestors' rows of x_in: their per-filter means, and the copy into x_out
// unless it is null (the gather folded into the next propagation).
static void launch_gather_means(const Ctx &c, const float *x_in, float *x_out, cudaStream_t s)
{
    const int dx = c.mp.dx;
    if (dx % 4 == 0) {
        const int th = rows4_threads(dx / 4);
        dim3 g(c.n_mchunks, (dx / 4 + th - 1) / th);
        k_gather_mean_rows4<<<g, th, 0, s>>>(c.filt, c.mchunks, c.anc, x_in, x_out, dx, c.mean_part, c.mean_cnt,
                                             c.est);
    } else {
        dim3 g(c.n_mchunks, (dx + 255) / 256);
        k_gather_mean_rows<<<g, 256, 0, s>>>(c.filt, c.mchunks, c.anc, x_in, x_out, dx, c.mean_part, c.mean_cnt,
                                            c.est);
    }
}

// The (weighted) per-filter means of the lattice particles xn.
void launch_mean_rows(const Ctx &c, const float *xn, const float *lw2, const int32_t *fmax2, const double *fstats,
                      cudaStream_t s)
{
    const int dx = c.mp.dx;
    if (dx % 4 == 0) {
        const int th = rows4_threads(dx / 4);
        dim3 g(c.n_mchunks, (dx / 4 + th - 1) / th);
        k_mean_rows4<<<g, th, 0, s>>>(c.filt, c.mchunks, xn, dx, c.mean_part, c.mean_cnt, c.est, lw2, fmax2, fstats);
    } else {
        dim3 g(c.n_mchunks, (dx + 255) / 256);
        k_mean_rows<<<g, 256, 0, s>>>(c.filt, c.mchunks, xn, dx, c.mean_part, c.mean_cnt, c.est, lw2, fmax2, fstats);
    }
}

template <int D, bool Evidence = true>
__global__ void __launch_bounds__(kResampleThreads)
    k_weight_stats(const TileDesc *tiles, const FilterDesc *filt, const float *__restrict__ lw2,
                   const int32_t *__restrict__ fmax2, const float *__restrict__ x, int64_t P, double *tile_sums,
                   double *tile_est, int32_t *done, double *fstats, double *est, int32_t *err)
{
    constexpr int NV = D + 2;  // w, w^2, w x_v
    __shared__ double shd[kResampleThreads * NV + 2 * NV * 32];
    __shared__ int last;
    const TileDesc td = tiles[blockIdx.x];
    const FilterDesc fd = filter_of(td);
    const float mx = float_from_order_key(fmax2[td.m]);
    FF f[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) f[i] = FF{0.0f, 0.0f};
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const int64_t p = td.gstart + j;
        const float w = aux_weight(lw2[p], mx);
        f[0] = ff_add(f[0], w);
        f[1] = ff_add(f[1], w * w);
#pragma unroll
        for (int v = 0; v < D; ++v) f[2 + v] = ff_add(f[2 + v], w * x[v * P + p]);
    }
    double s[NV];
    block_sum_ff<NV>(f, s, shd);
    if (fd.tile_count > 1) {
        if (threadIdx.x == 0) {
            tile_sums[(int64_t)blockIdx.x * kTsCount + kTsW] = s[0];
            tile_sums[(int64_t)blockIdx.x * kTsCount + kTsW2] = s[1];
#pragma unroll
            for (int v = 0; v < D; ++v) tile_est[(int64_t)blockIdx.x * D + v] = s[2 + v];
            __threadfence();
            last = (atomicAdd(&done[td.m], 1) == fd.tile_count - 1);
        }
        __syncthreads();
        if (!last) return;
        double part[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = 0.0;
        for (int j = threadIdx.x; j < fd.tile_count; j += blockDim.x) {
            const int64_t b = fd.tile_begin + j;
            part[0] += __ldcg(&tile_sums[b * kTsCount + kTsW]);
            part[1] += __ldcg(&tile_sums[b * kTsCount + kTsW2]);
#pragma unroll
            for (int v = 0; v < D; ++v) part[2 + v] += __ldcg(&tile_est[b * D + v]);
        }
        block_sum_dd<NV>(part, shd);
#pragma unroll
        for (int i = 0; i < NV; ++i) s[i] = part[i];
        if (threadIdx.x == 0) done[td.m] = 0;
    }
    if (threadIdx.x == 0) {
        double *fs = fstats + (int64_t)td.m * kFsCount;
        const double sw = s[0];
        if (!(sw > 0.0)) {
            atomicOr(&err[0], kErrDegenerate);
            atomicCAS(&err[1], -1, td.m);
        }
        if (Evidence) {  // the auxiliary filter's second stage
            const double lse2 = (double)mx + log(sw);
            fs[kFsEss] = sw * sw / s[1];
            fs[kFsLogG] += lse2 - fs[kFsLse2];
            fs[kFsLse2] = lse2;
        }
        fs[kFsSumW] = sw;
#pragma unroll
        for (int v = 0; v < D; ++v) est[(int64_t)td.m * D + v] = s[2 + v] / sw;
    }
}

// Definition 1: ens[v] = (1/M) sum_m est[m][v] in FP64, one CTA per variable:
// each thread adds its filters m = t, t + T, ... in order, each warp folds
// its lanes by an xor tree and the first warp folds the warps' sums the same
// way (a fixed order: deterministic, and ten dependent FP64 adds after the
// strided ones instead of a 32-long chain); advances the step counter.
__global__ void __launch_bounds__(1024) k_ensemble(const double *est, int dx, int32_t M, double *ens, int32_t *d_t)
{
    __shared__ double sh[32];
    const int v = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double s = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += est[(int64_t)m * dx + v];
    s = warp_sum_d(s);
    if (nw > 1) {
        if (lane == 0) sh[w] = s;
        __syncthreads();
        if (w == 0) s = warp_sum_d(lane < nw ? sh[lane] : 0.0);
    }
    if (threadIdx.x == 0) {
        ens[v] = s / (double)M;
        if (v == 0 && d_t) *d_t += 1;
    }
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
    if (mp.kind == kFhnPaper) {
        x[2 * nn + n0] = x0[2 * nn + n0];
        x[2 * nn + n1] = x0[2 * nn + n1];
    }
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
__global__ void k_rng_philox(int64_t n, const uint4 *ctr, Key key, uint4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

__global__ void k_rng_normals(int64_t n, const uint4 *ctr, Key key, float4 *z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(ctr[i], key);
    float a, b, c, d;
    box_muller<float>(r.x, r.y, a, b);
    box_muller<float>(r.z, r.w, c, d);
    z[i] = make_float4(a, b, c, d);
}

// ------------------------------------------------------------------ launchers
namespace {

// Threads of a lattice CTA: ppc particles x J^2/2 node pairs, rounded up to
// whole warps (the extra threads hold no particle).  want = 0 picks as many
// particles as fit in 1024 threads (at most 8).
// Threads of a lattice CTA carrying up to `want` particles (0: as many as fit
// in 1024 threads -- fhn4_max_threads(nodes) for the four- and eight-node
// kernels --, at most 8) with `nodes` (2, 4 or 8) nodes per thread.
int fhn_threads(const ModelParams &mp, int *ppc, int want = 0, int nodes = 2)
{
    const int per = mp.J * mp.J / nodes, cap = nodes >= 4 ? fhn4_max_threads(nodes) : 1024;
    int n = 1;
    while ((n + 1) * per <= cap && n < 8) ++n;
    if (want > 0 && want < n) n = want;
    *ppc = n;
    return (n * per + 31) / 32 * 32;
}

size_t fhn_smem(const ModelParams &mp, int threads, int ppc, size_t real_bytes)
{
    const size_t planes = 2 * (size_t)ppc * mp.J * mp.J * real_bytes;  // two buffers of ppc v-planes
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
    k_propagate_small<D, 0><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xi, xo, c.P, c.logw, c.fmax_key,
                                                              d_obs, stride, c.d_t, AuxPtrs{});
    return cudaGetLastError();
}

// Threads of the M-average: enough to have a few filters each, 32..1024.
int ensemble_threads(int32_t M)
{
    int th = 32;
    while (th < 1024 && th * 8 < M) th *= 2;
    return th;
}

ResampleArgs ctx_args(const Ctx &c)
{
    ResampleArgs a{};
    a.tiles = c.tiles;
    a.filt = c.filt;
    a.logw = c.logw;
    a.key = c.key;
    a.d_t = c.d_t;
    a.fmax_key = c.fmax_key;
    a.tile_sums = c.tile_sums;
    a.tile_q = c.tile_q;
    a.fstats = c.fstats;
    a.fint = c.fint;
    a.C = c.C;
    a.B = c.B;
    a.anc = c.anc;
    a.tile_anc0 = c.tile_anc0;
    a.err = c.err;
    a.done = c.done;
    a.log_const = -0.5 * c.mp.dy * log(2.0 * M_PI * c.mp.sigma_obs * c.mp.sigma_obs);
    a.ess_threshold = c.ess_threshold;
    return a;
}

}  // namespace

cudaError_t launch_init(const Ctx &c, cudaStream_t s)
{
    if (is_lattice(c.mp.kind)) {
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

// n_steps lattice sub-steps of every particle, xi -> xo, with the weights and
// per-filter maxima when `weigh` (the pair or the four-node kernel).
cudaError_t launch_fhn_interval(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                int32_t n_steps, bool weigh, cudaStream_t s, float *logw = nullptr,
                                int32_t *fmax = nullptr, AuxPtrs aux = AuxPtrs{}, int32_t noise = 1)
{
    if (!logw) logw = c.logw;
    if (!fmax) fmax = c.fmax_key;
    const int nodes = fhn_nodes(c);
    int ppc;
    const int threads = fhn_threads(c.mp, &ppc, c.fhn_ppc, nodes);
    const size_t smem = fhn_smem(c.mp, threads, ppc, sizeof(float));
    const unsigned grid = (unsigned)((c.P + ppc - 1) / ppc);
    static bool carveout_set = false;  // prefer shared memory so that several CTAs fit per SM
    if (!carveout_set) {
        cudaFuncSetAttribute(k_propagate_fhn<float, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn<float, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<true, 2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<false, 2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<true, 3, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<false, 3, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<true, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<false, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<true, 4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_propagate_fhn4<false, 4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        carveout_set = true;
    }
    float *lw = weigh ? logw : nullptr;
    int32_t *fm = weigh ? fmax : nullptr;
    const bool four = c.fhn_quad_ctas == 4;
    if (nodes == 8) {  // eight nodes per thread: built for two or three CTAs per SM
        const bool three = c.fhn_quad_ctas >= 3;
        if (noise && three)
            k_propagate_fhn4<true, 3, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw,
                                                                     d_obs, stride, c.obs_slot, c.d_t, ppc, fm, n_steps,
                                                                     aux, 1);
        else if (noise)
            k_propagate_fhn4<true, 2, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw,
                                                                     d_obs, stride, c.obs_slot, c.d_t, ppc, fm, n_steps,
                                                                     aux, 1);
        else if (three)
            k_propagate_fhn4<false, 3, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw,
                                                                      d_obs, stride, c.obs_slot, c.d_t, ppc, fm,
                                                                      n_steps, aux, 0);
        else
            k_propagate_fhn4<false, 2, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw,
                                                                      d_obs, stride, c.obs_slot, c.d_t, ppc, fm,
                                                                      n_steps, aux, 0);
    } else if (nodes == 4 && noise && four)
        k_propagate_fhn4<true, 4><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw, d_obs,
                                                              stride, c.obs_slot, c.d_t, ppc, fm, n_steps, aux, 1);
    else if (nodes == 4 && noise)
        k_propagate_fhn4<true, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw, d_obs,
                                                              stride, c.obs_slot, c.d_t, ppc, fm, n_steps, aux, 1);
    else if (nodes == 4 && four)
        k_propagate_fhn4<false, 4><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw, d_obs,
                                                               stride, c.obs_slot, c.d_t, ppc, fm, n_steps, aux, 0);
    else if (nodes == 4)
        k_propagate_fhn4<false, 2><<<grid, threads, smem, s>>>(c.mp, c.key, c.pfilt, c.filt, xi, xo, c.P, lw, d_obs,
                                                               stride, c.obs_slot, c.d_t, ppc, fm, n_steps, aux, 0);
    else if (noise)
        k_propagate_fhn<float, true><<<grid, threads, smem, s>>>(c.mp, c.key, kStreamDyn, c.pfilt, c.filt, xi, xo, c.P,
                                                                 lw, d_obs, stride, c.obs_slot, c.d_t, 0, 0, 0, ppc,
                                                                 fm, n_steps, aux, 1);
    else
        k_propagate_fhn<float, false><<<grid, threads, smem, s>>>(c.mp, c.key, kStreamDyn, c.pfilt, c.filt, xi, xo,
                                                                  c.P, lw, d_obs, stride, c.obs_slot, c.d_t, 0, 0, 0,
                                                                  ppc, fm, n_steps, aux, 0);
    return cudaGetLastError();
}

cudaError_t launch_propagate(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                             cudaStream_t s)
{
    if (is_lattice(c.mp.kind)) {
        if (c.mp.kind == kFhnPaper)
            return launch_fhnp_interval(c, d_obs, stride, xi, xo, c.mp.K, c.logw, c.fmax_key, AuxPtrs{}, 1, s);
        return launch_fhn_interval(c, d_obs, stride, xi, xo, c.mp.K, true, s);
    }
    switch (c.mp.dx) {
    case 1: return propagate_small_launch<1>(c, d_obs, stride, xi, xo, s);
    case 2: return propagate_small_launch<2>(c, d_obs, stride, xi, xo, s);
    case 3: return propagate_small_launch<3>(c, d_obs, stride, xi, xo, s);
    case 4: return propagate_small_launch<4>(c, d_obs, stride, xi, xo, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fhn_substeps(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                const int32_t *gather, int32_t n_steps, cudaStream_t s)
{
    const AuxPtrs g{nullptr, nullptr, nullptr, nullptr, gather};
    return launch_fhn_interval(c, d_obs, stride, xi, xo, n_steps, false, s, nullptr, nullptr, g, 1);
}

cudaError_t launch_refresh_max(const Ctx &c, cudaStream_t s)
{
    k_fill_i32<<<(c.M + 255) / 256, 256, 0, s>>>(c.fmax_key, c.M, kNegInfKey);
    k_refresh_max<<<c.n_tiles, kResampleThreads, 0, s>>>(c.tiles, c.logw, c.fmax_key);
    return cudaGetLastError();
}

// The tile chain over the first n tiles: weights -> scan -> ancestors (with the
// gather and the per-filter means for the small models, D > 0).  Each CTA of
// c.resample_threads threads covers one tile with 4 particles per thread, or 8
// where 4 per thread do not cover the longest tile.
template <int D, bool Adaptive, int IT>
void tile_chain_it(const Ctx &c, const ResampleArgs &a, int32_t n, const float *xi, float *xo, cudaStream_t s)
{
    const int th = c.resample_threads;
    k_weights<false, IT><<<n, th, 0, s>>>(a);
    k_scan_scatter<false, Adaptive, IT><<<n, th, 0, s>>>(a);
    k_ancestors_small<D, IT, true><<<n, th, 0, s>>>(a, xi, xo, c.P, c.tile_est, c.est);
}

template <int D, bool Adaptive>
void tile_chain(const Ctx &c, const ResampleArgs &a, int32_t n, const float *xi, float *xo, cudaStream_t s)
{
    if (n <= 0) return;
    if (c.resample_threads * kItems >= c.max_tile_len) tile_chain_it<D, Adaptive, kItems>(c, a, n, xi, xo, s);
    else tile_chain_it<D, Adaptive, 2 * kItems>(c, a, n, xi, xo, s);
}

// Adaptive resampling: the weights carried into the next step (0 where the
// filter resampled, the step's log-weight where it kept its particles; the
// particles' order is unchanged then, the gather being the identity), and
// their per-filter maximum for the weighted estimates.
__global__ void __launch_bounds__(256) k_carry(const int32_t *__restrict__ pfilt, const double *__restrict__ fstats,
                                               const float *__restrict__ logw, float *lw_c, int32_t *fmax_c, int64_t P)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t m = p < P ? pfilt[p] : -1;
    float l = -INFINITY;
    if (p < P) {
        l = fstats[(int64_t)m * kFsCount + kFsResampled] != 0.0 ? 0.0f : logw[p];
        lw_c[p] = l;
    }
    // one atomic per run of equal filters within the warp (a single large filter would
    // otherwise serialise every particle on one address)
    const int lane = threadIdx.x & 31;
    float mx = (l > -INFINITY && l < INFINITY) ? l : -INFINITY;
    const int32_t m0 = __shfl_sync(0xffffffffu, m, 0);
    const bool uniform = __all_sync(0xffffffffu, m == m0);
    if (uniform) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && m0 >= 0 && mx > -INFINITY) atomicMax(&fmax_c[m0], float_order_key(mx));
    } else if (m >= 0 && mx > -INFINITY) {
        atomicMax(&fmax_c[m], float_order_key(mx));
    }
}

template <int D>
cudaError_t adaptive_small(const Ctx &c, const ResampleArgs &a, const float *d_obs, int32_t stride, float *x,
                           float *xn, cudaStream_t s)
{
    const int th = c.resample_threads;
    k_propagate_small<D, 3><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, x, x, c.P, c.logw, c.fmax_key,
                                                              d_obs, stride, c.d_t, AuxPtrs{c.lw2, nullptr, nullptr,
                                                                                            nullptr});
    tile_chain<D, true>(c, a, c.n_tiles, x, xn, s);
    k_carry<<<(unsigned)((c.P + 255) / 256), 256, 0, s>>>(c.pfilt, c.fstats, c.logw, c.lw2, c.fmax2, c.P);
    k_weight_stats<D, false><<<c.n_tiles, th, 0, s>>>(c.tiles, c.filt, c.lw2, c.fmax2, xn, c.P, c.tile_sums,
                                                      c.tile_est, c.done, c.fstats, c.est, c.err);
    return cudaGetLastError();
}

cudaError_t launch_adaptive_step(const Ctx &c, const float *d_obs, int32_t stride, cudaStream_t s)
{
    ResampleArgs a = ctx_args(c);
    a.ess_threshold = c.ess_threshold;
    const int dx = c.mp.dx, th = c.resample_threads;
    float *x = c.x[c.cur];
    float *xn = c.x[c.cur ^ 1];
    k_fill_i32<<<(c.M + 255) / 256, 256, 0, s>>>(c.fmax2, c.M, kNegInfKey);
    cudaError_t e = cudaSuccess;
    if (is_lattice(c.mp.kind)) {
        const AuxPtrs carry{c.lw2, c.la, nullptr, nullptr};
        if (c.mp.kind == kFhnPaper)
            e = launch_fhnp_interval(c, d_obs, stride, x, x, c.mp.K, c.logw, c.fmax_key, carry, 1, s);
        else
            e = launch_fhn_interval(c, d_obs, stride, x, x, c.mp.K, true, s, c.logw, c.fmax_key, carry, 1);
        if (e != cudaSuccess) return e;
        tile_chain<0, true>(c, a, c.n_tiles, nullptr, nullptr, s);
        k_gather_rows<<<(unsigned)c.P, 256, 0, s>>>(c.anc, c.pfilt, c.filt, reinterpret_cast<const float4 *>(x),
                                                   reinterpret_cast<float4 *>(xn), dx / 4);
        k_carry<<<(unsigned)((c.P + 255) / 256), 256, 0, s>>>(c.pfilt, c.fstats, c.logw, c.lw2, c.fmax2, c.P);
        k_weight_stats<0, false><<<c.n_tiles, th, 0, s>>>(c.tiles, c.filt, c.lw2, c.fmax2, nullptr, c.P, c.tile_sums,
                                                          nullptr, c.done, c.fstats, c.est, c.err);
        launch_mean_rows(c, xn, c.lw2, c.fmax2, c.fstats, s);
    } else {
        switch (dx) {
        case 1: e = adaptive_small<1>(c, a, d_obs, stride, x, xn, s); break;
        case 2: e = adaptive_small<2>(c, a, d_obs, stride, x, xn, s); break;
        case 3: e = adaptive_small<3>(c, a, d_obs, stride, x, xn, s); break;
        case 4: e = adaptive_small<4>(c, a, d_obs, stride, x, xn, s); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    k_ensemble<<<dx, ensemble_threads(c.M), 0, s>>>(c.est, dx, c.M, c.ens, c.d_t);
    return cudaGetLastError();
}

// Bootstrap resampling of every filter (no adaptive decision): filters of
// several tiles take the tile chain (weights, scan, ancestors), the tiles of
// one-tile filters follow theirs and take one fused kernel per filter.
// Small models: with the gather and the per-filter means.
// One launch of the fused kernel per size class, with as many threads as the
// class's largest filter needs (kItems particles each).
template <int D>
void resample_whole(const Ctx &c, const ResampleArgs &a, const float *xi, float *xo, cudaStream_t s)
{
    {  // class 0: a warp per filter
        const int32_t b0 = c.whole_bounds[0], n = c.whole_bounds[1] - b0;
        if (n) k_resample_warp<D><<<(n + kWarpFilters - 1) / kWarpFilters, 32 * kWarpFilters, 0, s>>>(a, b0, n, xi, xo,
                                                                                                      c.P, c.est);
    }
    for (int k = 1; k < kWholeClasses; ++k) {  // class k: a CTA of 32 2^k threads, kWholeItems particles each
        const int32_t b0 = c.whole_bounds[k], n = c.whole_bounds[k + 1] - b0;
        if (n) k_resample_whole<D, kWholeItems><<<n, 32 << k, 0, s>>>(a, b0, xi, xo, c.P, c.est);
    }
    const int32_t b0 = c.whole_bounds[0], n = c.whole_bounds[kWholeClasses] - b0;
    // one warp per CTA: the FP64 work spreads over every SM's FP64 units
    if (n) k_whole_finish<<<(n + 31) / 32, 32, 0, s>>>(c.tiles, b0, n, D, c.fstats, c.est, a.d_t, a.log_const);
}

// The two groups of filters share no data (every buffer is split by filter,
// tile or particle, and the error word takes atomics), so when both are present
// the fused one-tile kernels run on the side stream next to the tile chain:
// fork from s, join back into s before anything reads every filter.
cudaStream_t fork_side(const Ctx &c, cudaStream_t s)
{
    const bool both = c.n_multi_tiles > 0 && c.whole_bounds[kWholeClasses] > c.whole_bounds[0];
    if (!both) return s;
    cudaEventRecord(c.fork_ev, s);
    cudaStreamWaitEvent(c.side_stream, c.fork_ev, 0);
    return c.side_stream;
}

void join_side(const Ctx &c, cudaStream_t side, cudaStream_t s)
{
    if (side == s) return;
    cudaEventRecord(c.join_ev, side);
    cudaStreamWaitEvent(s, c.join_ev, 0);
}

template <int D>
void resample_small(const Ctx &c, const ResampleArgs &a, const float *xi, float *xo, int th, cudaStream_t s)
{
    const int32_t nm = c.n_multi_tiles;
    const cudaStream_t side = fork_side(c, s);
    resample_whole<D>(c, a, xi, xo, side);
    if (nm) {
        tile_chain<D, false>(c, a, nm, xi, xo, s);
    }
    join_side(c, side, s);
}

// The whole bootstrap resampling up to the ancestors (lattice models).
void resample_ancestors(const Ctx &c, const ResampleArgs &a, int th, cudaStream_t s)
{
    const int32_t nm = c.n_multi_tiles;
    const cudaStream_t side = fork_side(c, s);
    resample_whole<0>(c, a, nullptr, nullptr, side);
    if (nm) {
        tile_chain<0, false>(c, a, nm, nullptr, nullptr, s);
    }
    join_side(c, side, s);
}

// One step of the ensemble of auxiliary particle filters: look-ahead weights
// (noise-free prediction), first-stage systematic resampling and gather, the
// second-stage propagation and weights, weighted estimates, the M-average.
template <int D>
cudaError_t apf_small(const Ctx &c, const ResampleArgs &a, const float *d_obs, int32_t stride, const float *x, float *xn,
                      cudaStream_t s)
{
    const int th = c.resample_threads;
    k_propagate_small<D, 1><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, x, nullptr, c.P, c.logw,
                                                              c.fmax_key, d_obs, stride, c.d_t,
                                                              AuxPtrs{c.lw2, c.la, nullptr, nullptr});
    resample_small<D>(c, a, x, xn, th, s);
    k_propagate_small<D, 2><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xn, xn, c.P, c.lw2, c.fmax2, d_obs,
                                                              stride, c.d_t, AuxPtrs{nullptr, nullptr, c.la, c.anc});
    k_weight_stats<D><<<c.n_tiles, th, 0, s>>>(c.tiles, c.filt, c.lw2, c.fmax2, xn, c.P, c.tile_sums, c.tile_est,
                                               c.done, c.fstats, c.est, c.err);
    return cudaGetLastError();
}

cudaError_t launch_apf_step(const Ctx &c, const float *d_obs, int32_t stride, cudaStream_t s)
{
    const ResampleArgs a = ctx_args(c);
    const int dx = c.mp.dx, th = c.resample_threads;
    const float *x = c.x[c.cur];
    float *xn = c.x[c.cur ^ 1];
    k_fill_i32<<<(c.M + 255) / 256, 256, 0, s>>>(c.fmax2, c.M, kNegInfKey);
    cudaError_t e = cudaSuccess;
    if (is_lattice(c.mp.kind)) {
        if (c.mp.kind == kFhnPaper)
            e = launch_fhnp_interval(c, d_obs, stride, x, nullptr, c.mp.K, c.logw, c.fmax_key,
                                     AuxPtrs{c.lw2, c.la, nullptr, nullptr}, 0, s);
        else
            e = launch_fhn_interval(c, d_obs, stride, x, nullptr, c.mp.K, true, s, c.logw, c.fmax_key,
                                    AuxPtrs{c.lw2, c.la, nullptr, nullptr}, 0);
        if (e != cudaSuccess) return e;
        resample_ancestors(c, a, th, s);
        // the second stage starts from the ancestors' rows of x: no separate gather pass
        if (c.mp.kind == kFhnPaper)
            e = launch_fhnp_interval(c, d_obs, stride, x, xn, c.mp.K, c.lw2, c.fmax2,
                                     AuxPtrs{nullptr, nullptr, c.la, c.anc, c.anc}, 1, s);
        else
            e = launch_fhn_interval(c, d_obs, stride, x, xn, c.mp.K, true, s, c.lw2, c.fmax2,
                                    AuxPtrs{nullptr, nullptr, c.la, c.anc, c.anc}, 1);
        if (e != cudaSuccess) return e;
        k_weight_stats<0><<<c.n_tiles, th, 0, s>>>(c.tiles, c.filt, c.lw2, c.fmax2, nullptr, c.P, c.tile_sums, nullptr,
                                                   c.done, c.fstats, c.est, c.err);
        launch_mean_rows(c, xn, c.lw2, c.fmax2, c.fstats, s);
    } else {
        switch (dx) {
        case 1: e = apf_small<1>(c, a, d_obs, stride, x, xn, s); break;
        case 2: e = apf_small<2>(c, a, d_obs, stride, x, xn, s); break;
        case 3: e = apf_small<3>(c, a, d_obs, stride, x, xn, s); break;
        case 4: e = apf_small<4>(c, a, d_obs, stride, x, xn, s); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    k_ensemble<<<dx, ensemble_threads(c.M), 0, s>>>(c.est, dx, c.M, c.ens, c.d_t);
    return cudaGetLastError();
}

// Small models: the resampled SoA state written out from the ancestors,
// x_out[v][p] = x_in[v][off_m + anc[p]], a CTA per tile.
template <int D>
__global__ void __launch_bounds__(256) k_gather_small(const TileDesc *__restrict__ tiles, const int32_t *__restrict__ anc,
                                                      const float *__restrict__ x_in, float *__restrict__ x_out,
                                                      int64_t P)
{
    const TileDesc td = tiles[blockIdx.x];
    const int64_t off = td.gstart - td.lstart;
    for (int j = threadIdx.x; j < td.len; j += blockDim.x) {
        const int64_t p = td.gstart + j, src = off + anc[p];
#pragma unroll
        for (int v = 0; v < D; ++v) x_out[v * P + p] = x_in[v * P + src];
    }
}

// Bootstrap filters with the resampling's gather folded into the next
// propagation: x_in holds the previous step's weighted particles and `gather`
// (null on a first step) their ancestors, so particle p starts from particle
// off_m + gather[p] of x_in; the result goes to x_out (never in place: a
// particle of x_in is read by all its offspring).
cudaError_t launch_propagate_fold(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                  const int32_t *gather, cudaStream_t s)
{
    const AuxPtrs g{nullptr, nullptr, nullptr, nullptr, gather};
    if (c.mp.kind == kFhnPaper) return launch_fhnp_interval(c, d_obs, stride, xi, xo, c.mp.K, c.logw, c.fmax_key, g, 1, s);
    if (is_lattice(c.mp.kind)) return launch_fhn_interval(c, d_obs, stride, xi, xo, c.mp.K, true, s, c.logw, c.fmax_key, g, 1);
    switch (c.mp.dx) {
    case 1: k_propagate_small<1, 0><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xi, xo, c.P, c.logw, c.fmax_key, d_obs, stride, c.d_t, g); break;
    case 2: k_propagate_small<2, 0><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xi, xo, c.P, c.logw, c.fmax_key, d_obs, stride, c.d_t, g); break;
    case 3: k_propagate_small<3, 0><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xi, xo, c.P, c.logw, c.fmax_key, d_obs, stride, c.d_t, g); break;
    case 4: k_propagate_small<4, 0><<<c.n_subs, kPropThreads, 0, s>>>(c.mp, c.key, c.subs, xi, xo, c.P, c.logw, c.fmax_key, d_obs, stride, c.d_t, g); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ... and its resampling: the ancestors and the per-filter means of the
// ancestors' values (read, not copied), then the M-average.
cudaError_t launch_resample_fold(const Ctx &c, const float *x, cudaStream_t s)
{
    const ResampleArgs a = ctx_args(c);
    const int dx = c.mp.dx, th = c.resample_threads;
    if (is_lattice(c.mp.kind)) {
        resample_ancestors(c, a, th, s);
        launch_gather_means(c, x, nullptr, s);
    } else {
        switch (dx) {
        case 1: resample_small<1>(c, a, x, nullptr, th, s); break;
        case 2: resample_small<2>(c, a, x, nullptr, th, s); break;
        case 3: resample_small<3>(c, a, x, nullptr, th, s); break;
        case 4: resample_small<4>(c, a, x, nullptr, th, s); break;
        default: return cudaErrorInvalidValue;
        }
    }
    k_ensemble<<<dx, ensemble_threads(c.M), 0, s>>>(c.est, dx, c.M, c.ens, c.d_t);
    return cudaGetLastError();
}

// The resampled particles as a state of their own: the ancestors' rows
// (lattice) or variables (small models) of x_in.
cudaError_t launch_materialise(const Ctx &c, const float *xi, float *xo, cudaStream_t s)
{
    if (is_lattice(c.mp.kind)) {
        k_gather_rows<<<(unsigned)c.P, 256, 0, s>>>(c.anc, c.pfilt, c.filt, reinterpret_cast<const float4 *>(xi),
                                                   reinterpret_cast<float4 *>(xo), c.mp.dx / 4);
        return cudaGetLastError();
    }
    switch (c.mp.dx) {
    case 1: k_gather_small<1><<<c.n_tiles, 256, 0, s>>>(c.tiles, c.anc, xi, xo, c.P); break;
    case 2: k_gather_small<2><<<c.n_tiles, 256, 0, s>>>(c.tiles, c.anc, xi, xo, c.P); break;
    case 3: k_gather_small<3><<<c.n_tiles, 256, 0, s>>>(c.tiles, c.anc, xi, xo, c.P); break;
    case 4: k_gather_small<4><<<c.n_tiles, 256, 0, s>>>(c.tiles, c.anc, xi, xo, c.P); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_resample(const Ctx &c, const float *xi, float *xo, cudaStream_t s)
{
    const ResampleArgs a = ctx_args(c);
    const int dx = c.mp.dx, th = c.resample_threads;
    if (is_lattice(c.mp.kind)) {
        resample_ancestors(c, a, th, s);
        launch_gather_means(c, xi, xo, s);
    } else {
        switch (dx) {
        case 1: resample_small<1>(c, a, xi, xo, th, s); break;
        case 2: resample_small<2>(c, a, xi, xo, th, s); break;
        case 3: resample_small<3>(c, a, xi, xo, th, s); break;
        case 4: resample_small<4>(c, a, xi, xo, th, s); break;
        default: return cudaErrorInvalidValue;
        }
    }
    k_ensemble<<<dx, ensemble_threads(c.M), 0, s>>>(c.est, dx, c.M, c.ens, c.d_t);
    return cudaGetLastError();
}

cudaError_t launch_systematic(int32_t M, int32_t n_tiles, const ResampleArgs &a, cudaStream_t s)
{
    (void)M;
    k_weights<true, kItems><<<n_tiles, kResampleThreads, 0, s>>>(a);
    k_scan_scatter<true, false, kItems><<<n_tiles, kResampleThreads, 0, s>>>(a);
    k_ancestors_small<0, kItems, false><<<n_tiles, kResampleThreads, 0, s>>>(a, nullptr, nullptr, 0, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_rng_philox(int64_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_rng_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        n, reinterpret_cast<const uint4 *>(ctr), make_key((uint64_t)k0 | ((uint64_t)k1 << 32)),
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
    if (!is_lattice(mp.kind)) {
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
    const int threads = (pairs + 31) / 32 * 32;
    const size_t smem = fhn_smem(mp, threads, 1, sizeof(double));
    for (int32_t t = 1; t <= T; ++t) {
        const double *xi = d_x + (int64_t)(t - 1) * mp.dx;
        double *xo = d_x + (int64_t)t * mp.dx;
        if (mp.kind == kFhnPaper) {
            const cudaError_t e = launch_fhnp_truth_step(mp, key, record, t, xi, xo, s);
            if (e != cudaSuccess) return e;
        } else {
            k_propagate_fhn<double><<<1, threads, smem, s>>>(mp, key, kStreamTruth, nullptr, nullptr, xi, xo, 1,
                                                             nullptr, nullptr, 0, nullptr, nullptr, 0, record, t, 1,
                                                             nullptr, mp.K, AuxPtrs{}, 1);
        }
        if (d_y)
            k_observe<<<(mp.dy + 255) / 256, 256, 0, s>>>(mp, key, d_obs_idx, t, record, xo,
                                                          d_y + (int64_t)(t - 1) * mp.dy);
    }
    return cudaGetLastError();
}

}  // namespace pf
