// pf_internal.h -- host-side layout of a filter context and the kernel
// launchers shared by the translation units of the library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pf.h"
#include "pf_device.cuh"

namespace pf {

// Particles of all filters sit contiguously, filter after filter.  Each filter
// is cut into tiles of at most kTile particles; a tile never spans two filters,
// so every per-filter reduction is a reduction over that filter's tiles.
constexpr int kTile = 1024;
constexpr int kResampleThreads = 256;
constexpr int kItems = kTile / kResampleThreads;  // particles per thread in the tile kernels
// Size classes of one-tile filters for the fused resampling kernels: class c
// holds N <= 32 kWholeItems 2^c; class 0 runs a warp per filter, class c > 0
// CTAs of 32 2^c threads, kWholeItems particles per thread.
constexpr int kWholeItems = 8;
constexpr int kWholeClasses = 3;
static_assert((32 * kWholeItems << (kWholeClasses - 1)) == kTile, "the largest class fills a tile");
constexpr int kSubTile = 128;                     // propagation block of the thread-per-particle models
// Threads per CTA of the four- and eight-node lattice kernels at most (their
// launch bounds): 512 with four nodes per thread; 416 with eight, so that the
// eight-node build for three CTAs per SM gets 48 registers instead of 40 and
// stops spilling in its loop (400 threads carry two 40x40 particles).  A
// particle's J^2 / nodes threads must fit.
constexpr int fhn4_max_threads(int nodes) { return nodes == 8 ? 416 : 512; }
inline bool fhn_nodes_fit(int J, int nodes) { return J % nodes == 0 && J * J / nodes <= fhn4_max_threads(nodes); }
// The same bound of the paper lattice's four- and eight-node kernels.
constexpr int kFhnp4MaxThreads = 512;
constexpr int kMeanChunk = 256;                   // particles per partial sum of the lattice means

// A tile also carries the fields of its filter that the tile kernels need,
// so that a CTA reads one descriptor, not a tile and then (dependent) its
// filter.
struct TileDesc {
    int32_t m;           // filter
    int32_t lstart;      // filter-local index of the tile's first particle
    int32_t len;         // particles in the tile
    int32_t N;           // the filter's particles
    int64_t gstart;      // global index of the tile's first particle
    int32_t tile_begin;  // the filter's first tile
    int32_t tile_count;  // the filter's tiles
    int32_t shift;       // the filter's weight quantisation exponent (FilterDesc::shift)
    int32_t pad;
};

struct FilterDesc {
    int64_t off;         // global index of particle 0
    int32_t N;           // particles
    int32_t tile_begin;  // first tile
    int32_t tile_count;  // tiles
    int32_t shift;       // 52 - ceil(log2 N): weight quantisation exponent
    int32_t mc_begin;    // first chunk of kMeanChunk particles (lattice means)
    int32_t mc_count;    // chunks
    int32_t pad;
};

// Order-preserving int image of a float (signed-int max = float max), so the
// per-filter maximum log-weight can be taken with atomicMax.
__host__ __device__ __forceinline__ int32_t float_order_key(float f)
{
    union { float f; int32_t i; } u{f};
    return u.i >= 0 ? u.i : (u.i ^ 0x7FFFFFFF);
}
__host__ __device__ __forceinline__ float float_from_order_key(int32_t k)
{
    union { int32_t i; float f; } u{k >= 0 ? k : (k ^ 0x7FFFFFFF)};
    return u.f;
}
constexpr int32_t kNegInfKey = (int32_t)0x807FFFFF;  // float_order_key(-inf)

// Per-filter scalars kept in FP64 on the device.
enum FStat : int {
    kFsLogZ = 0, kFsEss = 1, kFsLogG = 2, kFsMax = 3, kFsDegenerate = 4, kFsFallback = 5,
    kFsLse2 = 6,  // auxiliary filter: log sum of the second-stage weights (log N before the first step)
    kFsSumW = 7,  // auxiliary filter: sum of exp(lw2 - max) behind the weighted means
    kFsResampled = 8,  // adaptive resampling: 1 where the filter resampled this step
    kFsS0 = 9, kFsS1 = 10,  // one-tile filters: sum w and sum w^2, finished by a thread per filter
    kFsCount = 12
};
// Per-tile FP64 partial sums.
enum TSum : int { kTsW = 0, kTsW2 = 1, kTsCount = 2 };

// Device error word: bit flags plus the first offending filter.
enum : int32_t { kErrDegenerate = 1, kErrTimeout = 2 };

// Everything the resampling kernels need, by value.
struct ResampleArgs {
    const TileDesc *tiles;
    const FilterDesc *filt;
    const float *logw;       // FP32 log-weights (null when w_direct is used)
    const double *w_direct;  // FP64 weights in [0, 1] (stateless entry point)
    const double *u_direct;  // per-filter uniforms (stateless entry point), else drawn from Philox
    Key key;
    const int32_t *d_t;      // completed steps; the step being resampled is *d_t + 1
    int32_t *fmax_key;       // [M] order key of each filter's maximum log-weight (atomicMax; -inf between steps)
    double *tile_sums;       // [tiles][kTsCount]
    uint64_t *tile_q;        // [tiles] exact sum of the quantised weights
    double *fstats;          // [M][kFsCount]
    uint64_t *fint;          // [M][2]: C_{N-1} and the resampling uniform U (u = U 2^-32)
    uint64_t *C;             // [P] the quantised weights q (k_weights -> k_scan_scatter)
    int32_t *B;              // [P] ancestor start markers
    int32_t *anc;            // [P] filter-local ancestors
    int32_t *tile_anc0;      // [tiles] ancestor of each tile's first output (written by the scan)
    int32_t *err;            // [2]
    double log_const;        // -dy/2 log(2 pi sigma_obs^2), added to log G only
    double ess_threshold;    // adaptive resampling: resample a filter only when ESS < this x N
    int32_t *done;           // [M] per-filter completion counters, kept at 0 between steps
};

// Extra pointers of the auxiliary particle filter's two propagations (all
// null for the bootstrap filter):
//   look-ahead (noise off): la_out[p] = log g(y | mu_p), logw[p] = lw_prev[p] + la_out[p];
//   second stage:           logw[p] = log g(y | x_p) - la_src[off_m + anc[p]].
struct AuxPtrs {
    const float *lw_prev;
    float *la_out;
    const float *la_src;
    const int32_t *anc;
    const int32_t *gather;  // lattice kernels: particle p starts from row off_m + gather[p] of x_in (the
                            // resampling's gather folded into the propagation's first load)
};

struct Ctx;

// Launchers (k_filter.cu).  All enqueue on `s` and return cudaGetLastError().
cudaError_t launch_init(const Ctx &c, cudaStream_t s);
cudaError_t launch_propagate(const Ctx &c, const float *d_obs, int32_t obs_stride, const float *x_in, float *x_out,
                             cudaStream_t s);
cudaError_t launch_resample(const Ctx &c, const float *x_in, float *x_out, cudaStream_t s);
// Bootstrap steps with the resampling's gather folded into the next
// propagation (Ctx::fold_gather): the propagation from the ancestors
// (gather null: from particle p), the resampling without the copy, and the
// copy itself for readers of the resampled state.
cudaError_t launch_propagate_fold(const Ctx &c, const float *d_obs, int32_t obs_stride, const float *x_in,
                                  float *x_out, const int32_t *gather, cudaStream_t s);
cudaError_t launch_resample_fold(const Ctx &c, const float *x, cudaStream_t s);
cudaError_t launch_materialise(const Ctx &c, const float *x_in, float *x_out, cudaStream_t s);
cudaError_t launch_refresh_max(const Ctx &c, cudaStream_t s);  // after the log-weights were replaced
// The paper's own lattice variant (k_fhn_paper.cu): n_steps Euler steps of every
// particle xi -> xo (xo null: not stored), weights into logw / fmax when non-null.
cudaError_t launch_fhnp_interval(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                 int32_t n_steps, float *logw, int32_t *fmax, AuxPtrs aux, int32_t noise,
                                 cudaStream_t s);
cudaError_t launch_fhnp_truth_step(const ModelParams &mp, Key key, int32_t record, int32_t t, const double *xi,
                                   double *xo, cudaStream_t s);
// One step of bootstrap filters that resample only when the ESS is low (k_filter.cu).
cudaError_t launch_adaptive_step(const Ctx &c, const float *d_obs, int32_t obs_stride, cudaStream_t s);
// One observation step of the ensemble of auxiliary particle filters (k_filter.cu).
cudaError_t launch_apf_step(const Ctx &c, const float *d_obs, int32_t obs_stride, cudaStream_t s);
// Learned proposal (k_filter.cu, k_proposal.cu, k_mlp.cu).
// n_steps ordinary sub-steps xi -> xo (xi == xo: in place), from the rows of
// the ancestors gather[p] when gather is non-null (a folded gather).
cudaError_t launch_fhn_substeps(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *xo,
                                const int32_t *gather, int32_t n_steps, cudaStream_t s);
// The learned-proposal step's propagation into x: its ordinary sub-steps from
// xi (through gather when non-null), then the proposal's span in place in x.
cudaError_t launch_propagate_split(const Ctx &c, const float *d_obs, int32_t stride, const float *xi, float *x,
                                   const int32_t *gather, cudaStream_t s);
cudaError_t launch_gather_tuples(const Ctx &c, const float *x_new, cudaStream_t s);
cudaError_t launch_mlp_pack(const float *theta, __nv_bfloat16 *wp, __nv_bfloat16 *w2t, cudaStream_t s);
// Network forward on the tcgen05 tensor cores fused with its input rows
// (k_proposal_tc.cu): out[(p dy + j)][4] for every particle p and observed
// node j; pfilt may be null when obs_stride is 0; err may be null.
cudaError_t launch_proposal_forward_tc(int32_t J, int32_t dx, int32_t dy, const float *x, int64_t P,
                                       const int32_t *pfilt, const int32_t *obs_idx, const float *obs,
                                       int32_t obs_stride, const __nv_bfloat16 *wp, const float *theta, float *out,
                                       int32_t *err, cudaStream_t s);
cudaError_t launch_train_forward_tc(const float *X, int64_t R, const __nv_bfloat16 *wp, const float *theta, float *out,
                                    __nv_bfloat16 *x0, float *z1, __nv_bfloat16 *a1, float *z2, __nv_bfloat16 *a2,
                                    int32_t *err, cudaStream_t s);
// The training step's backward GEMMs on the tensor cores (k_mlp_tc.cu).
cudaError_t launch_hidden_grad_tc(int64_t B, const __nv_bfloat16 *dz2, const __nv_bfloat16 *w2t, const float *z1,
                                  __nv_bfloat16 *dz1, int32_t *err, cudaStream_t s);
cudaError_t launch_weight_grad_tc(int64_t B, const __nv_bfloat16 *x0s, const __nv_bfloat16 *a1s,
                                  const __nv_bfloat16 *a2s, const __nv_bfloat16 *dz1, const __nv_bfloat16 *dz2,
                                  const float *dout, const float *row_loss, float *partial, int32_t *err,
                                  cudaStream_t s);
cudaError_t launch_systematic(int32_t M, int32_t n_tiles, const ResampleArgs &a, cudaStream_t s);
cudaError_t launch_rng_philox(int64_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                              cudaStream_t s);
cudaError_t launch_rng_normals(int64_t n, const uint32_t *ctr, uint64_t seed, float *z, cudaStream_t s);
cudaError_t launch_simulate(const ModelParams &mp, const double *d_x0, const int32_t *d_obs_idx, Key key,
                            int32_t T, int32_t record, int32_t init_random, double *d_x, float *d_y,
                            cudaStream_t s);

// Host helpers (pf_capi.cu).
int ceil_log2_host(int64_t n);
void set_global_error(const char *msg);  // text of pf_last_error(NULL) on this thread

struct Ctx {
    ModelParams mp{};
    Key key{};
    int32_t M = 0;
    int64_t P = 0;  // total particles
    int32_t n_tiles = 0;
    int32_t n_multi_tiles = 0;  // tiles of filters with more than one; the one-tile filters' tiles follow
    int32_t whole_bounds[kWholeClasses + 1] = {};  // one-tile filters of size class c: tiles [b[c], b[c+1])
    std::vector<int32_t> N;
    std::vector<int64_t> off;

    // device memory
    TileDesc *tiles = nullptr;
    TileDesc *subs = nullptr;     // sub-tiles of kSubTile particles (small models)
    TileDesc *mchunks = nullptr;  // chunks of kMeanChunk particles (lattice means)
    int32_t n_mchunks = 0;
    double *mean_part = nullptr;  // [n_mchunks][dx] FP64 partial sums (lattice)
    int32_t *mean_cnt = nullptr;  // [M][ceil(dx / 256)] chunk completion counters, zero between launches
    int32_t n_subs = 0;
    FilterDesc *filt = nullptr;
    int32_t *pfilt = nullptr;     // [P] filter of each particle (lattice kernels)
    float *x[2] = {nullptr, nullptr};
    float *logw = nullptr;
    int32_t *fmax_key = nullptr;  // [M]
    int resample_threads = kResampleThreads;
    int max_tile_len = kTile;  // the longest tile: with 4 particles per thread it needs max_tile_len / 4 threads
    int fhn_ppc = 0;               // lattice particles per CTA (0: as many as fit in 1024 threads, at most 8)
    int fhn_nodes = 0;             // lattice nodes per thread: 2, 4, 8, or 0 (4 where fhn_nodes_fit)
    int fhn_quad_ctas = 3;         // CTAs per SM the lattice build is compiled for (four nodes: 4, else 2; eight: 3, else 2; autotuned)
    // resampling only when the ESS is low (pf_set_resampling; < 0: every step)
    double ess_threshold = -1.0;
    bool adaptive() const { return ess_threshold >= 0.0 && ess_threshold <= 1.0; }
    // auxiliary particle filters (pf_set_auxiliary)
    bool aux = false;
    float *la = nullptr;           // [P] look-ahead log-likelihoods log g(y | mu)
    float *lw2 = nullptr;          // [P] second-stage log-weights
    int32_t *fmax2 = nullptr;      // [M] order keys of the second-stage maxima
    double *tile_sums = nullptr;
    uint64_t *tile_q = nullptr;
    double *fstats = nullptr;
    uint64_t *fint = nullptr;
    uint64_t *C = nullptr;
    int32_t *B = nullptr;
    int32_t *anc = nullptr;
    int32_t *tile_anc0 = nullptr; // [tiles]
    double *tile_est = nullptr;   // [tiles][dx] (small models)
    double *est = nullptr;        // [M][dx]
    double *ens = nullptr;        // [dx]
    float *d_obs = nullptr;       // [M * dy] the current observation on the device
    float *h_stage[2] = {nullptr, nullptr};        // pinned host staging, [M * dy] each
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};  // copy-out of each staging slot done
    cudaEvent_t est_ev = nullptr;    // the latest asynchronous estimate copy is done
    int32_t *h_err_async = nullptr;  // pinned copy of the error word taken with it
    bool stage_used[2] = {false, false};
    int stage_slot = 0;
    int32_t *d_t = nullptr;       // completed steps
    int32_t *err = nullptr;       // [2]
    int32_t *done = nullptr;      // [M]
    int32_t *obs_idx = nullptr;   // [dy]
    int32_t *obs_slot = nullptr;  // [J*J] lattice node -> observation index or -1
    double *x0 = nullptr;         // [dx]

    // learned proposal (lattice) and training-tuple recording
    bool prop_on = false;
    float prop_ess_frac = 0.1f;
    float *theta = nullptr;           // [PF_MLP_PARAMS] FP32
    __nv_bfloat16 *wpack = nullptr;   // packed BF16 weights (+ W2^T)
    __nv_bfloat16 *rows = nullptr;    // [P * dy][64] network inputs
    float *mlp_out = nullptr;         // [P * dy][4]
    float *xboot = nullptr;           // [P][dy][2] the transition's candidates at the observed nodes
    float *mp_obs = nullptr;          // [P][dy][2] transition means at the observed nodes
    float *logw_boot = nullptr;       // [P]
    float *lw_acc = nullptr;          // [P] log p - log q of the span's earlier sub-steps
    int32_t prop_span = 1;            // the proposal acts on the last prop_span sub-steps (pf_set_proposal_span)
    float *rec_X = nullptr, *rec_R = nullptr;  // caller's tuple buffers (recording armed when non-null)
    int64_t rec_cap = 0, rec_count = 0, rec_sel_total = 0;
    int32_t rec_stride = 1;
    int64_t *rec_sel_off = nullptr;   // [M] kept particles before each filter
    bool split_path() const { return prop_on || rec_X != nullptr; }
    // Bootstrap filters, and the learned proposal when its span leaves
    // ordinary sub-steps before it, fold the resampling's gather into the next
    // propagation (Alg. 1 step 2b's copy is never written): after such a step
    // the resampled particles are particles off_m + anc[p] of x[cur]
    // (gather_pending), and every other reader first materialises them.
    // Recording steps keep the copy (their tuples read the ancestors' rows).
    bool fold_gather() const { return !aux && !adaptive() && !rec_X && (!prop_on || mp.K > prop_span); }
    bool gather_pending = false;

    int cur = 0;  // x[cur] holds the current particles
    int32_t t = 0;
    int phase = 0;  // 0: ready to propagate; 1: propagated, ready to resample
    bool steps_done = false;
    int32_t graph_mode[2] = {-1, -1};  // obs layout (and folded-gather state) each captured graph was built for
    int32_t step_kernels = -1;         // kernel nodes of the latest captured step graph

    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    // A second stream for work of a step that is independent of the main chain
    // (the fused resampling of one-tile filters next to the tile chain of the
    // others): forked from and joined back into `stream` with the two events,
    // so a captured step graph holds both branches.
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};

    pf_alloc_fn alloc = nullptr;
    pf_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::vector<std::pair<void *, size_t>> allocations;

    int device = 0;
    int32_t fatal = 0;  // sticky pf_status
    std::string last_error;

    size_t dyn_obs() const { return (size_t)mp.dy; }
};
// Nodes per thread the lattice kernels of context c run with: 4 where the side
// allows it, unless the schedule asks for 2 or 8.
inline int fhn_nodes(const Ctx &c)
{
    if (c.fhn_nodes == 8 && fhn_nodes_fit(c.mp.J, 8)) return 8;
    return (c.fhn_nodes == 2 || !fhn_nodes_fit(c.mp.J, 4)) ? 2 : 4;
}


}  // namespace pf
