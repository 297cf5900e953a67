// pf_capi.cu -- the C ABI of include/pf.h: context life cycle, the per-step
// launch sequence (captured once per buffer parity into a CUDA graph), and
// the stateless building blocks.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pf.h"
#include "pf_internal.h"

namespace {
// A named NVTX range over one API call (a no-op unless a profiler attaches),
// so that traces show each step, propagation, resampling and estimate.
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};
}  // namespace

using namespace pf;

struct pf_ctx {
    Ctx c;
};

namespace {

std::mutex g_mu;
pf_alloc_fn g_alloc = nullptr;
pf_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;
thread_local std::string g_create_error;

pf_status fail(Ctx &c, pf_status st, const std::string &msg)
{
    c.last_error = msg;
    return st;
}

pf_status cuda_fail(Ctx &c, cudaError_t e, const char *where)
{
    c.last_error = std::string(where) + ": " + cudaGetErrorString(e);
    c.fatal = PF_ECUDA;
    return PF_ECUDA;
}

void *ctx_alloc(Ctx &c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c.alloc) {
        p = c.alloc(bytes, (void *)c.stream, c.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c.allocations.emplace_back(p, bytes);
    return p;
}

void ctx_free_all(Ctx &c)
{
    for (auto &a : c.allocations) {
        if (c.free_fn) c.free_fn(a.first, a.second, (void *)c.stream, c.alloc_user);
        else cudaFree(a.first);
    }
    c.allocations.clear();
}

template <typename T>
bool alloc_n(Ctx &c, T *&p, size_t n)
{
    p = static_cast<T *>(ctx_alloc(c, n * sizeof(T)));
    return p != nullptr;
}

// obs layout: 0 = one shared row of dy floats; 1 = M rows of dy floats.
int obs_mode(int32_t stride) { return stride == 0 ? 0 : 1; }

pf_status validate_step(Ctx &c, const float *obs, int32_t stride)
{
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (!obs) return fail(c, PF_EINVAL, "obs is NULL");
    if (stride != 0 && stride < c.mp.dy) return fail(c, PF_EINVAL, "obs_stride must be 0 or >= dy");
    return PF_OK;
}

// Copies y_t into the context's observation buffer.  Host observations go
// through one of two pinned staging slots (so the caller's buffer is free on
// return even when it is itself pinned); a slot is refilled only after its
// previous copy has completed.
cudaError_t stage_obs(Ctx &c, const float *obs, int32_t stride, cudaMemcpyKind kind)
{
    const size_t row = (size_t)c.mp.dy * sizeof(float);
    const size_t rows = stride == 0 ? 1 : (size_t)c.M;
    if (kind == cudaMemcpyDeviceToDevice) {
        if (stride == 0) return cudaMemcpyAsync(c.d_obs, obs, row, kind, c.stream);
        return cudaMemcpy2DAsync(c.d_obs, row, obs, (size_t)stride * sizeof(float), row, rows, kind, c.stream);
    }
    const int s = c.stage_slot;
    cudaError_t e = cudaSuccess;
    if (c.stage_used[s]) e = cudaEventSynchronize(c.stage_ev[s]);
    if (e != cudaSuccess) return e;
    for (size_t r = 0; r < rows; ++r)
        std::memcpy(c.h_stage[s] + r * c.mp.dy, obs + r * (size_t)(stride ? stride : 0), row);
    e = cudaMemcpyAsync(c.d_obs, c.h_stage[s], rows * row, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.stage_ev[s], c.stream);
    c.stage_used[s] = true;
    c.stage_slot ^= 1;
    return e;
}

int32_t kernel_stride(const Ctx &c, int mode) { return mode == 0 ? 0 : c.mp.dy; }

// Folded steps (Ctx::fold_gather) propagate x[cur] -> x[cur ^ 1], from the
// ancestors' rows when the previous step left its gather pending, and resample
// x[cur ^ 1] without copying it; other steps propagate x[cur] in place and
// gather into x[cur ^ 1].  Either way the step's particles end in x[cur ^ 1].
cudaError_t enqueue_propagate(Ctx &c, int mode, bool fold = false)
{
    if (c.split_path())
        return launch_propagate_split(c, c.d_obs, kernel_stride(c, mode), c.x[c.cur], c.x[fold ? c.cur ^ 1 : c.cur],
                                      fold && c.gather_pending ? c.anc : nullptr, c.stream);
    if (fold)
        return launch_propagate_fold(c, c.d_obs, kernel_stride(c, mode), c.x[c.cur], c.x[c.cur ^ 1],
                                     c.gather_pending ? c.anc : nullptr, c.stream);
    return launch_propagate(c, c.d_obs, kernel_stride(c, mode), c.x[c.cur], c.x[c.cur], c.stream);
}

cudaError_t enqueue_resample(Ctx &c, bool fold = false)
{
    const int nxt = c.cur ^ 1;
    if (fold) return launch_resample_fold(c, c.x[nxt], c.stream);
    cudaError_t e = launch_resample(c, c.x[c.cur], c.x[nxt], c.stream);
    if (e == cudaSuccess && c.rec_X && c.rec_count < c.rec_cap) {
        e = launch_gather_tuples(c, c.x[nxt], c.stream);
        c.rec_count += c.rec_sel_total * c.mp.dy;
    }
    return e;
}

cudaError_t enqueue_step(Ctx &c, int mode)
{
    if (c.aux) return launch_apf_step(c, c.d_obs, kernel_stride(c, mode), c.stream);
    if (c.adaptive()) return launch_adaptive_step(c, c.d_obs, kernel_stride(c, mode), c.stream);
    const bool fold = c.fold_gather();
    cudaError_t e = enqueue_propagate(c, mode, fold);
    if (e != cudaSuccess) return e;
    return enqueue_resample(c, fold);
}

// Writes the resampled particles of a folded step out as a state of their own
// (x[cur ^ 1] = the ancestors' rows of x[cur]) for every reader other than the
// next folded propagation.
cudaError_t materialise(Ctx &c)
{
    if (!c.gather_pending) return cudaSuccess;
    const cudaError_t e = launch_materialise(c, c.x[c.cur], c.x[c.cur ^ 1], c.stream);
    if (e != cudaSuccess) return e;
    c.cur ^= 1;
    c.gather_pending = false;
    return cudaSuccess;
}

// Per-particle weight buffers shared by the auxiliary filter and adaptive resampling.
bool ensure_weight_buffers(Ctx &c)
{
    if (c.la) return true;
    return alloc_n(c, c.la, (size_t)c.P) && alloc_n(c, c.lw2, (size_t)c.P) && alloc_n(c, c.fmax2, (size_t)c.M);
}

// Second-stage (auxiliary filter) or carried (adaptive resampling) weights back
// to uniform (lw2 = 0, and the running log sum of them = log N_m), e.g. when
// the mode is switched on or the state is replaced.
pf_status reset_aux_weights(Ctx &c)
{
    std::vector<double> fs((size_t)c.M * kFsCount);
    cudaError_t e = cudaMemsetAsync(c.lw2, 0, (size_t)c.P * sizeof(float), c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fs.data(), c.fstats, fs.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "auxiliary weights reset");
    for (int m = 0; m < c.M; ++m) fs[(size_t)m * kFsCount + kFsLse2] = std::log((double)c.N[m]);
    e = cudaMemcpy(c.fstats, fs.data(), fs.size() * sizeof(double), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "auxiliary weights reset");
}

pf_status run_step(Ctx &c, const float *obs, int32_t stride, cudaMemcpyKind kind)
{
    pf_status st = validate_step(c, obs, stride);
    if (st != PF_OK) return st;
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_step called between pf_propagate and pf_resample");
    cudaSetDevice(c.device);
    cudaError_t e = stage_obs(c, obs, stride, kind);
    if (e != cudaSuccess) return cuda_fail(c, e, "observation copy");
    const int mode = obs_mode(stride);
    const int par = c.cur;
    const bool fold = c.fold_gather();
    // a captured step depends on the observation layout and on whether the gather is folded
    // and pending from the previous step
    const int32_t key = mode | (fold ? 2 : 0) | (fold && c.gather_pending ? 4 : 0);
    if (c.rec_X) {  // recording steps carry a moving output offset: launched directly
        e = enqueue_step(c, mode);
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        c.gather_pending = false;
        c.cur ^= 1;
        c.t += 1;
        c.steps_done = true;
        return PF_OK;
    }
    if (!c.graph[par] || c.graph_mode[par] != key) {
        if (c.graph[par]) {
            cudaGraphExecDestroy(c.graph[par]);
            c.graph[par] = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture begin");
        const cudaError_t le = enqueue_step(c, mode);
        e = cudaStreamEndCapture(c.stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(c, le, "step launch (capture)");
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture end");
        size_t n_nodes = 0;
        e = cudaGraphGetNodes(g, nullptr, &n_nodes);
        if (e == cudaSuccess) {
            std::vector<cudaGraphNode_t> nodes(n_nodes);
            e = cudaGraphGetNodes(g, nodes.data(), &n_nodes);
            int32_t k = 0;
            for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
                cudaGraphNodeType ty;
                e = cudaGraphNodeGetType(nodes[i], &ty);
                if (ty == cudaGraphNodeTypeKernel) ++k;
            }
            c.step_kernels = k;
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(c, e, "graph inspection");
        }
        e = cudaGraphInstantiate(&c.graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
        c.graph_mode[par] = key;
    }
    e = cudaGraphLaunch(c.graph[par], c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c.cur ^= 1;
    c.t += 1;
    c.steps_done = true;
    c.gather_pending = fold;
    return PF_OK;
}

pf_status sync(Ctx &c, const char *where)
{
    cudaSetDevice(c.device);
    const cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return PF_OK;
}

// sync, after writing out a pending folded gather (for readers and mode switches)
pf_status sync_materialised(Ctx &c, const char *where)
{
    cudaSetDevice(c.device);
    const cudaError_t e = materialise(c);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return sync(c, where);
}

pf_status check_device_flags(Ctx &c)
{
    int32_t err[2];
    const cudaError_t e = cudaMemcpy(err, c.err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error word read");
    if (err[0] & kErrDegenerate) {
        c.fatal = PF_ENUMERIC;
        return fail(c, PF_ENUMERIC, "filter " + std::to_string(err[1]) +
                                        " had no finite positive weight (all log-weights -inf or NaN)");
    }
    if (err[0] & kErrTimeout) {
        c.fatal = PF_ETIMEOUT;
        return fail(c, PF_ETIMEOUT, "a tensor-core wait in the proposal network expired");
    }
    return PF_OK;
}

bool model_ok(const pf_model *m, std::string &why)
{
    if (!m) { why = "model is NULL"; return false; }
    if (m->steps_per_obs < 1) { why = "steps_per_obs must be >= 1"; return false; }
    switch (m->kind) {
    case PF_MODEL_LINEAR_GAUSSIAN:
        if (m->dx < 1 || m->dx > kMaxLgDim) { why = "linear-Gaussian dx must be in [1, 4]"; return false; }
        if (!m->params || m->n_params != m->dx * m->dx) { why = "linear-Gaussian params must hold dx*dx values"; return false; }
        return true;
    case PF_MODEL_LORENZ63:
        if (m->dx != 3) { why = "Lorenz 63 has dx = 3"; return false; }
        if (!m->params || m->n_params != 3) { why = "Lorenz 63 params are (s, r, b)"; return false; }
        return true;
    case PF_MODEL_FHN_LATTICE:
        if (m->J < 2 || m->J > 44 || (m->J & 1)) { why = "lattice side J must be even, 2..44"; return false; }
        if (m->dx != 2 * m->J * m->J) { why = "lattice dx must be 2 J^2"; return false; }
        if (!m->params || m->n_params != 9) { why = "lattice params are (a, b, c1, c2, d, D, amp, steps, block)"; return false; }
        return true;
    case PF_MODEL_FHN_PAPER:
        if (m->J < 2 || m->J > 44 || (m->J & 1)) { why = "lattice side J must be even, 2..44"; return false; }
        if (m->dx != 3 * m->J * m->J) { why = "the paper's lattice has dx = 3 J^2 (U, V, stimulus counters)"; return false; }
        if (!m->params || m->n_params != 17) { why = "the paper's lattice takes 17 params (see pf.h)"; return false; }
        if (!(m->params[9] >= 1.0) || !(m->params[16] >= 1.0)) { why = "forcing period and l0 must be >= 1"; return false; }
        return true;
    default:
        why = "unknown model kind";
        return false;
    }
}

bool fill_params(const pf_model *model, double dt, const pf_obs_op *obs, const pf_noise *noise, ModelParams &mp,
                 std::string &why)
{
    if (!model_ok(model, why)) return false;
    if (!(dt > 0.0) || !std::isfinite(dt)) { why = "dt must be positive"; return false; }
    if (!obs || obs->dy < 1 || obs->dy > 4096 || !obs->idx) { why = "obs op needs 1 <= dy <= 4096 and idx"; return false; }
    if (!(obs->sigma_obs > 0.0)) { why = "sigma_obs must be positive"; return false; }
    if (!noise || !noise->x0_mean) { why = "noise needs x0_mean"; return false; }
    if (!(noise->sigma_dyn >= 0.0) || !(noise->sigma0 >= 0.0)) { why = "noise scales must be >= 0"; return false; }
    if (!is_lattice(model->kind) && obs->dy > kMaxObsSmall) { why = "small models observe at most 8 components"; return false; }
    for (int j = 0; j < obs->dy; ++j) {
        const int32_t i = obs->idx[j];
        const int32_t lim = is_lattice(model->kind) ? model->J * model->J : model->dx;
        if (i < 0 || i >= lim) { why = "observation index out of range (lattice: v-plane nodes only)"; return false; }
    }
    mp = ModelParams{};
    mp.kind = model->kind;
    mp.dx = model->dx;
    mp.J = model->J;
    mp.K = model->steps_per_obs;
    mp.dt = dt;
    mp.sigma_dyn = noise->sigma_dyn;
    mp.sigma0 = noise->sigma0;
    mp.sigma_obs = obs->sigma_obs;
    for (int i = 0; i < model->n_params && i < 24; ++i) mp.p[i] = model->params[i];
    mp.dy = obs->dy;
    for (int j = 0; j < obs->dy && j < kMaxObsSmall; ++j) mp.obs_small[j] = obs->idx[j];
    if (!is_lattice(model->kind))
        for (int v = 0; v < model->dx; ++v) mp.x0_small[v] = noise->x0_mean[v];
    for (int i = 0; i < 24; ++i) {
        mp.fp[i] = (float)mp.p[i];
        mp.ip[i] = (std::isfinite(mp.p[i]) && std::fabs(mp.p[i]) < 9.0e18) ? (int64_t)mp.p[i] : 0;
    }
    mp.fdt = (float)dt;
    mp.dsq = noise->sigma_dyn * std::sqrt(dt);
    mp.fsq = (float)mp.dsq;
    mp.dhalf_prec = -0.5 / (obs->sigma_obs * obs->sigma_obs);
    mp.fhalf_prec = (float)mp.dhalf_prec;
    return true;
}

// Tiles of at most kTile particles, never spanning two filters; sub-tiles of
// at most kSubTile particles inside them.  Per-filter partial maxima come from
// the sub-tiles (small models) or the tiles (lattice, stateless resampling).
// With `bounds` (kWholeClasses + 1 entries), the tiles of filters with more
// than one tile come first (in filter order), then the single tiles of the
// other filters grouped by size class c (N <= 32 * kWholeItems << c), and
// bounds[c] .. bounds[c + 1] are class c's tiles (bounds[0]: the count of the
// former); a filter's tiles are always consecutive.
int whole_class(int32_t n)
{
    int c = 0;
    while (c + 1 < kWholeClasses && n > (32 * kWholeItems << c)) ++c;
    return c;
}

void make_tiles(const std::vector<int32_t> &N, std::vector<TileDesc> &tiles, std::vector<FilterDesc> &filt,
                std::vector<int64_t> &off, std::vector<TileDesc> *subs = nullptr,
                std::vector<TileDesc> *mchunks = nullptr, int32_t *bounds = nullptr)
{
    const int32_t M = (int32_t)N.size();
    off.assign(M + 1, 0);
    for (int m = 0; m < M; ++m) off[m + 1] = off[m] + N[m];
    tiles.clear();
    filt.assign(M, FilterDesc{});
    for (int pass = 0; pass < (bounds ? 1 + kWholeClasses : 1); ++pass) {
        if (pass > 0) bounds[pass - 1] = (int32_t)tiles.size();
        for (int m = 0; m < M; ++m) {
            if (bounds && (pass == 0 ? N[m] <= kTile : (N[m] > kTile || whole_class(N[m]) != pass - 1))) continue;
            FilterDesc &fd = filt[m];
            fd.tile_begin = (int32_t)tiles.size();
            for (int32_t s = 0; s < N[m]; s += kTile) {
                TileDesc td{};
                td.m = m;
                td.lstart = s;
                td.len = std::min(kTile, N[m] - s);
                td.gstart = off[m] + s;
                tiles.push_back(td);
            }
            fd.tile_count = (int32_t)tiles.size() - fd.tile_begin;
        }
    }
    if (bounds) bounds[kWholeClasses] = (int32_t)tiles.size();
    for (int m = 0; m < M; ++m) {
        FilterDesc &fd = filt[m];
        fd.off = off[m];
        fd.N = N[m];
        fd.shift = 52 - ceil_log2_host(N[m]);
        for (int32_t i = fd.tile_begin; i < fd.tile_begin + fd.tile_count; ++i) {
            TileDesc &td = tiles[i];
            td.N = fd.N;
            td.tile_begin = fd.tile_begin;
            td.tile_count = fd.tile_count;
            td.shift = fd.shift;
        }
        if (mchunks) {
            fd.mc_begin = (int32_t)mchunks->size();
            for (int32_t s = 0; s < N[m]; s += kMeanChunk) {
                TileDesc mc{};
                mc.m = m;
                mc.lstart = s;
                mc.len = std::min(kMeanChunk, N[m] - s);
                mc.gstart = off[m] + s;
                mchunks->push_back(mc);
            }
            fd.mc_count = (int32_t)mchunks->size() - fd.mc_begin;
        }
        if (subs) {
            for (int32_t s = 0; s < N[m]; s += kSubTile) {
                TileDesc st{};
                st.m = m;
                st.lstart = s;
                st.len = std::min(kSubTile, N[m] - s);
                st.gstart = off[m] + s;
                subs->push_back(st);
            }
        }
    }
}

}  // namespace

namespace pf {
void set_global_error(const char *msg) { g_create_error = msg; }

int ceil_log2_host(int64_t n)
{
    int L = 0;
    while (((int64_t)1 << L) < n) ++L;
    return L;
}
}  // namespace pf

// Schedules chosen by pf_autotune, per (model, J, K, dx, particles, filters).
static std::mutex g_tune_mu;
// keyed by model kind, lattice side, K, dx, total particles, filters and a
// hash (FNV-1a) of the particle counts, so ragged batches of the same total
// are told apart
static std::map<std::tuple<int, int, int, int, int64_t, int32_t, uint64_t>, std::tuple<int, int, int, int>> g_tune_cache;

static uint64_t counts_hash(const std::vector<int32_t> &N)
{
    uint64_t h = 1469598103934665603ull;
    for (int32_t n : N) {
        h ^= (uint32_t)n;
        h *= 1099511628211ull;
    }
    return h;
}

// Median time of `reps` launches of fn on the context's stream (ms).
template <typename F>
static float time_ms(Ctx &c, int reps, F fn)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> ts;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, c.stream);
        fn();
        cudaEventRecord(b, c.stream);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        ts.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

extern "C" {

const char *pf_version(void) { return "paper_1407_8071_gb300 0.1 (sm_103a)"; }

pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return PF_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return PF_OK;
}

// The context's own streams and fork / join events (null handles are skipped).
static void destroy_streams(Ctx &c)
{
    if (c.fork_ev) cudaEventDestroy(c.fork_ev);
    if (c.join_ev) cudaEventDestroy(c.join_ev);
    if (c.side_stream) cudaStreamDestroy(c.side_stream);
    if (c.own_stream) cudaStreamDestroy(c.own_stream);
    c.fork_ev = c.join_ev = nullptr;
    c.side_stream = c.own_stream = nullptr;
}

pf_status pf_create(const pf_model *model, int32_t M, const int32_t *N, double dt, const pf_obs_op *obs,
                    const pf_noise *noise, pf_ctx **out)
{
    if (!out) return PF_EINVAL;
    *out = nullptr;
    std::string why;
    ModelParams mp;
    if (!fill_params(model, dt, obs, noise, mp, why)) {
        g_create_error = why;
        return PF_EINVAL;
    }
    if (M < 1 || !N) {
        g_create_error = "M must be >= 1 and N non-NULL";
        return PF_EINVAL;
    }
    for (int m = 0; m < M; ++m)
        if (N[m] < 1 || N[m] > (1 << 24)) {
            g_create_error = "every N[m] must be in [1, 2^24]";
            return PF_EINVAL;
        }
    pf_ctx *h = new (std::nothrow) pf_ctx();
    if (!h) return PF_ENOMEM;
    Ctx &c = h->c;
    c.mp = mp;
    c.key = make_key(noise->seed);
    c.M = M;
    c.N.assign(N, N + M);
    cudaGetDevice(&c.device);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        c.alloc = g_alloc;
        c.free_fn = g_free;
        c.alloc_user = g_alloc_user;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&c.own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_create_error = std::string("stream create: ") + cudaGetErrorString(e);
        destroy_streams(c);
        delete h;
        return PF_ECUDA;
    }
    c.stream = c.own_stream;

    std::vector<TileDesc> tiles, subs, mchunks;
    std::vector<FilterDesc> filt;
    const bool small = !is_lattice(mp.kind);
    make_tiles(c.N, tiles, filt, c.off, small ? &subs : nullptr, small ? nullptr : &mchunks, c.whole_bounds);
    c.n_multi_tiles = c.whole_bounds[0];
    c.P = c.off[M];
    c.n_tiles = (int32_t)tiles.size();
    c.n_subs = (int32_t)subs.size();
    c.n_mchunks = (int32_t)mchunks.size();
    {
        int max_len = 1;
        for (const TileDesc &td : tiles) max_len = std::max(max_len, td.len);
        // threads per tile CTA: whole warps, 64..256, enough for 8 particles each (the tile
        // kernels take 4 per thread where that covers the longest tile)
        int th = 64;
        while (th < kResampleThreads && th * 2 * kItems < max_len) th *= 2;
        c.resample_threads = th;
        c.max_tile_len = max_len;
    }
    const int dx = mp.dx;
    const int64_t P = c.P;
    bool ok = alloc_n(c, c.tiles, tiles.size()) && alloc_n(c, c.filt, filt.size()) &&
              alloc_n(c, c.done, (size_t)M) && alloc_n(c, c.fmax_key, (size_t)M) &&
              (!small || alloc_n(c, c.subs, subs.size())) &&
              alloc_n(c, c.x[0], (size_t)P * dx) && alloc_n(c, c.x[1], (size_t)P * dx) && alloc_n(c, c.logw, P) &&
              alloc_n(c, c.tile_sums, (size_t)c.n_tiles * kTsCount) &&
              alloc_n(c, c.tile_q, c.n_tiles) && alloc_n(c, c.fint, (size_t)M * 2) &&
              alloc_n(c, c.fstats, (size_t)M * kFsCount) && alloc_n(c, c.C, P) && alloc_n(c, c.B, P) &&
              alloc_n(c, c.anc, P) && alloc_n(c, c.tile_anc0, (size_t)c.n_tiles) &&
              alloc_n(c, c.est, (size_t)M * dx) && alloc_n(c, c.ens, dx) &&
              alloc_n(c, c.d_obs, (size_t)M * mp.dy) && alloc_n(c, c.d_t, 1) && alloc_n(c, c.err, 2) &&
              alloc_n(c, c.obs_idx, mp.dy) && alloc_n(c, c.x0, dx);
    if (ok) ok = alloc_n(c, c.pfilt, P);
    if (ok && is_lattice(mp.kind))
        ok = alloc_n(c, c.obs_slot, mp.J * mp.J) && alloc_n(c, c.mchunks, mchunks.size()) &&
             alloc_n(c, c.mean_part, mchunks.size() * (size_t)dx) &&
             alloc_n(c, c.mean_cnt, (size_t)M * ((dx + 255) / 256));
    else if (ok) ok = alloc_n(c, c.tile_est, (size_t)c.n_tiles * dx);
    if (!ok) {
        g_create_error = "device allocation failed";
        ctx_free_all(c);
        destroy_streams(c);
        delete h;
        return PF_ENOMEM;
    }
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaMallocHost(&c.h_stage[k], (size_t)M * mp.dy * sizeof(float)) == cudaSuccess &&
             cudaEventCreateWithFlags(&c.stage_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        g_create_error = "pinned staging allocation failed";
        for (int k = 0; k < 2; ++k) {
            if (c.h_stage[k]) cudaFreeHost(c.h_stage[k]);
            if (c.stage_ev[k]) cudaEventDestroy(c.stage_ev[k]);
        }
        ctx_free_all(c);
        destroy_streams(c);
        delete h;
        return PF_ENOMEM;
    }
    std::vector<int32_t> pf_host;
    std::vector<int32_t> slot;
    const int32_t zero = 0, err_init[2] = {0, -1};
    e = cudaMemcpyAsync(c.tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.filt, filt.data(), filt.size() * sizeof(FilterDesc), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.obs_idx, obs->idx, mp.dy * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.x0, noise->x0_mean, dx * sizeof(double), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_t, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.fstats, 0, (size_t)M * kFsCount * sizeof(double), c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.done, 0, (size_t)M * sizeof(int32_t), c.stream);
    std::vector<int32_t> neg_inf((size_t)M, kNegInfKey);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.fmax_key, neg_inf.data(), (size_t)M * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess && small)
        e = cudaMemcpyAsync(c.subs, subs.data(), subs.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) {
        pf_host.resize(P);
        for (int m = 0; m < M; ++m) std::fill(pf_host.begin() + c.off[m], pf_host.begin() + c.off[m + 1], m);
        e = cudaMemcpyAsync(c.pfilt, pf_host.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
    }
    if (e == cudaSuccess && is_lattice(mp.kind)) {
        slot.assign(mp.J * mp.J, -1);
        for (int j = 0; j < mp.dy; ++j) slot[obs->idx[j]] = j;
        e = cudaMemcpyAsync(c.obs_slot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.mchunks, mchunks.data(), mchunks.size() * sizeof(TileDesc), cudaMemcpyHostToDevice,
                                c.stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c.mean_cnt, 0, (size_t)M * ((dx + 255) / 256) * sizeof(int32_t), c.stream);
    }
    if (e == cudaSuccess) e = launch_init(c, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);  // host staging vectors go out of scope
    if (e != cudaSuccess) {
        g_create_error = std::string("create: ") + cudaGetErrorString(e);
        for (int k = 0; k < 2; ++k) {
            cudaFreeHost(c.h_stage[k]);
            cudaEventDestroy(c.stage_ev[k]);
        }
        ctx_free_all(c);
        destroy_streams(c);
        delete h;
        return PF_ECUDA;
    }
    *out = h;
    return PF_OK;
}

void pf_destroy(pf_ctx *h)
{
    if (!h) return;
    Ctx &c = h->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    for (auto &g : c.graph)
        if (g) cudaGraphExecDestroy(g);
    for (int k = 0; k < 2; ++k) {
        if (c.h_stage[k]) cudaFreeHost(c.h_stage[k]);
        if (c.stage_ev[k]) cudaEventDestroy(c.stage_ev[k]);
    }
    if (c.h_err_async) cudaFreeHost(c.h_err_async);
    if (c.est_ev) cudaEventDestroy(c.est_ev);
    ctx_free_all(c);
    destroy_streams(c);
    delete h;
}

const char *pf_last_error(const pf_ctx *h)
{
    if (!h) return g_create_error.c_str();
    return h->c.last_error.c_str();
}

pf_status pf_set_stream(pf_ctx *h, void *stream)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    cudaStream_t s = stream ? (cudaStream_t)stream : c.own_stream;
    if (s != c.stream) {
        cudaStreamSynchronize(c.stream);
        c.stream = s;
    }
    return PF_OK;
}

pf_status pf_step(pf_ctx *h, const float *h_obs, int32_t obs_stride)
{
    Trace trace("pf_step");
    if (!h) return PF_EINVAL;
    return run_step(h->c, h_obs, obs_stride, cudaMemcpyHostToDevice);
}

pf_status pf_step_device(pf_ctx *h, const float *d_obs, int32_t obs_stride)
{
    Trace trace("pf_step_device");
    if (!h) return PF_EINVAL;
    return run_step(h->c, d_obs, obs_stride, cudaMemcpyDeviceToDevice);
}

pf_status pf_step_timed(pf_ctx *h, const float *d_obs, int32_t obs_stride, float *h_ms)
{
    Trace trace("pf_step_timed");
    if (!h || !h_ms) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = validate_step(c, d_obs, obs_stride);
    if (st != PF_OK) return st;
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_step_timed between pf_propagate and pf_resample");
    if (c.aux || c.adaptive() || c.rec_X) return fail(c, PF_EUNSUPPORTED, "timed steps are for the bootstrap filter");
    cudaSetDevice(c.device);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    const int mode = obs_mode(obs_stride);
    const bool fold = c.fold_gather();
    if (e == cudaSuccess) e = stage_obs(c, d_obs, obs_stride, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], c.stream);
    if (e == cudaSuccess) e = enqueue_propagate(c, mode, fold);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c.stream);
    if (e == cudaSuccess) e = enqueue_resample(c, fold);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&h_ms[0], ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&h_ms[1], ev[1], ev[2]);
    for (int i = 0; i < 3; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(c, e, "timed step");
    c.cur ^= 1;
    c.t += 1;
    c.steps_done = true;
    c.gather_pending = fold;
    return PF_OK;
}

static pf_status propagate_impl(pf_ctx *h, const float *obs, int32_t obs_stride, cudaMemcpyKind kind)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = validate_step(c, obs, obs_stride);
    if (st != PF_OK) return st;
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_propagate called twice without pf_resample");
    if (c.aux) return fail(c, PF_EUNSUPPORTED, "the auxiliary filter steps as a whole: use pf_step");
    if (c.adaptive()) return fail(c, PF_EUNSUPPORTED, "adaptive resampling steps as a whole: use pf_step");
    cudaSetDevice(c.device);
    cudaError_t e = materialise(c);  // the two halves take the unfolded path
    if (e == cudaSuccess) e = stage_obs(c, obs, obs_stride, kind);
    if (e == cudaSuccess) e = enqueue_propagate(c, obs_mode(obs_stride));
    if (e != cudaSuccess) return cuda_fail(c, e, "propagate");
    c.phase = 1;
    return PF_OK;
}

pf_status pf_propagate(pf_ctx *h, const float *h_obs, int32_t obs_stride)
{
    Trace trace("pf_propagate");
    return propagate_impl(h, h_obs, obs_stride, cudaMemcpyHostToDevice);
}

pf_status pf_propagate_device(pf_ctx *h, const float *d_obs, int32_t obs_stride)
{
    Trace trace("pf_propagate_device");
    return propagate_impl(h, d_obs, obs_stride, cudaMemcpyDeviceToDevice);
}

pf_status pf_resample(pf_ctx *h)
{
    Trace trace("pf_resample");
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 1) return fail(c, PF_ESTATE, "pf_resample needs a preceding pf_propagate");
    cudaSetDevice(c.device);
    const cudaError_t e = enqueue_resample(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "resample");
    c.cur ^= 1;
    c.t += 1;
    c.phase = 0;
    c.steps_done = true;
    return PF_OK;
}

pf_status pf_estimate(pf_ctx *h, const pf_stat *stat, double *out)
{
    Trace trace("pf_estimate");
    if (!h || !stat || !out) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal == PF_ECUDA) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (!c.steps_done) return fail(c, PF_ESTATE, "no step has completed");
    pf_status st = sync(c, "estimate");
    if (st != PF_OK) return st;
    st = check_device_flags(c);
    if (st != PF_OK) return st;
    const int dx = c.mp.dx, M = c.M;
    cudaError_t e = cudaSuccess;
    if (stat->kind == PF_STAT_MEAN) {
        if (stat->var < -1 || stat->var >= dx) return fail(c, PF_EINVAL, "var out of range");
        if (stat->per_filter) {
            std::vector<double> est((size_t)M * dx);
            e = cudaMemcpy(est.data(), c.est, est.size() * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(c, e, "estimate copy");
            if (stat->var < 0) std::memcpy(out, est.data(), est.size() * sizeof(double));
            else for (int m = 0; m < M; ++m) out[m] = est[(size_t)m * dx + stat->var];
        } else if (stat->var < 0) {
            e = cudaMemcpy(out, c.ens, dx * sizeof(double), cudaMemcpyDeviceToHost);
        } else {
            e = cudaMemcpy(out, c.ens + stat->var, sizeof(double), cudaMemcpyDeviceToHost);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "estimate copy");
        return PF_OK;
    }
    int slot;
    switch (stat->kind) {
    case PF_STAT_LOG_EVIDENCE: slot = kFsLogG; break;
    case PF_STAT_ESS: slot = kFsEss; break;
    case PF_STAT_LOG_Z: slot = kFsLogZ; break;
    case PF_STAT_FALLBACK: slot = kFsFallback; break;
    default: return fail(c, PF_EINVAL, "unknown statistic");
    }
    std::vector<double> fs((size_t)M * kFsCount);
    e = cudaMemcpy(fs.data(), c.fstats, fs.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "statistic copy");
    if (stat->per_filter) {
        for (int m = 0; m < M; ++m) out[m] = fs[(size_t)m * kFsCount + slot];
    } else {
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += fs[(size_t)m * kFsCount + slot];
        out[0] = s / M;
    }
    return PF_OK;
}

pf_status pf_step_kernels(pf_ctx *h, int32_t *n)
{
    if (!h || !n) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.step_kernels < 0) return fail(c, PF_ESTATE, "no step graph has been captured");
    *n = c.step_kernels;
    return PF_OK;
}

pf_status pf_estimate_async(pf_ctx *h, const pf_stat *stat, double *h_out)
{
    Trace trace("pf_estimate_async");
    if (!h || !stat || !h_out) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal == PF_ECUDA) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (!c.steps_done) return fail(c, PF_ESTATE, "no step has completed");
    cudaSetDevice(c.device);
    const int dx = c.mp.dx, M = c.M;
    cudaError_t e = cudaSuccess;
    if (!c.est_ev) {
        e = cudaEventCreateWithFlags(&c.est_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&c.h_err_async, 2 * sizeof(int32_t));
        if (e != cudaSuccess) return cuda_fail(c, e, "asynchronous estimate setup");
    }
    if (stat->kind == PF_STAT_MEAN) {
        if (stat->var < -1 || stat->var >= dx) return fail(c, PF_EINVAL, "var out of range");
        if (stat->per_filter && stat->var < 0)
            e = cudaMemcpyAsync(h_out, c.est, (size_t)M * dx * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
        else if (stat->per_filter)
            e = cudaMemcpy2DAsync(h_out, sizeof(double), c.est + stat->var, (size_t)dx * sizeof(double), sizeof(double),
                                  (size_t)M, cudaMemcpyDeviceToHost, c.stream);
        else if (stat->var < 0)
            e = cudaMemcpyAsync(h_out, c.ens, (size_t)dx * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
        else
            e = cudaMemcpyAsync(h_out, c.ens + stat->var, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    } else {
        if (!stat->per_filter) return fail(c, PF_EUNSUPPORTED, "asynchronous statistics other than MEAN are per filter");
        int slot;
        switch (stat->kind) {
        case PF_STAT_LOG_EVIDENCE: slot = kFsLogG; break;
        case PF_STAT_ESS: slot = kFsEss; break;
        case PF_STAT_LOG_Z: slot = kFsLogZ; break;
        case PF_STAT_FALLBACK: slot = kFsFallback; break;
        default: return fail(c, PF_EINVAL, "unknown statistic");
        }
        e = cudaMemcpy2DAsync(h_out, sizeof(double), c.fstats + slot, (size_t)kFsCount * sizeof(double),
                              sizeof(double), (size_t)M, cudaMemcpyDeviceToHost, c.stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.h_err_async, c.err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.est_ev, c.stream);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "asynchronous estimate copy");
}

pf_status pf_estimate_wait(pf_ctx *h)
{
    Trace trace("pf_estimate_wait");
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (!c.est_ev) return fail(c, PF_ESTATE, "no asynchronous estimate was enqueued");
    cudaSetDevice(c.device);
    const cudaError_t e = cudaEventSynchronize(c.est_ev);
    if (e != cudaSuccess) return cuda_fail(c, e, "asynchronous estimate wait");
    const int32_t err0 = c.h_err_async[0], err1 = c.h_err_async[1];
    if (err0 & kErrDegenerate) {
        c.fatal = PF_ENUMERIC;
        return fail(c, PF_ENUMERIC, "filter " + std::to_string(err1) +
                                        " had no finite positive weight (all log-weights -inf or NaN)");
    }
    if (err0 & kErrTimeout) {
        c.fatal = PF_ETIMEOUT;
        return fail(c, PF_ETIMEOUT, "a tensor-core wait in the proposal network expired");
    }
    return PF_OK;
}

pf_status pf_inject_error(pf_ctx *h, int32_t code, int32_t filter)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (code != PF_ETIMEOUT && code != PF_ENUMERIC) return fail(c, PF_EINVAL, "only PF_ETIMEOUT and PF_ENUMERIC are injected");
    if (filter < 0 || filter >= c.M) return fail(c, PF_EINVAL, "filter out of range");
    cudaSetDevice(c.device);
    // The words the device would have written: the flag of the failed wait or of
    // the degenerate normaliser, and the filter it names.  Enqueued behind the
    // work already on the stream, so the next check sees them like a real failure.
    const int32_t word[2] = {code == PF_ETIMEOUT ? kErrTimeout : kErrDegenerate, filter};
    cudaError_t e = cudaMemcpyAsync(c.err, word, sizeof(word), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "error injection");
}

static void drop_graphs(Ctx &c)
{
    for (int k = 0; k < 2; ++k) {
        if (c.graph[k]) cudaGraphExecDestroy(c.graph[k]);
        c.graph[k] = nullptr;
        c.graph_mode[k] = -1;
    }
}

// Buffers shared by the learned proposal and the tuple recording.
static pf_status ensure_proposal_buffers(Ctx &c)
{
    if (c.rows) return PF_OK;
    const size_t R = (size_t)c.P * c.mp.dy;
    const bool ok = alloc_n(c, c.theta, (size_t)PF_MLP_PARAMS) &&
                    alloc_n(c, c.wpack, (size_t)(128 * 64 + 128 * 128 + 8 * 128) + 128 * 128) &&
                    alloc_n(c, c.rows, R * 64) && alloc_n(c, c.mlp_out, R * 4) && alloc_n(c, c.xboot, R * 2) &&
                    alloc_n(c, c.mp_obs, R * 2) && alloc_n(c, c.logw_boot, (size_t)c.P) &&
                    alloc_n(c, c.lw_acc, (size_t)c.P) &&
                    alloc_n(c, c.rec_sel_off, (size_t)c.M);
    return ok ? PF_OK : fail(c, PF_ENOMEM, "proposal buffers: device allocation failed");
}

pf_status pf_set_proposal(pf_ctx *h, const float *h_theta, int32_t n_params, double ess_frac)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_set_proposal between pf_propagate and pf_resample");
    if (c.mp.kind != PF_MODEL_FHN_LATTICE) return fail(c, PF_EUNSUPPORTED, "the learned proposal is for the lattice");
    if ((c.aux || c.adaptive()) && h_theta)
        return fail(c, PF_EUNSUPPORTED, "the learned proposal is not combined with the auxiliary filter or adaptive resampling");
    if (h_theta && (n_params != PF_MLP_PARAMS || !(ess_frac >= 0.0 && ess_frac <= 1.0)))
        return fail(c, PF_EINVAL, "n_params must be PF_MLP_PARAMS and ess_frac in [0, 1]");
    pf_status st = sync_materialised(c, "set_proposal");
    if (st != PF_OK) return st;
    drop_graphs(c);
    if (!h_theta) {
        c.prop_on = false;
        return PF_OK;
    }
    st = ensure_proposal_buffers(c);
    if (st != PF_OK) return st;
    cudaError_t e = cudaMemcpy(c.theta, h_theta, PF_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_mlp_pack(c.theta, c.wpack, c.wpack + (128 * 64 + 128 * 128 + 8 * 128), c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_proposal");
    c.prop_on = true;
    c.prop_ess_frac = (float)ess_frac;
    return PF_OK;
}

pf_status pf_set_proposal_span(pf_ctx *h, int32_t span)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_set_proposal_span between pf_propagate and pf_resample");
    if (c.mp.kind != PF_MODEL_FHN_LATTICE) return fail(c, PF_EUNSUPPORTED, "the learned proposal is for the lattice");
    if (span < 1 || span > c.mp.K) return fail(c, PF_EINVAL, "span must be in [1, steps_per_obs]");
    if (span > 1 && c.mp.J % 4 != 0) return fail(c, PF_EUNSUPPORTED, "a span above one needs J divisible by 4");
    pf_status st = sync_materialised(c, "set_proposal_span");
    if (st != PF_OK) return st;
    drop_graphs(c);
    c.prop_span = span;
    return PF_OK;
}

pf_status pf_record_tuples(pf_ctx *h, float *d_X, float *d_R, int64_t capacity, int32_t stride)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.mp.kind != PF_MODEL_FHN_LATTICE) return fail(c, PF_EUNSUPPORTED, "tuple recording is for the lattice");
    if ((c.aux || c.adaptive()) && d_X) return fail(c, PF_EUNSUPPORTED, "tuple recording is for the bootstrap filter");
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_record_tuples between pf_propagate and pf_resample");
    pf_status st = sync_materialised(c, "record_tuples");
    if (st != PF_OK) return st;
    drop_graphs(c);
    if (!d_X) {
        c.rec_X = c.rec_R = nullptr;
        return PF_OK;
    }
    if (!d_R || capacity < 1 || stride < 1) return fail(c, PF_EINVAL, "d_R, capacity >= 1 and stride >= 1 needed");
    st = ensure_proposal_buffers(c);
    if (st != PF_OK) return st;
    std::vector<int64_t> sel(c.M);
    int64_t acc = 0;
    for (int m = 0; m < c.M; ++m) {
        sel[m] = acc;
        acc += (c.N[m] + stride - 1) / stride;
    }
    const cudaError_t e = cudaMemcpy(c.rec_sel_off, sel.data(), c.M * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "record_tuples");
    c.rec_X = d_X;
    c.rec_R = d_R;
    c.rec_cap = capacity;
    c.rec_count = 0;
    c.rec_stride = stride;
    c.rec_sel_total = acc;
    return PF_OK;
}

pf_status pf_recorded_tuples(const pf_ctx *h, int64_t *count)
{
    if (!h || !count) return PF_EINVAL;
    *count = std::min(h->c.rec_count, h->c.rec_cap);
    return PF_OK;
}

pf_status pf_autotune(pf_ctx *h, int32_t *h_choice)
{
    Trace trace("pf_autotune");
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0 || c.rec_X) return fail(c, PF_ESTATE, "pf_autotune needs a context between steps, not recording");
    pf_status st = sync_materialised(c, "autotune");
    if (st != PF_OK) return st;
    const auto key = std::make_tuple((int)c.mp.kind, (int)c.mp.J, (int)c.mp.K, (int)c.mp.dx, (int64_t)c.P, c.M,
                                     counts_hash(c.N));
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c.fhn_ppc = std::get<0>(it->second);
            c.resample_threads = std::get<1>(it->second);
            c.fhn_nodes = std::get<2>(it->second);
            c.fhn_quad_ctas = std::get<3>(it->second);
            cached = true;
        }
    }
    if (!cached) {
        // Trials run on copies: the current particles are copied into the other
        // buffer and propagated there; resampling writes into a temporary
        // buffer.  Everything a caller can read afterwards -- log-weights,
        // ancestors, per-filter scalars, estimates, the step counter -- is saved
        // before and restored after.
        const size_t P = (size_t)c.P, dx = (size_t)c.mp.dx, M = (size_t)c.M;
        const size_t xb = P * dx * sizeof(float);
        const size_t save_bytes = P * 4 + P * 4 + M * kFsCount * 8 + M * dx * 8 + dx * 8 + M * 4 + M * 16 + 8;
        char *tmp = nullptr, *save = nullptr;
        cudaError_t e = cudaMalloc(&tmp, xb);
        if (e == cudaSuccess) e = cudaMalloc(&save, save_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (tmp) cudaFree(tmp);
            return fail(c, PF_ENOMEM, "autotune: no room for its trial buffers");
        }
        struct Span { void *dev; size_t bytes; };
        const Span spans[] = {{c.logw, P * 4}, {c.anc, P * 4}, {c.fstats, M * kFsCount * 8}, {c.est, M * dx * 8},
                              {c.ens, dx * 8}, {c.fmax_key, M * 4}, {c.fint, M * 16}, {c.err, 8}};
        size_t o = 0;
        for (const Span &sp : spans) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(save + o, sp.dev, sp.bytes, cudaMemcpyDeviceToDevice, c.stream);
            o += sp.bytes;
        }
        float *scratch = c.x[c.cur ^ 1];
        float *dest = reinterpret_cast<float *>(tmp);
        std::vector<float> zeros(M * c.mp.dy, 0.0f);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_obs, zeros.data(), zeros.size() * 4, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        int best_ppc = c.fhn_ppc, best_rt = c.resample_threads, best_nodes = c.fhn_nodes, best_qc = c.fhn_quad_ctas;
        auto trial_step = [&] {
            cudaMemcpyAsync(scratch, c.x[c.cur], xb, cudaMemcpyDeviceToDevice, c.stream);
            launch_propagate(c, c.d_obs, 0, scratch, scratch, c.stream);
        };
        if (e == cudaSuccess && is_lattice(c.mp.kind)) {  // nodes per thread, particles per CTA
            float best = 1e30f;
            for (int nodes = 2; nodes <= 8; nodes *= 2) {
                const int cap4 = c.mp.kind == kFhnPaper ? kFhnp4MaxThreads : fhn4_max_threads(nodes);
                if (nodes > 2 && (c.mp.J % nodes != 0 || c.mp.J * c.mp.J / nodes > cap4)) continue;
                const int per = c.mp.J * c.mp.J / nodes, cap = nodes >= 4 ? cap4 : 1024;
                int maxp = 1;
                while ((maxp + 1) * per <= cap && maxp < 8) ++maxp;
                // the builds' CTAs per SM: four nodes 2 or 4, eight 2 or 3 (two nodes: one build)
                const int qcs[2] = {nodes == 2 ? 3 : 2, nodes == 4 ? 4 : 3}, n_qc = nodes == 2 ? 1 : 2;
                for (int ppc = 1; ppc <= maxp; ++ppc)
                    for (int iq = 0; iq < n_qc; ++iq) {
                        const int qc = qcs[iq];
                        c.fhn_nodes = nodes;
                        c.fhn_ppc = ppc;
                        c.fhn_quad_ctas = qc;
                        const float ms = time_ms(c, 3, trial_step);
                        if (ms < best) { best = ms; best_ppc = ppc; best_nodes = nodes; best_qc = qc; }
                    }
            }
            c.fhn_ppc = best_ppc;
            c.fhn_nodes = best_nodes;
            c.fhn_quad_ctas = best_qc;
        }
        if (e == cudaSuccess) {  // threads per resampling tile CTA
            int max_len = 1;
            for (int32_t n : c.N) max_len = std::max(max_len, std::min(n, kTile));
            std::vector<int> cands;
            for (int th = 64; th <= kResampleThreads; th *= 2)
                if (th * 2 * kItems >= max_len) cands.push_back(th);
            // the form the steps take (folded: the means read from the
            // propagated rows, nothing copied), two interleaved rounds, the
            // better median of five per candidate
            const bool fold = c.fold_gather();
            std::vector<float> best_ms(cands.size(), 1e30f);
            for (int round = 0; round < 2; ++round)
                for (size_t i = 0; i < cands.size(); ++i) {
                    c.resample_threads = cands[i];
                    trial_step();
                    // each resampling consumes the per-filter maxima the propagation
                    // left (and resets them), so every trial recomputes them first
                    const float ms = time_ms(c, 5, [&] {
                        launch_refresh_max(c, c.stream);
                        if (fold) launch_resample_fold(c, scratch, c.stream);
                        else launch_resample(c, scratch, dest, c.stream);
                    });
                    best_ms[i] = std::min(best_ms[i], ms);
                }
            float best = 1e30f;
            for (size_t i = 0; i < cands.size(); ++i)
                if (best_ms[i] < best) { best = best_ms[i]; best_rt = cands[i]; }
            c.resample_threads = best_rt;
        }
        o = 0;
        for (const Span &sp : spans) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(sp.dev, save + o, sp.bytes, cudaMemcpyDeviceToDevice, c.stream);
            o += sp.bytes;
        }
        const int32_t t_now = c.t;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_t, &t_now, sizeof(int32_t), cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        cudaFree(tmp);
        cudaFree(save);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(c.fhn_ppc, c.resample_threads, c.fhn_nodes, c.fhn_quad_ctas);
    }
    drop_graphs(c);
    if (h_choice) {
        h_choice[0] = c.fhn_ppc;
        h_choice[1] = c.resample_threads;
        h_choice[2] = c.mp.kind == PF_MODEL_FHN_LATTICE ? fhn_nodes(c)
                      : (c.mp.kind == PF_MODEL_FHN_PAPER ? (c.fhn_nodes ? c.fhn_nodes : 2) : 1);
    }
    return PF_OK;
}

pf_status pf_set_auxiliary(pf_ctx *h, int32_t on)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_set_auxiliary between pf_propagate and pf_resample");
    if (on && (c.prop_on || c.rec_X || c.adaptive()))
        return fail(c, PF_EUNSUPPORTED,
                    "the auxiliary filter is not combined with the learned proposal, recording or adaptive resampling");
    pf_status st = sync_materialised(c, "set_auxiliary");
    if (st != PF_OK) return st;
    drop_graphs(c);
    if (!on) {
        c.aux = false;
        return PF_OK;
    }
    if (!ensure_weight_buffers(c)) return fail(c, PF_ENOMEM, "auxiliary filter buffers: device allocation failed");
    c.aux = true;
    return reset_aux_weights(c);
}

pf_status pf_set_resampling(pf_ctx *h, double ess_threshold)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_set_resampling between pf_propagate and pf_resample");
    if (std::isnan(ess_threshold)) return fail(c, PF_EINVAL, "ess_threshold is NaN");
    const bool adaptive = ess_threshold >= 0.0 && ess_threshold <= 1.0;
    if (adaptive && (c.aux || c.prop_on || c.rec_X))
        return fail(c, PF_EUNSUPPORTED,
                    "adaptive resampling is not combined with the auxiliary filter, the learned proposal or recording");
    pf_status st = sync_materialised(c, "set_resampling");
    if (st != PF_OK) return st;
    drop_graphs(c);
    c.ess_threshold = adaptive ? ess_threshold : -1.0;
    if (!adaptive) return PF_OK;
    if (!ensure_weight_buffers(c)) return fail(c, PF_ENOMEM, "adaptive resampling buffers: device allocation failed");
    return reset_aux_weights(c);
}

pf_status pf_set_schedule(pf_ctx *h, int32_t nodes_per_thread, int32_t particles_per_cta, int32_t resample_threads)
{
    if (!h) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.fatal) return fail(c, PF_ESTATE, "context is in an error state: " + c.last_error);
    if (c.phase != 0) return fail(c, PF_ESTATE, "pf_set_schedule between pf_propagate and pf_resample");
    const bool lattice = is_lattice(c.mp.kind);
    if (nodes_per_thread != 0 &&
        !(lattice && (nodes_per_thread == 2 ||
                      ((nodes_per_thread == 4 || nodes_per_thread == 8) &&
                       (c.mp.kind == kFhnPaper ? c.mp.J % nodes_per_thread == 0
                                               : fhn_nodes_fit(c.mp.J, nodes_per_thread))))))
        return fail(c, PF_EINVAL, "nodes_per_thread: 0, 2, 4 or 8 (4 and 8: J divisible by them and J^2 / nodes "
                                  "threads within the kernel's bound)");
    if (particles_per_cta < 0 || (particles_per_cta > 0 && !lattice))
        return fail(c, PF_EINVAL, "particles_per_cta: 0, or >= 1 for the lattice");
    int max_len = 1;
    for (int32_t n : c.N) max_len = std::max(max_len, std::min(n, kTile));
    if (resample_threads != 0 && !((resample_threads == 64 || resample_threads == 128 || resample_threads == 256) &&
                                   resample_threads * 2 * kItems >= max_len))
        return fail(c, PF_EINVAL, "resample_threads: 0, or 64/128/256 with 8 particles per thread covering a tile");
    pf_status st = sync(c, "set_schedule");
    if (st != PF_OK) return st;
    c.fhn_nodes = nodes_per_thread;
    c.fhn_ppc = particles_per_cta;
    if (resample_threads) c.resample_threads = resample_threads;
    drop_graphs(c);
    return PF_OK;
}

pf_status pf_get_time(const pf_ctx *h, int32_t *t)
{
    if (!h || !t) return PF_EINVAL;
    *t = h->c.t;
    return PF_OK;
}

pf_status pf_get_state(pf_ctx *h, float *h_x)
{
    Trace trace("pf_get_state");
    if (!h || !h_x) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = sync_materialised(c, "get_state");
    if (st != PF_OK) return st;
    const int dx = c.mp.dx;
    const size_t n = (size_t)c.P * dx;
    if (is_lattice(c.mp.kind)) {
        const cudaError_t e = cudaMemcpy(h_x, c.x[c.cur], n * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_state copy");
        return PF_OK;
    }
    std::vector<float> soa(n);
    const cudaError_t e = cudaMemcpy(soa.data(), c.x[c.cur], n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state copy");
    for (int64_t p = 0; p < c.P; ++p)
        for (int v = 0; v < dx; ++v) h_x[p * dx + v] = soa[(size_t)v * c.P + p];
    return PF_OK;
}

pf_status pf_set_state(pf_ctx *h, const float *h_x, int32_t t)
{
    Trace trace("pf_set_state");
    if (!h || !h_x || t < 0) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = sync(c, "set_state");
    if (st != PF_OK) return st;
    const int dx = c.mp.dx;
    const size_t n = (size_t)c.P * dx;
    cudaError_t e;
    if (is_lattice(c.mp.kind)) {
        e = cudaMemcpy(c.x[c.cur], h_x, n * sizeof(float), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> soa(n);
        for (int64_t p = 0; p < c.P; ++p)
            for (int v = 0; v < dx; ++v) soa[(size_t)v * c.P + p] = h_x[p * dx + v];
        e = cudaMemcpy(c.x[c.cur], soa.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(c.d_t, &t, sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state copy");
    c.t = t;
    c.phase = 0;
    c.gather_pending = false;  // the state is the one given
    if (c.aux || c.adaptive()) return reset_aux_weights(c);
    return PF_OK;
}

pf_status pf_get_logw(pf_ctx *h, float *h_l)
{
    if (!h || !h_l) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = sync(c, "get_logw");
    if (st != PF_OK) return st;
    const cudaError_t e = cudaMemcpy(h_l, c.aux ? c.lw2 : c.logw, c.P * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "get_logw copy");
}

pf_status pf_set_logw(pf_ctx *h, const float *h_l)
{
    if (!h || !h_l) return PF_EINVAL;
    Ctx &c = h->c;
    if (c.aux) return fail(c, PF_EUNSUPPORTED, "pf_set_logw: not with the auxiliary filter");
    if (c.phase != 1) return fail(c, PF_ESTATE, "pf_set_logw needs a preceding pf_propagate");
    pf_status st = sync(c, "set_logw");
    if (st != PF_OK) return st;
    cudaError_t e = cudaMemcpy(c.logw, h_l, c.P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_refresh_max(c, c.stream);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "set_logw copy");
}

pf_status pf_get_ancestors(pf_ctx *h, int32_t *h_a)
{
    if (!h || !h_a) return PF_EINVAL;
    Ctx &c = h->c;
    pf_status st = sync(c, "get_ancestors");
    if (st != PF_OK) return st;
    const cudaError_t e = cudaMemcpy(h_a, c.anc, c.P * sizeof(int32_t), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PF_OK : cuda_fail(c, e, "get_ancestors copy");
}

pf_status pf_rng_philox(int64_t n, const uint32_t *d_ctr, uint32_t key0, uint32_t key1, uint32_t *d_out, void *stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return PF_EINVAL;
    return launch_rng_philox(n, d_ctr, key0, key1, d_out, (cudaStream_t)stream) == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_status pf_rng_normals(int64_t n, const uint32_t *d_ctr, uint64_t seed, float *d_z, void *stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_z))) return PF_EINVAL;
    return launch_rng_normals(n, d_ctr, seed, d_z, (cudaStream_t)stream) == cudaSuccess ? PF_OK : PF_ECUDA;
}

// Scratch layout of the stateless resampler (each piece 256-byte aligned).
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int64_t max_tiles(int32_t M, int64_t total) { return (int64_t)M + total / kTile + 1; }

size_t pf_systematic_scratch_bytes(int32_t M, int64_t total)
{
    if (M < 1 || total < 0) return 0;
    const int64_t nt = max_tiles(M, total);
    return align256(nt * sizeof(TileDesc)) + align256((size_t)M * sizeof(FilterDesc)) +
           align256(nt * kTsCount * sizeof(double)) + align256(nt * sizeof(uint64_t)) +
           align256((size_t)M * kFsCount * sizeof(double)) + align256((size_t)M * 2 * sizeof(uint64_t)) +
           align256(total * sizeof(uint64_t)) + align256(total * sizeof(int32_t)) + align256(2 * sizeof(int32_t)) +
           align256(nt * sizeof(int32_t));
}

pf_status pf_systematic_resample(int32_t M, const int32_t *h_N, const double *d_w, const double *d_u, int32_t *d_anc,
                                 void *d_scratch, size_t scratch_bytes, void *stream)
{
    if (M < 1 || !h_N || !d_w || !d_u || !d_anc || !d_scratch) return PF_EINVAL;
    if (((uintptr_t)d_scratch & 255) != 0) return PF_EINVAL;
    std::vector<int32_t> N(h_N, h_N + M);
    for (int m = 0; m < M; ++m)
        if (N[m] < 1 || N[m] > (1 << 24)) return PF_EINVAL;
    std::vector<TileDesc> tiles;
    std::vector<FilterDesc> filt;
    std::vector<int64_t> off;
    make_tiles(N, tiles, filt, off);
    const int64_t total = off[M];
    if (scratch_bytes < pf_systematic_scratch_bytes(M, total)) return PF_EINVAL;
    const int64_t nt = max_tiles(M, total);
    char *p = static_cast<char *>(d_scratch);
    auto take = [&p](size_t b) { char *r = p; p += align256(b); return r; };
    ResampleArgs a{};
    TileDesc *d_tiles = reinterpret_cast<TileDesc *>(take(nt * sizeof(TileDesc)));
    FilterDesc *d_filt = reinterpret_cast<FilterDesc *>(take((size_t)M * sizeof(FilterDesc)));
    a.tiles = d_tiles;
    a.filt = d_filt;
    a.tile_sums = reinterpret_cast<double *>(take(nt * kTsCount * sizeof(double)));
    a.tile_q = reinterpret_cast<uint64_t *>(take(nt * sizeof(uint64_t)));
    a.fstats = reinterpret_cast<double *>(take((size_t)M * kFsCount * sizeof(double)));
    a.fint = reinterpret_cast<uint64_t *>(take((size_t)M * 2 * sizeof(uint64_t)));
    a.C = reinterpret_cast<uint64_t *>(take(total * sizeof(uint64_t)));
    a.B = reinterpret_cast<int32_t *>(take(total * sizeof(int32_t)));
    a.err = reinterpret_cast<int32_t *>(take(2 * sizeof(int32_t)));
    a.tile_anc0 = reinterpret_cast<int32_t *>(take(nt * sizeof(int32_t)));
    a.w_direct = d_w;
    a.u_direct = d_u;
    a.anc = d_anc;
    a.d_t = nullptr;
    a.logw = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_filt, filt.data(), filt.size() * sizeof(FilterDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, 2 * sizeof(int32_t), s);
    // the plan is staged from host vectors: let the stream consume them first
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = launch_systematic(M, (int32_t)tiles.size(), a, s);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_status pf_simulate(const pf_model *model, double dt, const pf_obs_op *obs, const pf_noise *noise, int32_t T,
                      int32_t record, int32_t init_random, double *h_x, float *h_y)
{
    std::string why;
    ModelParams mp;
    if (!fill_params(model, dt, obs, noise, mp, why)) {
        g_create_error = why;
        return PF_EINVAL;
    }
    if (T < 0 || !h_x) return PF_EINVAL;
    const size_t nx = (size_t)(T + 1) * mp.dx, ny = (size_t)T * mp.dy;
    double *d_x = nullptr, *d_x0 = nullptr;
    float *d_y = nullptr;
    int32_t *d_idx = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d_x, nx * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_x0, mp.dx * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_y, (ny ? ny : 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_idx, mp.dy * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x0, noise->x0_mean, mp.dx * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_idx, obs->idx, mp.dy * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_simulate(mp, d_x0, d_idx, make_key(noise->seed), T, record, init_random, d_x, d_y, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_x, d_x, nx * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_y && ny) e = cudaMemcpyAsync(h_y, d_y, ny * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_x);
    cudaFree(d_x0);
    cudaFree(d_y);
    cudaFree(d_idx);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        g_create_error = std::string("simulate: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
    }
    return PF_OK;
}

}  // extern "C"
