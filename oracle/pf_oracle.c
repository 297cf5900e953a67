/*
 * pf_oracle.c -- plain, slow FP64 CPU oracle for an ensemble of M independent
 * bootstrap particle filters (Crisan, Miguez & Rios, "A simple scheme for the
 * parallelisation of particle filters ...", arXiv:1407.8071).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant generator with
 * the CUDA path; the counter-based generator below is written separately on
 * each side from its published definition.
 *
 * Everything is computed in double precision, in the order the paper states:
 *   - Algorithm 1 (bootstrap filter): initialisation (step 1), propagation and
 *     normalised weights (step 2a), resampling (step 2b).
 *   - eq. (eqGtN): the running normalising-constant estimate G_t^N.
 *   - Definition 1: the ensemble average of the M per-filter estimates.
 *   - Sec. 4.1 eqs. (eqDiscreteLorenz-1..3): Euler-Maruyama Lorenz 63.
 *   - Sec. 5.1: a diffusively coupled stochastic FitzHugh-Nagumo lattice,
 *     here in the Rogers-McCulloch form with zero-flux boundaries.
 * Resampling is systematic (allowed by the remark after Algorithm 1, which
 * admits schemes other than multinomial); multinomial resampling, the form
 * Algorithm 1 step 2b states literally, is kept for the rate tests.
 *
 * Compile with -ffp-contract=off so that every product and sum is rounded
 * separately, as written.
 *
 * Parity status per function is stated in the Python wrapper's header.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LG 0
#define ORC_LORENZ63 1
#define ORC_FHN 2
#define ORC_FHNP 3 /* the paper's own lattice variant, Sec. 5.1-5.2 */

#define ORC_STREAM_TRUTH 0u
#define ORC_STREAM_OBS 1u
#define ORC_STREAM_INIT 2u
#define ORC_STREAM_DYN 3u
#define ORC_STREAM_RESAMPLE 4u
#define ORC_STREAM_PROPOSAL 5u
#define ORC_STREAM_MISC 6u        /* also the particles' random stimulus (lattice variant of Sec. 5.1) */
#define ORC_STREAM_STIM_TRUTH 7u  /* the truth's random stimulus */

/* Model description, filled from Python (ctypes mirror in oracle/__init__.py). */
typedef struct {
    int32_t kind;      /* ORC_LG, ORC_LORENZ63, ORC_FHN                         */
    int32_t dx;        /* state dimension                                        */
    int32_t J;         /* FHN lattice side (dx = 2 J^2), else 0                  */
    int32_t K;         /* Euler-Maruyama sub-steps between observations          */
    double dt;         /* Euler-Maruyama step                                    */
    double sigma_dyn;  /* dynamical noise scale: increment sigma*sqrt(dt)*z      */
    double sigma0;     /* prior std around x0_mean                               */
    double sigma_obs;  /* observation noise std                                  */
    int32_t dy;        /* number of observed components                          */
    int32_t n_params;  /* length of params                                       */
    const double *params;   /* LG: A (dx*dx, drift -A x); L63: s,r,b; FHN: below */
    const double *x0_mean;  /* dx                                               */
    const int32_t *obs_idx; /* dy indices into the state vector                  */
} orc_model;

/* FHN parameter layout: a, b, c1, c2, d, D, stim_amp, stim_steps, stim_block */
/* FHNP (the paper's variant) parameter layout:
 *   0..3  alpha_3, alpha_2, alpha_1, alpha_0   (p3(u) = sum alpha_r u^r)
 *   4..6  beta_0, beta_1, beta_2               (eq. eqVd)
 *   7     coupling 1/D                          (eq. eqUd: (1/D) sum of the neighbours' U)
 *   8     F~, forcing amplitude;  9 forcing period (sub-steps);  10 pulse width (sub-steps)
 *   11    forced columns (m_ij = 1 for j < this)
 *   12, 13  u-, u+ thresholds of the stimulus region (eq. eqStimulusRegion)
 *   14    epsilon (Bernoulli), as an integer threshold on 24-bit uniforms: round(eps 2^24)
 *   15    stimulus amplitude;  16  l0 (steps a stimulus is held)
 * State: planes U, V and S = sub-steps since the node's last stimulus event, capped at l0
 * (Psi = amplitude while S < l0). */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox bijection; the key */
/* is bumped by the Weyl constants (golden ratio and sqrt(3)-1 in 0.32 fixed  */
/* point) between rounds.                                                     */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for the tests: ctr is n x 4, out is n x 4. */
void orc_philox_batch(int64_t n, const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out)
{
    uint32_t key[2] = {key0, key1};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Box & Muller (1958): two independent N(0,1) from two uniforms.
 * u1 = (top 24 bits of a + 1) * 2^-24 lies in (0, 1]; u2 = (top 24 bits of b) * 2^-24
 * lies in [0, 1).  Both are exact in binary32 and binary64. */
static void box_muller(uint32_t a, uint32_t b, double *z0, double *z1)
{
    double u1 = ((double)(a >> 8) + 1.0) * 0x1p-24;
    double u2 = (double)(b >> 8) * 0x1p-24;
    double R = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    *z0 = R * cos(th);
    *z1 = R * sin(th);
}

/* Four normals for one Philox block: lanes (0,1) from words (0,1), lanes (2,3) from (2,3). */
static void normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    box_muller(r[0], r[1], &z[0], &z[1]);
    box_muller(r[2], r[3], &z[2], &z[3]);
}

/* Box-Muller on raw word pairs (ab: n x 2) -> z: n x 2. */
void orc_box_muller_batch(int64_t n, const uint32_t *ab, double *z)
{
    for (int64_t i = 0; i < n; ++i) box_muller(ab[2 * i], ab[2 * i + 1], &z[2 * i], &z[2 * i + 1]);
}

void orc_normals_batch(int64_t n, const uint32_t *ctr, uint64_t seed, double *z)
{
    for (int64_t i = 0; i < n; ++i)
        normals4(seed, ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], z + 4 * i);
}

/* Normal number nu of the stream addressed by (c0, c1, c2, stream):
 * block nu/4 of the counter's last word, lane nu%4.  A one-block cache keeps
 * the oracle from recomputing Philox four times per block. */
typedef struct {
    uint64_t seed;
    uint32_t c0, c1, c2, stream;
    int64_t block;
    double z[4];
} nstream;

static void ns_init(nstream *s, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t stream)
{
    s->seed = seed; s->c0 = c0; s->c1 = c1; s->c2 = c2; s->stream = stream; s->block = -1;
}

static double ns_get(nstream *s, int64_t nu)
{
    int64_t b = nu >> 2;
    if (b != s->block) {
        normals4(s->seed, s->c0, s->c1, s->c2, (s->stream << 24) | (uint32_t)b, s->z);
        s->block = b;
    }
    return s->z[nu & 3];
}

/* ------------------------------------------------------------------------- */
/* Models.                                                                    */
/* ------------------------------------------------------------------------- */

/* Position of variable v's normal within one sub-step's block of dx normals.
 * LG and Lorenz: identity.  FHN (variable = plane*J^2 + node, plane 0 = v,
 * plane 1 = w): 2*node + plane, so the (v, w) pair of a node is adjacent. */
static int64_t noise_slot(const orc_model *md, int64_t v)
{
    if (md->kind == ORC_FHN || md->kind == ORC_FHNP) {
        int64_t nn = (int64_t)md->J * md->J;
        int64_t plane = v / nn, node = v % nn;
        return 2 * node + plane;
    }
    return v;
}

/* Drift f(x) at sub-step n (the step from x_{n-1} to x_n, n >= 1). */
static void drift(const orc_model *md, int64_t n, const double *x, double *f)
{
    const double *p = md->params;
    if (md->kind == ORC_LG) {
        int d = md->dx;
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += p[i * d + j] * x[j];
            f[i] = -s;
        }
    } else if (md->kind == ORC_LORENZ63) {
        /* Sec. 4.1; the continuous form's first equation reads -s(X1 - X2) as in
         * eq. (eqDiscreteLorenz-1). */
        double s = p[0], r = p[1], b = p[2];
        f[0] = -s * (x[0] - x[1]);
        f[1] = r * x[0] - x[1] - x[0] * x[2];
        f[2] = x[0] * x[1] - b * x[2];
    } else if (md->kind == ORC_FHNP) {
        /* eqs. eqUd, eqVd: f_U = p3(U) - V + (1/D) sum_nbr U + m F_n + Psi, f_V = b0 U + b1 V + b2;
         * the neighbour sets are the von Neumann ones of Sec. 5.2 (edges and corners have fewer) */
        int J = md->J, nn = J * J;
        double per = p[9], wid = p[10];
        int fcols = (int)p[11];
        double l0 = p[16];
        int on = fmod((double)(n - 1), per) < wid;
        const double *U = x, *V = x + nn, *S = x + 2 * nn;
        for (int i = 0; i < J; ++i)
            for (int j = 0; j < J; ++j) {
                int k = i * J + j;
                double u = U[k];
                double nb = 0.0;
                if (i > 0) nb += U[k - J];
                if (i < J - 1) nb += U[k + J];
                if (j > 0) nb += U[k - 1];
                if (j < J - 1) nb += U[k + 1];
                double p3 = ((p[0] * u + p[1]) * u + p[2]) * u + p[3];
                double force = (on && j < fcols) ? p[8] : 0.0;
                double psi = S[k] < l0 ? p[15] : 0.0;
                f[k] = p3 - V[k] + p[7] * nb + force + psi;
                f[nn + k] = p[4] * u + p[5] * V[k] + p[6];
                f[2 * nn + k] = 0.0;
            }
    } else { /* ORC_FHN */
        double a = p[0], bb = p[1], c1 = p[2], c2 = p[3], dd = p[4], D = p[5];
        double amp = p[6];
        int64_t stim_steps = (int64_t)p[7];
        int blk = (int)p[8];
        int J = md->J, nn = J * J;
        const double *vv = x, *ww = x + nn;
        for (int i = 0; i < J; ++i) {
            for (int j = 0; j < J; ++j) {
                int k = i * J + j;
                double v = vv[k], w = ww[k];
                /* zero-flux 5-point Laplacian: existing 4-neighbours minus count * v */
                double lap = 0.0;
                int cnt = 0;
                if (i > 0) { lap += vv[k - J]; cnt++; }
                if (i < J - 1) { lap += vv[k + J]; cnt++; }
                if (j > 0) { lap += vv[k - 1]; cnt++; }
                if (j < J - 1) { lap += vv[k + 1]; cnt++; }
                lap -= (double)cnt * v;
                double I = (i < blk && j < blk && (n - 1) < stim_steps) ? amp : 0.0;
                f[k] = c1 * v * (v - a) * (1.0 - v) - c2 * v * w + D * lap + I;
                f[nn + k] = bb * (v - dd * w);
            }
        }
    }
}

/* One Euler-Maruyama step x <- x + dt f(x) + sigma sqrt(dt) z, z[v] = normal of
 * variable v.  f must have room for dx doubles. */
static void em_step(const orc_model *md, int64_t n, double *x, const double *z, double *f)
{
    drift(md, n, x, f);
    double sq = md->sigma_dyn * sqrt(md->dt);
    for (int v = 0; v < md->dx; ++v) x[v] = x[v] + md->dt * f[v] + sq * z[v];
}

/* Propagate one particle (filter-local index i of filter m, or the truth with
 * c0 = 0, c2 = record) over the K sub-steps from observation t-1 to t.
 * Normal number nu = k*dx + slot(v) for sub-step k = 0..K-1, counter
 * (c0, t, c2, stream<<24 | nu/4). */
/* The lattice variant's random stimulus before sub-step k of interval t
 * (eqs. eqStimulusRegion-eqPsi_ijt): one Philox block (c0, t, c2, stream<<24 | k)
 * gives r0, r1; an event happens when (r0 >> 8) < round(eps 2^24) and the
 * stimulus region S (nodes whose U, or a neighbour's U, lies in (u-, u+)) is
 * not empty; it hits the node of rank floor((r1 >> 8) |S| / 2^24) in S
 * (row-major order) and its neighbours.  Every node's counter S ages by one
 * (capped at l0) or restarts at 0 where the event hits.  events = 0 ages only
 * (the auxiliary filter's noise-free look-ahead). */
static void fhnp_stimulus(const orc_model *md, uint64_t seed, uint32_t stream, uint32_t c0, uint32_t t, uint32_t c2,
                          int k, int events, double *x)
{
    const double *p = md->params;
    int J = md->J, nn = J * J;
    double *U = x, *S = x + 2 * nn;
    double l0 = p[16];
    int target = -1;
    if (events) {
        uint32_t ctr[4] = {c0, t, c2, (stream << 24) | (uint32_t)k}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        if ((r[0] >> 8) < (uint32_t)p[14]) {
            int64_t cnt = 0;
            for (int pass = 0; pass < 2; ++pass) {
                int64_t rank = pass ? (int64_t)(((uint64_t)(r[1] >> 8) * (uint64_t)cnt) >> 24) : -1, seen = 0;
                for (int i = 0; i < J && target < 0; ++i)
                    for (int j = 0; j < J; ++j) {
                        int q = i * J + j, in = 0;
                        int nb[5] = {q, i > 0 ? q - J : -1, i < J - 1 ? q + J : -1, j > 0 ? q - 1 : -1, j < J - 1 ? q + 1 : -1};
                        for (int e = 0; e < 5; ++e)
                            if (nb[e] >= 0 && U[nb[e]] > p[12] && U[nb[e]] < p[13]) in = 1;
                        if (!in) continue;
                        if (pass == 1 && seen == rank) { target = q; break; }
                        ++seen;
                    }
                if (pass == 0) cnt = seen;
                if (cnt == 0) break;
            }
        }
    }
    int ti = target >= 0 ? target / J : -10, tj = target >= 0 ? target % J : -10;
    for (int i = 0; i < J; ++i)
        for (int j = 0; j < J; ++j) {
            int q = i * J + j;
            int hit = (i == ti && j == tj) || (i == ti && (j == tj - 1 || j == tj + 1)) ||
                      (j == tj && (i == ti - 1 || i == ti + 1));
            S[q] = hit ? 0.0 : (S[q] + 1.0 < l0 ? S[q] + 1.0 : l0);
        }
}

static void propagate_one(const orc_model *md, uint64_t seed, uint32_t stream, uint32_t c0, uint32_t c2,
                          int32_t t, double *x, double *z, double *f)
{
    nstream ns;
    ns_init(&ns, seed, c0, (uint32_t)t, c2, stream);
    const int64_t nn = (int64_t)md->J * md->J;
    for (int k = 0; k < md->K; ++k) {
        if (md->kind == ORC_FHNP)
            fhnp_stimulus(md, seed, stream == ORC_STREAM_TRUTH ? ORC_STREAM_STIM_TRUTH : ORC_STREAM_MISC, c0,
                          (uint32_t)t, c2, k, 1, x);
        for (int v = 0; v < md->dx; ++v)
            z[v] = (md->kind == ORC_FHNP && v >= nn) ? 0.0 : ns_get(&ns, (int64_t)k * md->dx + noise_slot(md, v));
        int64_t n = (int64_t)(t - 1) * md->K + k + 1;
        em_step(md, n, x, z, f);
    }
}

/* Prior draw x0 = x0_mean + sigma0 z, z from (c0, 0, c2, stream<<24 | slot/4). */
static void prior_one(const orc_model *md, uint64_t seed, uint32_t stream, uint32_t c0, uint32_t c2, double *x)
{
    nstream ns;
    ns_init(&ns, seed, c0, 0u, c2, stream);
    const int64_t s_plane = md->kind == ORC_FHNP ? 2 * (int64_t)md->J * md->J : md->dx;  /* S starts exact */
    for (int v = 0; v < md->dx; ++v)
        x[v] = md->x0_mean[v] + (v < s_plane ? md->sigma0 * ns_get(&ns, noise_slot(md, v)) : 0.0);
}

/* log g without its constant: -1/2 sum_j (y_j - x[idx_j])^2 / sigma_obs^2. */
static double loglik(const orc_model *md, const double *x, const double *y)
{
    double s = 0.0;
    for (int j = 0; j < md->dy; ++j) {
        double e = y[j] - x[md->obs_idx[j]];
        s += e * e;
    }
    return -0.5 * s / (md->sigma_obs * md->sigma_obs);
}

/* ------------------------------------------------------------------------- */
/* Learned proposal (growth direction; the paper admits tailored importance   */
/* functions, Sec. 6 footnote).  At the observed lattice nodes, the last      */
/* Euler-Maruyama sub-step before an observation is drawn from               */
/*   q = N(m + h o_mu, (h exp(clip(o_s, -3, 3)))^2),  h = sigma sqrt(dt),      */
/* with the same normals the transition would use, and the weight gains      */
/* log p - log q.  o = MLP(5x5 patch of v, 5x5 patch of w, y at the node).    */
/* ------------------------------------------------------------------------- */
#define MLP_IN 51
#define MLP_HID 128
#define MLP_OUT 4
#define MLP_CLAMP 3.0

typedef struct {
    const float *theta; /* W1 (128x51), b1, W2 (128x128), b2, W3 (4x128), b3 */
    int32_t bf16;       /* round weights and layer inputs to bfloat16          */
    double ess_frac;    /* fall back to the transition when ESS < ess_frac N    */
    int32_t span;       /* the proposal acts on the last `span` sub-steps (1..K) */
} orc_proposal;

static double bf16r(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return x; /* inf / nan */
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* GELU in its tanh form (Hendrycks & Gimpel 2016), the network's activation:
 * x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) / 2. */
static double gelu(double x) { return 0.5 * x * (1.0 + tanh(sqrt(2.0 / M_PI) * (x + 0.044715 * x * x * x))); }

void orc_mlp_forward(const orc_proposal *pr, int64_t rows, const double *in, double *out)
{
    const float *W1 = pr->theta, *b1 = W1 + MLP_HID * MLP_IN, *W2 = b1 + MLP_HID, *b2 = W2 + MLP_HID * MLP_HID;
    const float *W3 = b2 + MLP_HID, *b3 = W3 + MLP_OUT * MLP_HID;
    double a0[MLP_IN], a1[MLP_HID], a2[MLP_HID];
    for (int64_t r = 0; r < rows; ++r) {
        for (int i = 0; i < MLP_IN; ++i) a0[i] = pr->bf16 ? bf16r(in[r * MLP_IN + i]) : in[r * MLP_IN + i];
        for (int o = 0; o < MLP_HID; ++o) {
            double z = b1[o];
            for (int i = 0; i < MLP_IN; ++i) z += (pr->bf16 ? bf16r(W1[o * MLP_IN + i]) : W1[o * MLP_IN + i]) * a0[i];
            a1[o] = pr->bf16 ? bf16r(gelu(z)) : gelu(z);
        }
        for (int o = 0; o < MLP_HID; ++o) {
            double z = b2[o];
            for (int i = 0; i < MLP_HID; ++i) z += (pr->bf16 ? bf16r(W2[o * MLP_HID + i]) : W2[o * MLP_HID + i]) * a1[i];
            a2[o] = pr->bf16 ? bf16r(gelu(z)) : gelu(z);
        }
        for (int o = 0; o < MLP_OUT; ++o) {
            double z = b3[o];
            for (int i = 0; i < MLP_HID; ++i) z += (pr->bf16 ? bf16r(W3[o * MLP_HID + i]) : W3[o * MLP_HID + i]) * a2[i];
            out[r * MLP_OUT + o] = z;
        }
    }
}

/* The network input of lattice node `node`: 5x5 patches of v and w (row-major,
 * mirrored at the edges: index -1 -> 0, -2 -> 1, J -> J-1, J+1 -> J-2) and y. */
static int mirror(int k, int J) { return k < 0 ? -k - 1 : (k >= J ? 2 * J - k - 1 : k); }

void orc_patch_row(const orc_model *md, const double *x, int32_t node, double y, double *row)
{
    int J = md->J, nn = J * J, i = node / J, j = node % J, r = 0;
    for (int di = -2; di <= 2; ++di)
        for (int dj = -2; dj <= 2; ++dj, ++r) {
            int k = mirror(i + di, J) * J + mirror(j + dj, J);
            row[r] = x[k];
            row[25 + r] = x[nn + k];
        }
    row[50] = y;
}

/* K - L ordinary sub-steps (L = pr->span, 1..K), then the network once, on
 * the state reached and y, and the last L sub-steps with the proposal at the
 * observed nodes: at each of them the node's (v, w) is drawn from
 * N(m + h o_mu, (h e^s)^2) with the sub-step's own normal, m the transition
 * mean and s = clip(o_s, -3, 3), the same outputs o for all L sub-steps; the
 * other nodes take the transition.  On return x holds the proposed state,
 * *lw = sum over the L sub-steps and observed nodes of (log p - log q), and
 * xb (dx) the state the transition alone would have produced from the state
 * before the last sub-step (the fallback's candidate; meaningful for L = 1).
 * o_rec (dy x 4) and zm_rec (dy x 4: the normals and the transition means of
 * (v, w) at the last sub-step) receive the network outputs and what they act
 * on, and row_rec (dy x 51) the network inputs, when not NULL. */
static void propagate_proposal(const orc_model *md, const orc_proposal *pr, uint64_t seed, uint32_t c0,
                               uint32_t c2, int32_t t, const double *y, double *x, double *xb, double *lw,
                               double *z, double *f, double *o_rec, double *zm_rec, double *row_rec)
{
    nstream ns;
    ns_init(&ns, seed, c0, (uint32_t)t, c2, ORC_STREAM_DYN);
    const int K = md->K, dx = md->dx, nn = md->J * md->J, dy = md->dy;
    const int L = pr->span < 1 ? 1 : (pr->span > K ? K : pr->span);
    for (int k = 0; k < K - L; ++k) {
        for (int v = 0; v < dx; ++v) z[v] = ns_get(&ns, (int64_t)k * dx + noise_slot(md, v));
        em_step(md, (int64_t)(t - 1) * K + k + 1, x, z, f);
    }
    /* the network, once, on the state before the proposed sub-steps */
    double row[MLP_IN];
    double *o = (double *)malloc(sizeof(double) * MLP_OUT * dy);
    for (int j = 0; j < dy; ++j) {
        orc_patch_row(md, x, md->obs_idx[j], y[j], row);
        if (row_rec) memcpy(row_rec + MLP_IN * j, row, sizeof(row));
        orc_mlp_forward(pr, 1, row, o + MLP_OUT * j);
    }
    if (o_rec) memcpy(o_rec, o, sizeof(double) * MLP_OUT * dy);
    const double h = md->sigma_dyn * sqrt(md->dt);
    double *prop = (double *)malloc(sizeof(double) * 2 * dy);
    *lw = 0.0;
    for (int k = K - L; k < K; ++k) {
        for (int v = 0; v < dx; ++v) z[v] = ns_get(&ns, (int64_t)k * dx + noise_slot(md, v));
        drift(md, (int64_t)(t - 1) * K + k + 1, x, f);
        for (int j = 0; j < dy; ++j) {
            const int nd = md->obs_idx[j];
            for (int c = 0; c < 2; ++c) {
                const int var = c * nn + nd;
                const double m = x[var] + md->dt * f[var];
                const double oo = o[MLP_OUT * j + 2 + c];
                const double oc = oo < -MLP_CLAMP ? -MLP_CLAMP : (oo > MLP_CLAMP ? MLP_CLAMP : oo);
                const double mu = m + h * o[MLP_OUT * j + c], sd = h * exp(oc);
                const double xv = mu + sd * z[var];
                prop[2 * j + c] = xv;
                if (k == K - 1 && zm_rec) {
                    zm_rec[4 * j + c] = z[var];
                    zm_rec[4 * j + 2 + c] = m;
                }
                *lw += (-(xv - m) * (xv - m) / (2.0 * h * h) - log(h)) - (-(xv - mu) * (xv - mu) / (2.0 * sd * sd) - log(sd));
            }
        }
        for (int v = 0; v < dx; ++v) {
            x[v] = x[v] + md->dt * f[v] + h * z[v];
            if (k == K - 1) xb[v] = x[v];
        }
        for (int j = 0; j < dy; ++j)
            for (int c = 0; c < 2; ++c) x[c * nn + md->obs_idx[j]] = prop[2 * j + c];
    }
    free(prop);
    free(o);
}

/* ------------------------------------------------------------------------- */
/* Component entry points (particle-major x: n x dx).                        */
/* ------------------------------------------------------------------------- */

void orc_prior(const orc_model *md, int64_t n, const int32_t *pid, const int32_t *fid, uint64_t seed, double *x)
{
    for (int64_t q = 0; q < n; ++q)
        prior_one(md, seed, ORC_STREAM_INIT, (uint32_t)pid[q], (uint32_t)fid[q], x + q * md->dx);
}

void orc_propagate(const orc_model *md, int64_t n, const int32_t *pid, const int32_t *fid, int32_t t,
                   uint64_t seed, int32_t stream, double *x)
{
    double *z = (double *)malloc(sizeof(double) * md->dx);
    double *f = (double *)malloc(sizeof(double) * md->dx);
    for (int64_t q = 0; q < n; ++q)
        propagate_one(md, seed, (uint32_t)stream, (uint32_t)pid[q], (uint32_t)fid[q], t, x + q * md->dx, z, f);
    free(z);
    free(f);
}

/* One Euler-Maruyama step with explicit normals (z: n x dx), for the
 * closed-form single-step pins. */
/* One observation interval of the learned-proposal filter for each particle
 * row of x (lattice): K - 1 transition sub-steps, then the last one drawn from
 * the proposal at the observed nodes (see propagate_proposal).  x (n x dx) is
 * replaced by the proposed states; xb (n x dx) receives the transition's
 * candidates, lw (n) the sum over observed nodes of log p - log q; o (n x dy x 4),
 * zm (n x dy x 4) and rows (n x dy x 51), when not NULL, the network outputs,
 * the (normals, transition means) and the network inputs at the observed nodes. */
void orc_propagate_proposal(const orc_model *md, const orc_proposal *pr, int64_t n, const int32_t *pid,
                            const int32_t *fid, int32_t t, uint64_t seed, const double *y, double *x, double *xb,
                            double *lw, double *o, double *zm, double *rows)
{
    double *z = (double *)malloc(sizeof(double) * md->dx);
    double *f = (double *)malloc(sizeof(double) * md->dx);
    for (int64_t q = 0; q < n; ++q)
        propagate_proposal(md, pr, seed, (uint32_t)pid[q], (uint32_t)fid[q], t, y, x + q * md->dx, xb + q * md->dx,
                           lw + q, z, f, o ? o + q * md->dy * 4 : NULL, zm ? zm + q * md->dy * 4 : NULL,
                           rows ? rows + q * md->dy * MLP_IN : NULL);
    free(z);
    free(f);
}

void orc_em_step(const orc_model *md, int64_t n, int64_t step, double *x, const double *z)
{
    double *f = (double *)malloc(sizeof(double) * md->dx);
    for (int64_t q = 0; q < n; ++q) em_step(md, step, x + q * md->dx, z + q * md->dx, f);
    free(f);
}

void orc_drift(const orc_model *md, int64_t step, const double *x, double *f) { drift(md, step, x, f); }

void orc_loglik(const orc_model *md, int64_t n, const double *x, const double *y, double *l)
{
    for (int64_t q = 0; q < n; ++q) l[q] = loglik(md, x + q * md->dx, y);
}

/* Per-filter normaliser (Algorithm 1 step 2a in the log domain):
 * out[0] = max l, out[1] = log sum exp(l), out[2] = sum w, out[3] = sum w^2,
 * out[4] = ESS = (sum w)^2 / sum w^2, with w = exp(l - max) and Neumaier-
 * compensated sums. */
void orc_normalise(int64_t n, const double *l, double *out)
{
    double mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (l[i] > mx) mx = l[i];
    double s = 0.0, cs = 0.0, s2 = 0.0, cs2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double w = exp(l[i] - mx);
        double t = s + w;
        if (fabs(s) >= fabs(w)) cs += (s - t) + w; else cs += (w - t) + s;
        s = t;
        double w2 = w * w;
        double t2 = s2 + w2;
        if (fabs(s2) >= fabs(w2)) cs2 += (s2 - t2) + w2; else cs2 += (w2 - t2) + s2;
        s2 = t2;
    }
    s += cs;
    s2 += cs2;
    out[0] = mx;
    out[1] = mx + log(s);
    out[2] = s;
    out[3] = s2;
    out[4] = s * s / s2;
}

/* Systematic resampling in exact arithmetic.
 * L = ceil(log2 N), sh = 52 - L; q_k = floor(w_k 2^sh) for unnormalised weights
 * w_k in [0, 1] (an exact integer below 2^53); C_k = q_0 + ... + q_k (exact);
 * u = U 2^-32 with U = floor(u 2^32); a_i = min{k : C_k > (i + u) C_{N-1} / N},
 * the comparison made exactly as C_k N 2^32 > (i 2^32 + U) C_{N-1} in 128-bit
 * integers.  Since (i + u) / N < 1 every i has an ancestor; the last positive
 * q is the fallback only if every weight quantises to zero.  The plain
 * two-pointer merge below is that definition. */
static int ceil_log2(int64_t n)
{
    int L = 0;
    while (((int64_t)1 << L) < n) ++L;
    return L;
}

void orc_quantise(int64_t N, const double *w, double *q)
{
    int sh = 52 - ceil_log2(N);
    double scale = ldexp(1.0, sh);
    for (int64_t i = 0; i < N; ++i) q[i] = floor(w[i] * scale);
}

typedef unsigned __int128 u128;

/* cumulative quantised weights; returns the last k with q_k > 0 */
static int64_t cumulative(int64_t N, const double *w, uint64_t *C)
{
    double *q = (double *)malloc(sizeof(double) * N);
    orc_quantise(N, w, q);
    uint64_t run = 0;
    int64_t last_pos = 0;
    for (int64_t k = 0; k < N; ++k) {
        run += (uint64_t)q[k];
        if (q[k] > 0.0) last_pos = k;
        C[k] = run;
    }
    free(q);
    return last_pos;
}

void orc_systematic(int64_t N, const double *w, double u, int32_t *anc)
{
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * N);
    int64_t last_pos = cumulative(N, w, C);
    const uint64_t U = (uint64_t)floor(u * 4294967296.0);
    const u128 total = C[N - 1];
    int64_t k = 0;
    for (int64_t i = 0; i < N; ++i) {
        const u128 t = ((((u128)i) << 32) | U) * total; /* (i + u) C_{N-1} 2^32 */
        while (k < N && !(((u128)C[k] * (u128)N) << 32 > t)) ++k;
        anc[i] = (int32_t)(k < N ? k : last_pos);
    }
    free(C);
}

/* Multinomial resampling (Algorithm 1 step 2b as stated): a_i = min{k : C_k > U_i C_{N-1}}
 * with the same exact prefix and independent uniforms U_i (compared exactly on the
 * 2^-32 grid). */
void orc_multinomial(int64_t N, const double *w, const double *U, int32_t *anc)
{
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * N);
    int64_t last_pos = cumulative(N, w, C);
    const u128 total = C[N - 1];
    for (int64_t i = 0; i < N; ++i) {
        const u128 t = (u128)(uint64_t)floor(U[i] * 4294967296.0) * total;
        int64_t lo = 0, hi = N; /* first k with C_k 2^32 > t */
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (((u128)C[mid] << 32) > t) hi = mid; else lo = mid + 1;
        }
        anc[i] = (int32_t)(lo < N ? lo : last_pos);
    }
    free(C);
}

/* Resampling uniform for filter m at observation t: word 0 of Philox at
 * (0, t, m, RESAMPLE<<24) times 2^-32. */
double orc_resample_u(uint64_t seed, int32_t m, int32_t t)
{
    uint32_t ctr[4] = {0u, (uint32_t)t, (uint32_t)m, ORC_STREAM_RESAMPLE << 24};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    return (double)r[0] * 0x1p-32;
}

static double multinomial_u(uint64_t seed, int32_t m, int32_t t, int64_t i)
{
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)t, (uint32_t)m, (ORC_STREAM_RESAMPLE << 24) | 1u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    return (double)r[0] * 0x1p-32;
}

/* ------------------------------------------------------------------------- */
/* Synthetic truth and observation record (Sec. 4.2: one record, generated    */
/* once and shared by every filter).                                          */
/* init_mode 0: X_0 = x0_mean; 1: X_0 = x0_mean + sigma0 z (stream MISC).     */
/* Truth dynamics use stream TRUTH with c0 = 0, c2 = record; observation     */
/* noise uses stream OBS at (0, t, record, OBS<<24 | j/4), lane j%4.          */
/* x_out: (T+1) x dx, y_out: T x dy.                                          */
/* ------------------------------------------------------------------------- */
void orc_simulate(const orc_model *md, int32_t T, uint64_t seed, int32_t record, int32_t init_mode,
                  double *x_out, double *y_out)
{
    int dx = md->dx;
    double *x = (double *)malloc(sizeof(double) * dx);
    double *z = (double *)malloc(sizeof(double) * dx);
    double *f = (double *)malloc(sizeof(double) * dx);
    if (init_mode == 1) prior_one(md, seed, ORC_STREAM_MISC, 0u, (uint32_t)record, x);
    else memcpy(x, md->x0_mean, sizeof(double) * dx);
    memcpy(x_out, x, sizeof(double) * dx);
    for (int32_t t = 1; t <= T; ++t) {
        propagate_one(md, seed, ORC_STREAM_TRUTH, 0u, (uint32_t)record, t, x, z, f);
        memcpy(x_out + (int64_t)t * dx, x, sizeof(double) * dx);
        nstream ns;
        ns_init(&ns, seed, 0u, (uint32_t)t, (uint32_t)record, ORC_STREAM_OBS);
        for (int j = 0; j < md->dy; ++j)
            y_out[(int64_t)(t - 1) * md->dy + j] = x[md->obs_idx[j]] + md->sigma_obs * ns_get(&ns, j);
    }
    free(x);
    free(z);
    free(f);
}

/* ------------------------------------------------------------------------- */
/* The ensemble: M independent runs of Algorithm 1 and the average of          */
/* Definition 1.                                                              */
/*                                                                            */
/* obs: T x dy (obs_per_filter = 0) or T x M x dy (obs_per_filter = 1).       */
/* resampler: 0 systematic, 1 multinomial.                                    */
/* Outputs (any may be NULL), row-major over (t-1, m, e):                     */
/*   est_post[T][M][n_est]  (f, pi_t^{m,N}), post-resampling mean             */
/*   est_pre [T][M][n_est]  weighted pre-resampling mean                       */
/*   log_G   [T][M]         log G_t^N, eq. (eqGtN), with the Gaussian constant */
/*   ess     [T][M]         (sum w)^2 / sum w^2 before resampling              */
/*   ens     [T][n_est]     Definition 1: mean over m of est_post               */
/* x_final: sum_m N_m x dx particle-major filter-after-filter (or NULL).       */
/* ------------------------------------------------------------------------- */
int orc_bf_run_proposal(const orc_model *md, const orc_proposal *pr, int32_t M, const int32_t *N, int32_t T,
                        const double *obs, int32_t obs_per_filter, uint64_t seed, int32_t resampler, int32_t n_est,
                        const int32_t *est_idx, double *est_post, double *est_pre, double *log_G, double *ess,
                        double *ens, double *x_final, double *fallback, int32_t n_threads);

int orc_bf_run(const orc_model *md, int32_t M, const int32_t *N, int32_t T, const double *obs,
               int32_t obs_per_filter, uint64_t seed, int32_t resampler, int32_t n_est, const int32_t *est_idx,
               double *est_post, double *est_pre, double *log_G, double *ess, double *ens, double *x_final,
               int32_t n_threads)
{
    return orc_bf_run_proposal(md, NULL, M, N, T, obs, obs_per_filter, seed, resampler, n_est, est_idx, est_post,
                               est_pre, log_G, ess, ens, x_final, NULL, n_threads);
}

/* Algorithm 1 x M with an optional learned proposal (pr != NULL, lattice only):
 * fallback[T][M] = 1 where a filter's ESS under the proposal fell below
 * ess_frac N and the step used the transition instead. */
int orc_bf_run_proposal(const orc_model *md, const orc_proposal *pr, int32_t M, const int32_t *N, int32_t T,
                        const double *obs, int32_t obs_per_filter, uint64_t seed, int32_t resampler, int32_t n_est,
                        const int32_t *est_idx, double *est_post, double *est_pre, double *log_G, double *ess,
                        double *ens, double *x_final, double *fallback, int32_t n_threads)
{
    int dx = md->dx;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (M + 1));
    off[0] = 0;
    for (int m = 0; m < M; ++m) off[m + 1] = off[m] + N[m];
    const double log_const = -0.5 * md->dy * log(2.0 * M_PI * md->sigma_obs * md->sigma_obs);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < M; ++m) {
        int64_t Nm = N[m];
        double *x = (double *)malloc(sizeof(double) * Nm * dx);
        double *xn = (double *)malloc(sizeof(double) * Nm * dx);
        double *l = (double *)malloc(sizeof(double) * Nm);
        double *w = (double *)malloc(sizeof(double) * Nm);
        double *U = (double *)malloc(sizeof(double) * Nm);
        int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * Nm);
        double *z = (double *)malloc(sizeof(double) * dx);
        double *f = (double *)malloc(sizeof(double) * dx);
        double *xb = pr ? (double *)malloc(sizeof(double) * Nm * dx) : NULL;
        double *lb = pr ? (double *)malloc(sizeof(double) * Nm) : NULL;
        double lg = 0.0;
        /* Algorithm 1, step 1 */
        for (int64_t i = 0; i < Nm; ++i) prior_one(md, seed, ORC_STREAM_INIT, (uint32_t)i, (uint32_t)m, x + i * dx);
        for (int32_t t = 1; t <= T; ++t) {
            const double *y = obs_per_filter ? obs + ((int64_t)(t - 1) * M + m) * md->dy
                                             : obs + (int64_t)(t - 1) * md->dy;
            /* step 2a: propagate and weight */
            int used_fallback = 0;
            if (pr) {
                for (int64_t i = 0; i < Nm; ++i) {
                    double lw;
                    propagate_proposal(md, pr, seed, (uint32_t)i, (uint32_t)m, t, y, x + i * dx, xb + i * dx, &lw, z,
                                       f, NULL, NULL, NULL);
                    l[i] = loglik(md, x + i * dx, y) + lw;
                    lb[i] = loglik(md, xb + i * dx, y);
                }
                double np_[5];
                orc_normalise(Nm, l, np_);
                /* the bootstrap proposal instead; only a proposal on the last sub-step has the
                   transition's candidate from the same state to fall back to */
                if (pr->span <= 1 && np_[4] < pr->ess_frac * (double)Nm) {
                    used_fallback = 1;
                    memcpy(x, xb, sizeof(double) * Nm * dx);
                    memcpy(l, lb, sizeof(double) * Nm);
                }
            } else {
                for (int64_t i = 0; i < Nm; ++i) {
                    propagate_one(md, seed, ORC_STREAM_DYN, (uint32_t)i, (uint32_t)m, t, x + i * dx, z, f);
                    l[i] = loglik(md, x + i * dx, y);
                }
            }
            double nrm[5];
            orc_normalise(Nm, l, nrm);
            for (int64_t i = 0; i < Nm; ++i) w[i] = exp(l[i] - nrm[0]);
            /* eq. (eqGtN): log G_t = log G_{t-1} + log((1/N) sum_j g_t(x_j)) */
            lg += nrm[1] - log((double)Nm) + log_const;
            int64_t row = (int64_t)(t - 1) * M + m;
            if (fallback) fallback[row] = used_fallback;
            if (log_G) log_G[row] = lg;
            if (ess) ess[row] = nrm[4];
            if (est_pre) {
                for (int e = 0; e < n_est; ++e) {
                    double s = 0.0;
                    for (int64_t i = 0; i < Nm; ++i) s += w[i] * x[i * dx + est_idx[e]];
                    est_pre[row * n_est + e] = s / nrm[2];
                }
            }
            /* step 2b: resample */
            if (resampler == 1) {
                for (int64_t i = 0; i < Nm; ++i) U[i] = multinomial_u(seed, m, t, i);
                orc_multinomial(Nm, w, U, anc);
            } else {
                orc_systematic(Nm, w, orc_resample_u(seed, m, t), anc);
            }
            for (int64_t i = 0; i < Nm; ++i) memcpy(xn + i * dx, x + (int64_t)anc[i] * dx, sizeof(double) * dx);
            double *tmp = x; x = xn; xn = tmp;
            if (est_post) {
                for (int e = 0; e < n_est; ++e) {
                    double s = 0.0;
                    for (int64_t i = 0; i < Nm; ++i) s += x[i * dx + est_idx[e]];
                    est_post[row * n_est + e] = s / (double)Nm;
                }
            }
        }
        if (x_final) memcpy(x_final + off[m] * dx, x, sizeof(double) * Nm * dx);
        free(x); free(xn); free(l); free(w); free(U); free(anc); free(z); free(f);
        free(xb); free(lb);
    }
    /* Definition 1: the ensemble average over the M filters, in filter order */
    if (ens && est_post) {
        for (int32_t t = 0; t < T; ++t)
            for (int e = 0; e < n_est; ++e) {
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += est_post[((int64_t)t * M + m) * n_est + e];
                ens[(int64_t)t * n_est + e] = s / (double)M;
            }
    }
    free(off);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Ensemble of auxiliary particle filters (Pitt & Shephard 1999), the filter  */
/* the paper runs on its lattice (Sec. 5.3; the remark after Corollary 2      */
/* extends the analysis to it).  Per filter and observation t:                */
/*   mu_i  = the noise-free Euler prediction of particle i over interval t;  */
/*   first stage: a = systematic resampling with weights                      */
/*          lambda_i = W_{t-1,i} g_t(mu_i)  (W: second-stage weights of t-1); */
/*   x_i   = the transition from x_{t-1,a_i} (the filter's own noise, the same*/
/*           counters as the bootstrap filter's particle i at step t);        */
/*   second stage: w_i = g_t(x_i) / g_t(mu_{a_i});                            */
/*   estimate (f, pi_t) = sum_i w_i f(x_i) / sum_i w_i;                       */
/*   likelihood factor (unbiased): [sum_i W_{t-1,i} lambda_i]                 */
/*                      x [(1/N) sum_i w_i]  with W_{t-1} normalised, W_0 = 1/N.*/
/* est[T][M][n_est], log_G[T][M] (running), ess[T][M] (second stage),        */
/* ens[T][n_est] (Definition 1).                                              */
/* ------------------------------------------------------------------------- */
static void predict_one(const orc_model *md, int32_t t, double *x, double *f)
{
    for (int k = 0; k < md->K; ++k) {
        if (md->kind == ORC_FHNP) fhnp_stimulus(md, 0, 0, 0, 0, 0, k, 0, x);  /* no new events: ageing only */
        int64_t n = (int64_t)(t - 1) * md->K + k + 1;
        drift(md, n, x, f);
        for (int v = 0; v < md->dx; ++v) x[v] = x[v] + md->dt * f[v];
    }
}

int orc_apf_run(const orc_model *md, int32_t M, const int32_t *N, int32_t T, const double *obs,
                int32_t obs_per_filter, uint64_t seed, int32_t n_est, const int32_t *est_idx, double *est,
                double *log_G, double *ess, double *ens, int32_t n_threads)
{
    int dx = md->dx;
    const double log_const = -0.5 * md->dy * log(2.0 * M_PI * md->sigma_obs * md->sigma_obs);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < M; ++m) {
        int64_t Nm = N[m];
        double *x = (double *)malloc(sizeof(double) * Nm * dx);
        double *xn = (double *)malloc(sizeof(double) * Nm * dx);
        double *mu = (double *)malloc(sizeof(double) * dx);
        double *la = (double *)malloc(sizeof(double) * Nm);
        double *l1 = (double *)malloc(sizeof(double) * Nm);
        double *lw2 = (double *)malloc(sizeof(double) * Nm);
        double *w = (double *)malloc(sizeof(double) * Nm);
        int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * Nm);
        double *z = (double *)malloc(sizeof(double) * dx);
        double *f = (double *)malloc(sizeof(double) * dx);
        double lg = 0.0, lse2_prev = log((double)Nm);
        for (int64_t i = 0; i < Nm; ++i) {
            prior_one(md, seed, ORC_STREAM_INIT, (uint32_t)i, (uint32_t)m, x + i * dx);
            lw2[i] = 0.0;
        }
        for (int32_t t = 1; t <= T; ++t) {
            const double *y = obs_per_filter ? obs + ((int64_t)(t - 1) * M + m) * md->dy
                                             : obs + (int64_t)(t - 1) * md->dy;
            /* first stage: look-ahead weights and resampling */
            for (int64_t i = 0; i < Nm; ++i) {
                memcpy(mu, x + i * dx, sizeof(double) * dx);
                predict_one(md, t, mu, f);
                la[i] = loglik(md, mu, y);
                l1[i] = lw2[i] + la[i];
            }
            double n1[5];
            orc_normalise(Nm, l1, n1);
            for (int64_t i = 0; i < Nm; ++i) w[i] = exp(l1[i] - n1[0]);
            orc_systematic(Nm, w, orc_resample_u(seed, m, t), anc);
            /* second stage: propagate the selected particles, weight */
            for (int64_t i = 0; i < Nm; ++i) {
                memcpy(xn + i * dx, x + (int64_t)anc[i] * dx, sizeof(double) * dx);
                propagate_one(md, seed, ORC_STREAM_DYN, (uint32_t)i, (uint32_t)m, t, xn + i * dx, z, f);
            }
            for (int64_t i = 0; i < Nm; ++i) l1[i] = loglik(md, xn + i * dx, y) - la[anc[i]];
            memcpy(lw2, l1, sizeof(double) * Nm);
            double *tmp = x; x = xn; xn = tmp;
            double n2[5];
            orc_normalise(Nm, lw2, n2);
            lg += (n1[1] - lse2_prev) + (n2[1] - log((double)Nm)) + log_const;
            lse2_prev = n2[1];
            int64_t row = (int64_t)(t - 1) * M + m;
            if (log_G) log_G[row] = lg;
            if (ess) ess[row] = n2[4];
            if (est) {
                for (int e = 0; e < n_est; ++e) {
                    double s = 0.0;
                    for (int64_t i = 0; i < Nm; ++i) s += exp(lw2[i] - n2[0]) * x[i * dx + est_idx[e]];
                    est[row * n_est + e] = s / n2[2];
                }
            }
        }
        free(x); free(xn); free(mu); free(la); free(l1); free(lw2); free(w); free(anc); free(z); free(f);
    }
    if (ens && est) {
        for (int32_t t = 0; t < T; ++t)
            for (int e = 0; e < n_est; ++e) {
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += est[((int64_t)t * M + m) * n_est + e];
                ens[(int64_t)t * n_est + e] = s / (double)M;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Bootstrap filters with resampling only when the effective sample size      */
/* falls below ess_threshold N (the standard adaptive form of step 2b; with   */
/* ess_threshold > 1 every step resamples and the run equals orc_bf_run's     */
/* systematic one).  Per filter the log-weights are carried between           */
/* resamplings: logw = lw_c + log g_t(x); log G_t gains log sum exp(logw)    */
/* - log sum exp(lw_c); the estimate is the mean under the carried weights    */
/* after the step (uniform after a resampling).                               */
/* est[T][M][n_est], log_G[T][M], ess[T][M] (before the decision),            */
/* resampled[T][M] (1 where the filter resampled), ens[T][n_est].             */
/* ------------------------------------------------------------------------- */
int orc_sir_run(const orc_model *md, int32_t M, const int32_t *N, int32_t T, const double *obs,
                int32_t obs_per_filter, uint64_t seed, double ess_threshold, int32_t n_est, const int32_t *est_idx,
                double *est, double *log_G, double *ess, double *resampled, double *ens, int32_t n_threads)
{
    int dx = md->dx;
    const double log_const = -0.5 * md->dy * log(2.0 * M_PI * md->sigma_obs * md->sigma_obs);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < M; ++m) {
        int64_t Nm = N[m];
        double *x = (double *)malloc(sizeof(double) * Nm * dx);
        double *xn = (double *)malloc(sizeof(double) * Nm * dx);
        double *lw = (double *)malloc(sizeof(double) * Nm);
        double *w = (double *)malloc(sizeof(double) * Nm);
        int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * Nm);
        double *z = (double *)malloc(sizeof(double) * dx);
        double *f = (double *)malloc(sizeof(double) * dx);
        double lg = 0.0, lse_c = log((double)Nm);
        for (int64_t i = 0; i < Nm; ++i) {
            prior_one(md, seed, ORC_STREAM_INIT, (uint32_t)i, (uint32_t)m, x + i * dx);
            lw[i] = 0.0;
        }
        for (int32_t t = 1; t <= T; ++t) {
            const double *y = obs_per_filter ? obs + ((int64_t)(t - 1) * M + m) * md->dy
                                             : obs + (int64_t)(t - 1) * md->dy;
            for (int64_t i = 0; i < Nm; ++i) {
                propagate_one(md, seed, ORC_STREAM_DYN, (uint32_t)i, (uint32_t)m, t, x + i * dx, z, f);
                lw[i] += loglik(md, x + i * dx, y);
            }
            double nrm[5];
            orc_normalise(Nm, lw, nrm);
            lg += nrm[1] - lse_c + log_const;
            int64_t row = (int64_t)(t - 1) * M + m;
            int res = nrm[4] < ess_threshold * (double)Nm;
            if (res) {
                for (int64_t i = 0; i < Nm; ++i) w[i] = exp(lw[i] - nrm[0]);
                orc_systematic(Nm, w, orc_resample_u(seed, m, t), anc);
                for (int64_t i = 0; i < Nm; ++i) memcpy(xn + i * dx, x + (int64_t)anc[i] * dx, sizeof(double) * dx);
                double *tmp = x; x = xn; xn = tmp;
                for (int64_t i = 0; i < Nm; ++i) lw[i] = 0.0;
                lse_c = log((double)Nm);
            } else {
                lse_c = nrm[1];
            }
            if (log_G) log_G[row] = lg;
            if (ess) ess[row] = nrm[4];
            if (resampled) resampled[row] = res;
            if (est) {
                double mx = lw[0];
                for (int64_t i = 1; i < Nm; ++i) if (lw[i] > mx) mx = lw[i];
                double sw = 0.0;
                for (int64_t i = 0; i < Nm; ++i) { w[i] = exp(lw[i] - mx); sw += w[i]; }
                for (int e = 0; e < n_est; ++e) {
                    double s = 0.0;
                    for (int64_t i = 0; i < Nm; ++i) s += w[i] * x[i * dx + est_idx[e]];
                    est[row * n_est + e] = s / sw;
                }
            }
        }
        free(x); free(xn); free(lw); free(w); free(anc); free(z); free(f);
    }
    if (ens && est) {
        for (int32_t t = 0; t < T; ++t)
            for (int e = 0; e < n_est; ++e) {
                double s = 0.0;
                for (int m = 0; m < M; ++m) s += est[((int64_t)t * M + m) * n_est + e];
                ens[(int64_t)t * n_est + e] = s / (double)M;
            }
    }
    return 0;
}
