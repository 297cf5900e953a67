// k_mlp.cu -- the learned proposal's network: packing, the training step's
// loss gradient and Adam update (FP32 master weights), shuffled batches, and
// the C entry points of the network; the GEMMs of the forward and of the
// backward pass run on the tensor cores (tcgen05: k_proposal_tc.cu,
// k_mlp_tc.cu) with BF16 operands and FP32 accumulation.
//
// Training minimises the Gaussian negative log-likelihood of standardised
// residuals r = (x'_target - m_p) / h under q = N(m_p + h o_mu, (h e^{o_s})^2):
//   L = mean_rows sum_c [ (r_c - o_mu_c)^2 / (2 e^{2 s_c}) + s_c ],  s_c = clip(o_s_c, -3, 3).
// Every reduction runs in a fixed order, so a training step is deterministic.
#include <cmath>
#include <mutex>

#include "mlp_device.cuh"
#include "pf.h"
#include "pf_internal.h"

namespace pf {
namespace mlp {

// ---------------------------------------------------------------------------
// Packing: FP32 master parameters -> BF16 tiles (W1 padded to 64 columns,
// W3 padded to 8 rows) and W2^T (for the backward pass).
// ---------------------------------------------------------------------------
__global__ void k_pack(const float *__restrict__ theta, __nv_bfloat16 *__restrict__ wp, __nv_bfloat16 *__restrict__ w2t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kPackW1) {
        const int n = i / kInPad, k = i % kInPad;
        wp[i] = __float2bfloat16_rn(k < kIn ? theta[kOffW1 + n * kIn + k] : 0.0f);
    } else if (i < kPackW1 + kPackW2) {
        const int j = i - kPackW1;
        wp[i] = __float2bfloat16_rn(theta[kOffW2 + j]);
        const int o = j / kHid, in = j % kHid;
        w2t[in * kHid + o] = __float2bfloat16_rn(theta[kOffW2 + j]);
    } else if (i < kPackTotal) {
        const int j = i - kPackW1 - kPackW2;
        const int n = j / kHid, k = j % kHid;
        wp[i] = __float2bfloat16_rn(n < kOut ? theta[kOffW3 + n * kHid + k] : 0.0f);
    }
}

// ---------------------------------------------------------------------------
// Shuffled mini-batches.  pi is a keyed bijection of [0, n): four rounds of
// (add a key, multiply by an odd constant, xor with the upper half shifted
// down), each a bijection of the k-bit integers, 2^k >= n, and cycle-walking
// (apply the rounds again while the value is >= n) to stay inside [0, n).
// The round keys are the four words of Philox4x32-10 at counter
// (0, 0, 0, stream 6) under the caller's 64-bit seed.
// ---------------------------------------------------------------------------
struct Perm {
    uint64_t n, mask;
    int half;
    uint64_t key[4];
};

__device__ __forceinline__ Perm make_perm(uint64_t n, const Key &key)
{
    Perm p;
    p.n = n;
    int k = 1;
    while ((uint64_t(1) << k) < n) ++k;
    p.mask = (uint64_t(1) << k) - 1;
    p.half = (k + 1) / 2;
    const uint4 r = philox4x32_10(make_uint4(0u, 0u, 0u, 6u << 24), key);
    p.key[0] = r.x; p.key[1] = r.y; p.key[2] = r.z; p.key[3] = r.w;
    return p;
}

__device__ __forceinline__ uint64_t perm_rounds(uint64_t x, const Perm &p)
{
    const uint64_t C[4] = {0x9E3779B97F4A7C15ull, 0xC2B2AE3D27D4EB4Full, 0x165667B19E3779F9ull, 0xD6E8FEB86659FD93ull};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        x = (x + p.key[r]) & p.mask;
        x = (x * C[r]) & p.mask;
        x ^= x >> p.half;
    }
    return x;
}

// pi(i) for i < n: the walk stays on the cycle of i, which holds i itself, so it ends.
__device__ __forceinline__ uint64_t perm_apply(uint64_t i, const Perm &p)
{
    uint64_t y = perm_rounds(i, p);
    while (y >= p.n) y = perm_rounds(y, p);
    return y;
}

__global__ void k_permutation(int64_t n, Key key, int64_t *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Perm p = make_perm((uint64_t)n, key);
    out[i] = (int64_t)perm_apply((uint64_t)i, p);
}

// Rows pi(first + j), j < batch, of (X, R) into the batch buffers.
__global__ void k_gather_batch(int64_t n, const float *__restrict__ X, const float *__restrict__ R, int64_t batch,
                               int64_t first, Key key, float *__restrict__ Xb, float *__restrict__ Rb)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= batch) return;
    const Perm p = make_perm((uint64_t)n, key);
    const int64_t src = (int64_t)perm_apply((uint64_t)(first + j), p);
    for (int c = 0; c < kIn; ++c) Xb[j * kIn + c] = X[src * kIn + c];
    Rb[j * 2] = R[src * 2];
    Rb[j * 2 + 1] = R[src * 2 + 1];
}

// Output gradient (thread per row): d_out from the NLL, d_a2 = d_out W3,
// dz2 = d_a2 * gelu'(z2); stores d_out (FP32), dz2 (BF16) and the row loss.
__global__ void k_out_grad(int64_t B, const float *__restrict__ out, const float *__restrict__ Rres,
                           const __nv_bfloat16 *__restrict__ wp, const float *__restrict__ z2s,
                           float *__restrict__ dout, __nv_bfloat16 *__restrict__ dz2, float *__restrict__ row_loss)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float inv_b = 1.0f / (float)B;
    float d[4], loss = 0.0f;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
        const float mu = out[b * kOut + cc], sr = out[b * kOut + 2 + cc];
        const float s = fminf(fmaxf(sr, -kClamp), kClamp);
        const float inv = __expf(-2.0f * s), e = Rres[b * 2 + cc] - mu;
        loss += 0.5f * e * e * inv + s;
        d[cc] = -e * inv * inv_b;
        d[2 + cc] = (sr > -kClamp && sr < kClamp) ? (1.0f - e * e * inv) * inv_b : 0.0f;
    }
    row_loss[b] = loss;
#pragma unroll
    for (int o = 0; o < 4; ++o) dout[b * kOut + o] = d[o];
    const __nv_bfloat16 *w3 = wp + kPackW1 + kPackW2;
    for (int j = 0; j < kHid; j += 2) {
        float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            g0 = fmaf(d[o], __bfloat162float(w3[o * kHid + j]), g0);
            g1 = fmaf(d[o], __bfloat162float(w3[o * kHid + j + 1]), g1);
        }
        g0 *= gelu_grad(z2s[b * kHid + j]);
        g1 *= gelu_grad(z2s[b * kHid + j + 1]);
        *reinterpret_cast<uint32_t *>(&dz2[b * kHid + j]) = pack_bf16(g0, g1);
    }
}

// Sum of the chunk partials in chunk order, then Adam (FP32 master weights).
__global__ void k_adam(int n_chunks, const float *__restrict__ partial, float *theta, float *m, float *v, float *grad,
                       float lr, float beta1, float beta2, float eps, float bc1, float bc2)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > kParams) return;
    float gsum = 0.0f;
    for (int k = 0; k < n_chunks; ++k) gsum += partial[(int64_t)k * (kParams + 1) + j];
    grad[j] = gsum;
    if (j == kParams || lr == 0.0f) return;  // slot kParams carries the loss sum
    const float mj = beta1 * m[j] + (1.0f - beta1) * gsum;
    const float vj = beta2 * v[j] + (1.0f - beta2) * gsum * gsum;
    m[j] = mj;
    v[j] = vj;
    theta[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + eps);
}

}  // namespace mlp

// Launchers used by the filter (pf_capi.cu / k_proposal.cu).
cudaError_t launch_mlp_pack(const float *theta, __nv_bfloat16 *wp, __nv_bfloat16 *w2t, cudaStream_t s)
{
    mlp::k_pack<<<(mlp::kPackTotal + 255) / 256, 256, 0, s>>>(theta, wp, w2t);
    return cudaGetLastError();
}

}  // namespace pf

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace pf;

struct pf_mlp_trainer {
    int64_t max_batch = 0;
    int device = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *wp = nullptr, *w2t = nullptr;
    __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *dz1 = nullptr, *dz2 = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *out = nullptr, *dout = nullptr, *row_loss = nullptr, *partial = nullptr;
    float *xb = nullptr, *rb = nullptr;  // a shuffled batch's rows
    int32_t *err = nullptr;              // [2] an expired tensor-core wait
    int64_t step = 0;
};

static void trainer_free(pf_mlp_trainer *t)
{
    void *ptrs[] = {t->theta, t->m, t->v, t->grad, t->wp, t->w2t, t->x0, t->a1, t->a2, t->dz1, t->dz2,
                    t->z1, t->z2, t->out, t->dout, t->row_loss, t->partial, t->xb, t->rb, t->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

extern "C" {

pf_status pf_mlp_forward(int64_t rows, const float *d_in, const float *d_theta, float *d_out, void *stream)
{
    if (rows < 0 || (rows > 0 && (!d_in || !d_theta || !d_out))) return PF_EINVAL;
    if (((uintptr_t)d_out & 15u) != 0) return PF_EINVAL;  // float4 rows
    if (rows == 0) return PF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16 *wp = nullptr;
    // the packed weights live only for this call (stream-ordered allocation)
    cudaError_t e = cudaMallocAsync((void **)&wp, (mlp::kPackTotal + mlp::kHid * mlp::kHid) * sizeof(__nv_bfloat16), s);
    if (e != cudaSuccess) return PF_ENOMEM;
    e = launch_mlp_pack(d_theta, wp, wp + mlp::kPackTotal, s);
    if (e == cudaSuccess)
        e = launch_train_forward_tc(d_in, rows, wp, d_theta, d_out, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                    s);
    cudaFreeAsync(wp, s);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_status pf_mlp_trainer_create(const float *h_theta, int32_t n_params, int64_t max_batch, pf_mlp_trainer **out)
{
    if (!out) return PF_EINVAL;
    *out = nullptr;
    if (!h_theta || n_params != mlp::kParams || max_batch < 1) return PF_EINVAL;
    pf_mlp_trainer *t = new (std::nothrow) pf_mlp_trainer();
    if (!t) return PF_ENOMEM;
    t->max_batch = max_batch;
    cudaGetDevice(&t->device);
    const int64_t B = max_batch, P = mlp::kParams, chunks = (B + 127) / 128;  // 128-row chunks of the weight gradient
    bool ok = cudaMalloc(&t->theta, P * 4) == cudaSuccess && cudaMalloc(&t->m, P * 4) == cudaSuccess &&
              cudaMalloc(&t->v, P * 4) == cudaSuccess && cudaMalloc(&t->grad, (P + 1) * 4) == cudaSuccess &&
              cudaMalloc(&t->wp, mlp::kPackTotal * 2) == cudaSuccess &&
              cudaMalloc(&t->w2t, mlp::kHid * mlp::kHid * 2) == cudaSuccess &&
              cudaMalloc(&t->x0, B * mlp::kInPad * 2) == cudaSuccess && cudaMalloc(&t->a1, B * mlp::kHid * 2) == cudaSuccess &&
              cudaMalloc(&t->a2, B * mlp::kHid * 2) == cudaSuccess && cudaMalloc(&t->dz1, B * mlp::kHid * 2) == cudaSuccess &&
              cudaMalloc(&t->dz2, B * mlp::kHid * 2) == cudaSuccess && cudaMalloc(&t->z1, B * mlp::kHid * 4) == cudaSuccess &&
              cudaMalloc(&t->z2, B * mlp::kHid * 4) == cudaSuccess && cudaMalloc(&t->out, B * mlp::kOut * 4) == cudaSuccess &&
              cudaMalloc(&t->dout, B * mlp::kOut * 4) == cudaSuccess && cudaMalloc(&t->row_loss, B * 4) == cudaSuccess &&
              cudaMalloc(&t->partial, chunks * (P + 1) * 4) == cudaSuccess &&
              cudaMalloc(&t->xb, B * mlp::kIn * 4) == cudaSuccess && cudaMalloc(&t->rb, B * 2 * 4) == cudaSuccess &&
              cudaMalloc(&t->err, 2 * 4) == cudaSuccess;
    if (ok) ok = cudaMemcpy(t->theta, h_theta, P * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemset(t->m, 0, P * 4) == cudaSuccess && cudaMemset(t->v, 0, P * 4) == cudaSuccess &&
                 cudaMemset(t->err, 0, 2 * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        trainer_free(t);
        delete t;
        return PF_ENOMEM;
    }
    *out = t;
    return PF_OK;
}

void pf_mlp_trainer_destroy(pf_mlp_trainer *t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    trainer_free(t);
    delete t;
}

pf_status pf_mlp_train_step(pf_mlp_trainer *t, int64_t batch, const float *d_X, const float *d_R, float lr,
                            float *h_grad, double *h_loss, void *stream)
{
    if (!t || batch < 1 || batch > t->max_batch || !d_X || !d_R) return PF_EINVAL;
    cudaSetDevice(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t chunks = (batch + 127) / 128;
    cudaError_t e = launch_mlp_pack(t->theta, t->wp, t->w2t, s);
    if (e == cudaSuccess)
        e = launch_train_forward_tc(d_X, batch, t->wp, t->theta, t->out, t->x0, t->z1, t->a1, t->z2, t->a2, t->err, s);
    if (e == cudaSuccess) {
        mlp::k_out_grad<<<(unsigned)((batch + 127) / 128), 128, 0, s>>>(batch, t->out, d_R, t->wp, t->z2, t->dout, t->dz2,
                                                                       t->row_loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_hidden_grad_tc(batch, t->dz2, t->w2t, t->z1, t->dz1, t->err, s);
    if (e == cudaSuccess)
        e = launch_weight_grad_tc(batch, t->x0, t->a1, t->a2, t->dz1, t->dz2, t->dout, t->row_loss, t->partial, t->err, s);
    if (e == cudaSuccess) {
        const float b1 = 0.9f, b2 = 0.999f;
        const int64_t step = lr != 0.0f ? t->step + 1 : t->step;
        const float bc1 = 1.0f - powf(b1, (float)(step > 0 ? step : 1)), bc2 = 1.0f - powf(b2, (float)(step > 0 ? step : 1));
        mlp::k_adam<<<(mlp::kParams + 1 + 255) / 256, 256, 0, s>>>((int)chunks, t->partial, t->theta, t->m, t->v, t->grad,
                                                                  lr, b1, b2, 1e-8f, bc1, bc2);
        e = cudaGetLastError();
        if (lr != 0.0f) t->step = step;
    }
    if (e == cudaSuccess && (h_grad || h_loss)) {
        static thread_local float loss_sum;
        static thread_local int32_t err_word[2];
        if (h_grad) e = cudaMemcpyAsync(h_grad, t->grad, mlp::kParams * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&loss_sum, t->grad + mlp::kParams, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(err_word, t->err, sizeof(err_word), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && (err_word[0] & kErrTimeout)) return PF_ETIMEOUT;
        if (e == cudaSuccess && h_loss) *h_loss = (double)loss_sum / (double)batch;
    }
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_status pf_permutation(int64_t n, uint64_t seed, int64_t *d_perm, void *stream)
{
    if (n < 0 || (n > 0 && !d_perm)) return PF_EINVAL;
    if (n == 0) return PF_OK;
    mlp::k_permutation<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, make_key(seed), d_perm);
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_ECUDA;
}

pf_status pf_mlp_train_step_shuffled(pf_mlp_trainer *t, int64_t n, const float *d_X, const float *d_R, int64_t batch,
                                     int64_t first, uint64_t perm_seed, float lr, float *h_grad, double *h_loss,
                                     void *stream)
{
    if (!t || !d_X || !d_R || batch < 1 || batch > t->max_batch || first < 0 || n < 1 || first + batch > n)
        return PF_EINVAL;
    cudaSetDevice(t->device);
    cudaStream_t s = (cudaStream_t)stream;
    mlp::k_gather_batch<<<(unsigned)((batch + 255) / 256), 256, 0, s>>>(n, d_X, d_R, batch, first, make_key(perm_seed),
                                                                       t->xb, t->rb);
    if (cudaGetLastError() != cudaSuccess) return PF_ECUDA;
    return pf_mlp_train_step(t, batch, t->xb, t->rb, lr, h_grad, h_loss, stream);
}

pf_status pf_mlp_trainer_get(pf_mlp_trainer *t, float *h_theta)
{
    if (!t || !h_theta) return PF_EINVAL;
    cudaSetDevice(t->device);
    return cudaMemcpy(h_theta, t->theta, mlp::kParams * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PF_OK : PF_ECUDA;
}

}  // extern "C"
