// k_mlp.cu -- the learned proposal's network: BF16 tensor-core forward,
// backward and Adam (FP32 accumulation, FP32 master weights).
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

constexpr int kRowsPerCta = 64;  // 4 warps x 16 rows
constexpr int kFwdThreads = 128;

struct FwdSmem {
    __nv_bfloat16 w1[kHid * kLdIn];
    __nv_bfloat16 w2[kHid * kLdHid];
    __nv_bfloat16 w3[kOutPad * kLdHid];
    __nv_bfloat16 x[kRowsPerCta * kLdIn];
    __nv_bfloat16 h1[kRowsPerCta * kLdHid];
    __nv_bfloat16 h2[kRowsPerCta * kLdHid];
};

// Forward over R rows (persistent over 64-row tiles).  Input rows: FP32 with
// kIn columns (InBf16 = false) or BF16 with kInPad columns (InBf16 = true).
// Save = true also stores x0 (BF16), z1, z2 (FP32) and a1, a2 (BF16) for the
// backward pass.
template <bool InBf16, bool Save>
__global__ void __launch_bounds__(kFwdThreads) k_forward(const void *__restrict__ rows, int64_t R,
                                                         const __nv_bfloat16 *__restrict__ wp,
                                                         const float *__restrict__ theta, float *__restrict__ out,
                                                         __nv_bfloat16 *x0s, float *z1s, __nv_bfloat16 *a1s, float *z2s,
                                                         __nv_bfloat16 *a2s)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, c = lane & 3;
    for (int i = tid; i < kHid * kInPad; i += blockDim.x) S.w1[(i / kInPad) * kLdIn + i % kInPad] = wp[i];
    for (int i = tid; i < kHid * kHid; i += blockDim.x) S.w2[(i / kHid) * kLdHid + i % kHid] = wp[kPackW1 + i];
    for (int i = tid; i < kOutPad * kHid; i += blockDim.x)
        S.w3[(i / kHid) * kLdHid + i % kHid] = wp[kPackW1 + kPackW2 + i];
    const float *b1 = theta + kOffB1, *b2 = theta + kOffB2, *b3 = theta + kOffB3;
    const int r0 = warp * 16;
    for (int64_t base = (int64_t)blockIdx.x * kRowsPerCta; base < R; base += (int64_t)gridDim.x * kRowsPerCta) {
        __syncthreads();  // weights staged / previous tile done with sX
        for (int i = tid; i < kRowsPerCta * kInPad; i += blockDim.x) {
            const int r = i / kInPad, k = i % kInPad;
            const int64_t row = base + r;
            __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
            if (row < R) {
                if (InBf16) v = reinterpret_cast<const __nv_bfloat16 *>(rows)[row * kInPad + k];
                else if (k < kIn) v = __float2bfloat16_rn(reinterpret_cast<const float *>(rows)[row * kIn + k]);
            }
            S.x[r * kLdIn + k] = v;
            if (Save && row < R) x0s[row * kInPad + k] = v;
        }
        __syncthreads();
        // layer 1: 64 -> 128, two halves of 64 columns
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[8][4] = {};
            warp_gemm<8, kInPad>(acc, S.x, kLdIn, r0, S.w1, kLdIn, half * 64, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int row = r0 + g + 8 * hr, col = half * 64 + nt * 8 + 2 * c;
                    const float z0 = acc[nt][2 * hr] + b1[col], z1 = acc[nt][2 * hr + 1] + b1[col + 1];
                    const uint32_t a = pack_bf16(gelu(z0), gelu(z1));
                    *reinterpret_cast<uint32_t *>(&S.h1[row * kLdHid + col]) = a;
                    if (Save && base + row < R) {
                        const int64_t o = (base + row) * kHid + col;
                        z1s[o] = z0;
                        z1s[o + 1] = z1;
                        *reinterpret_cast<uint32_t *>(&a1s[o]) = a;
                    }
                }
        }
        __syncwarp();
        // layer 2: 128 -> 128
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[8][4] = {};
            warp_gemm<8, kHid>(acc, S.h1, kLdHid, r0, S.w2, kLdHid, half * 64, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int row = r0 + g + 8 * hr, col = half * 64 + nt * 8 + 2 * c;
                    const float z0 = acc[nt][2 * hr] + b2[col], z1 = acc[nt][2 * hr + 1] + b2[col + 1];
                    const uint32_t a = pack_bf16(gelu(z0), gelu(z1));
                    *reinterpret_cast<uint32_t *>(&S.h2[row * kLdHid + col]) = a;
                    if (Save && base + row < R) {
                        const int64_t o = (base + row) * kHid + col;
                        z2s[o] = z0;
                        z2s[o + 1] = z1;
                        *reinterpret_cast<uint32_t *>(&a2s[o]) = a;
                    }
                }
        }
        __syncwarp();
        // layer 3: 128 -> 4 (one 8-wide tile, columns 0..3 used)
        float acc[1][4] = {};
        warp_gemm<1, kHid>(acc, S.h2, kLdHid, r0, S.w3, kLdHid, 0, lane);
        if (c < 2) {
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                const int64_t row = base + r0 + g + 8 * hr;
                if (row < R) {
                    const int col = 2 * c;
                    out[row * kOut + col] = acc[0][2 * hr] + b3[col];
                    out[row * kOut + col + 1] = acc[0][2 * hr + 1] + b3[col + 1];
                }
            }
        }
    }
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

// dz1 = (dz2 W2) * gelu'(z1) on the tensor cores: rows of dz2 against W2^T.
__global__ void __launch_bounds__(kFwdThreads) k_hidden_grad(int64_t B, const __nv_bfloat16 *__restrict__ dz2,
                                                             const __nv_bfloat16 *__restrict__ w2t,
                                                             const float *__restrict__ z1s,
                                                             __nv_bfloat16 *__restrict__ dz1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(smem_raw);  // W2 as [in][out]: B^T for d_a1 = dz2 W2
    __nv_bfloat16 *sA = sW + kHid * kLdHid;                          // [64][kLdHid]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, c = lane & 3;
    for (int i = tid; i < kHid * kHid; i += blockDim.x) sW[(i / kHid) * kLdHid + i % kHid] = w2t[i];
    const int r0 = warp * 16;
    for (int64_t base = (int64_t)blockIdx.x * kRowsPerCta; base < B; base += (int64_t)gridDim.x * kRowsPerCta) {
        __syncthreads();
        for (int i = tid; i < kRowsPerCta * kHid; i += blockDim.x) {
            const int r = i / kHid, k = i % kHid;
            sA[r * kLdHid + k] = base + r < B ? dz2[(base + r) * kHid + k] : __float2bfloat16_rn(0.0f);
        }
        __syncthreads();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float acc[8][4] = {};
            warp_gemm<8, kHid>(acc, sA, kLdHid, r0, sW, kLdHid, half * 64, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int64_t row = base + r0 + g + 8 * hr;
                    const int col = half * 64 + nt * 8 + 2 * c;
                    if (row < B) {
                        const float v0 = acc[nt][2 * hr] * gelu_grad(z1s[row * kHid + col]);
                        const float v1 = acc[nt][2 * hr + 1] * gelu_grad(z1s[row * kHid + col + 1]);
                        *reinterpret_cast<uint32_t *>(&dz1[row * kHid + col]) = pack_bf16(v0, v1);
                    }
                }
        }
    }
}

// Weight gradients over one chunk of kChunk rows (tensor cores, the rows are
// the reduction dimension): dW2 = dz2^T a1, dW1 = dz1^T x0; plus, on the CUDA
// cores, dW3 = d_out^T a2 and the bias sums.  Writes the chunk's partial
// gradient (parameter layout) and its loss sum.
constexpr int kChunk = 128;
constexpr int kLdChunk = kChunk + 8;
constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads) k_weight_grad(int64_t B, const __nv_bfloat16 *__restrict__ x0s,
                                                              const __nv_bfloat16 *__restrict__ a1s,
                                                              const __nv_bfloat16 *__restrict__ a2s,
                                                              const __nv_bfloat16 *__restrict__ dz1,
                                                              const __nv_bfloat16 *__restrict__ dz2,
                                                              const float *__restrict__ dout,
                                                              const float *__restrict__ row_loss, float *partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *sDz2T = reinterpret_cast<__nv_bfloat16 *>(smem_raw);  // [128 out][chunk]
    __nv_bfloat16 *sDz1T = sDz2T + kHid * kLdChunk;                      // [128 out][chunk]
    __nv_bfloat16 *sA1T = sDz1T + kHid * kLdChunk;                       // [128 in][chunk]
    __nv_bfloat16 *sX0T = sA1T + kHid * kLdChunk;                        // [64 in][chunk]
    float *red = reinterpret_cast<float *>(sX0T + kInPad * kLdChunk);    // [kGradThreads]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, c = lane & 3;
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int n = (int)min((int64_t)kChunk, B - base);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int i = tid; i < kChunk * kHid; i += blockDim.x) {
        const int r = i / kHid, k = i % kHid;
        const bool ok = r < n;
        sDz2T[k * kLdChunk + r] = ok ? dz2[(base + r) * kHid + k] : zero;
        sDz1T[k * kLdChunk + r] = ok ? dz1[(base + r) * kHid + k] : zero;
        sA1T[k * kLdChunk + r] = ok ? a1s[(base + r) * kHid + k] : zero;
    }
    for (int i = tid; i < kChunk * kInPad; i += blockDim.x) {
        const int r = i / kInPad, k = i % kInPad;
        sX0T[k * kLdChunk + r] = r < n ? x0s[(base + r) * kInPad + k] : zero;
    }
    __syncthreads();
    float *pg = partial + (int64_t)blockIdx.x * (kParams + 1);
    // dW2 [128 out][128 in]: warp w owns output rows 16w..16w+15
    {
        float acc[16][4] = {};
        warp_gemm<16, kChunk>(acc, sDz2T, kLdChunk, warp * 16, sA1T, kLdChunk, 0, lane);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int o = warp * 16 + g + 8 * (e >> 1), in = nt * 8 + 2 * c + (e & 1);
                pg[kOffW2 + o * kHid + in] = acc[nt][e];
            }
    }
    // dW1 [128 out][51 in]
    {
        float acc[8][4] = {};
        warp_gemm<8, kChunk>(acc, sDz1T, kLdChunk, warp * 16, sX0T, kLdChunk, 0, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int o = warp * 16 + g + 8 * (e >> 1), in = nt * 8 + 2 * c + (e & 1);
                if (in < kIn) pg[kOffW1 + o * kIn + in] = acc[nt][e];
            }
    }
    // dW3 [4][128] = d_out^T a2 and the bias sums (rows in order)
    for (int j = tid; j < kOut * kHid; j += blockDim.x) {
        const int o = j / kHid, in = j % kHid;
        float s = 0.0f;
        for (int r = 0; r < n; ++r) s = fmaf(dout[(base + r) * kOut + o], __bfloat162float(a2s[(base + r) * kHid + in]), s);
        pg[kOffW3 + j] = s;
    }
    for (int j = tid; j < kHid; j += blockDim.x) {
        float s1 = 0.0f, s2 = 0.0f;
        for (int r = 0; r < n; ++r) {
            s1 += __bfloat162float(sDz1T[j * kLdChunk + r]);
            s2 += __bfloat162float(sDz2T[j * kLdChunk + r]);
        }
        pg[kOffB1 + j] = s1;
        pg[kOffB2 + j] = s2;
    }
    if (tid < kOut) {
        float s = 0.0f;
        for (int r = 0; r < n; ++r) s += dout[(base + r) * kOut + tid];
        pg[kOffB3 + tid] = s;
    }
    // loss sum of the chunk, fixed order
    float l = 0.0f;
    for (int r = tid; r < n; r += blockDim.x) l += row_loss[base + r];
    red[tid] = l;
    __syncthreads();
    if (tid == 0) {
        float s = 0.0f;
        for (int i = 0; i < (int)blockDim.x; ++i) s += red[i];
        pg[kParams] = s;
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

size_t fwd_smem() { return sizeof(FwdSmem); }

int persistent_grid(int64_t R)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int64_t tiles = (R + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t g = 2 * (int64_t)sms;
    return (int)(tiles < g ? (tiles > 0 ? tiles : 1) : g);
}

void set_smem_attrs()
{
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_forward<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        cudaFuncSetAttribute(k_forward<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        cudaFuncSetAttribute(k_forward<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        const int hs = (int)((kHid * kLdHid + kRowsPerCta * kLdHid) * sizeof(__nv_bfloat16));
        cudaFuncSetAttribute(k_hidden_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, hs);
        const int ws = (int)((3 * kHid + kInPad) * kLdChunk * sizeof(__nv_bfloat16) + kGradThreads * sizeof(float));
        cudaFuncSetAttribute(k_weight_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, ws);
    });
}

}  // namespace mlp

// Launchers used by the filter (pf_capi.cu / k_proposal.cu).
cudaError_t launch_mlp_pack(const float *theta, __nv_bfloat16 *wp, __nv_bfloat16 *w2t, cudaStream_t s)
{
    mlp::k_pack<<<(mlp::kPackTotal + 255) / 256, 256, 0, s>>>(theta, wp, w2t);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward_bf16(const __nv_bfloat16 *rows, int64_t R, const __nv_bfloat16 *wp, const float *theta,
                                    float *out, cudaStream_t s)
{
    if (R <= 0) return cudaSuccess;
    mlp::set_smem_attrs();
    mlp::k_forward<true, false><<<mlp::persistent_grid(R), mlp::kFwdThreads, mlp::fwd_smem(), s>>>(
        rows, R, wp, theta, out, nullptr, nullptr, nullptr, nullptr, nullptr);
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
    int64_t step = 0;
};

static void trainer_free(pf_mlp_trainer *t)
{
    void *ptrs[] = {t->theta, t->m, t->v, t->grad, t->wp, t->w2t, t->x0, t->a1, t->a2, t->dz1, t->dz2,
                    t->z1, t->z2, t->out, t->dout, t->row_loss, t->partial, t->xb, t->rb};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

extern "C" {

pf_status pf_mlp_forward(int64_t rows, const float *d_in, const float *d_theta, float *d_out, void *stream)
{
    if (rows < 0 || (rows > 0 && (!d_in || !d_theta || !d_out))) return PF_EINVAL;
    if (rows == 0) return PF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16 *wp = nullptr;
    // the packed weights live only for this call (stream-ordered allocation)
    cudaError_t e = cudaMallocAsync((void **)&wp, (mlp::kPackTotal + mlp::kHid * mlp::kHid) * sizeof(__nv_bfloat16), s);
    if (e != cudaSuccess) return PF_ENOMEM;
    e = launch_mlp_pack(d_theta, wp, wp + mlp::kPackTotal, s);
    if (e == cudaSuccess) {
        mlp::set_smem_attrs();
        mlp::k_forward<false, false><<<mlp::persistent_grid(rows), mlp::kFwdThreads, mlp::fwd_smem(), s>>>(
            d_in, rows, wp, d_theta, d_out, nullptr, nullptr, nullptr, nullptr, nullptr);
        e = cudaGetLastError();
    }
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
    const int64_t B = max_batch, P = mlp::kParams, chunks = (B + mlp::kChunk - 1) / mlp::kChunk;
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
              cudaMalloc(&t->xb, B * mlp::kIn * 4) == cudaSuccess && cudaMalloc(&t->rb, B * 2 * 4) == cudaSuccess;
    if (ok) ok = cudaMemcpy(t->theta, h_theta, P * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemset(t->m, 0, P * 4) == cudaSuccess && cudaMemset(t->v, 0, P * 4) == cudaSuccess;
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
    mlp::set_smem_attrs();
    const int64_t chunks = (batch + mlp::kChunk - 1) / mlp::kChunk;
    cudaError_t e = launch_mlp_pack(t->theta, t->wp, t->w2t, s);
    if (e == cudaSuccess) {
        mlp::k_forward<false, true><<<mlp::persistent_grid(batch), mlp::kFwdThreads, mlp::fwd_smem(), s>>>(
            d_X, batch, t->wp, t->theta, t->out, t->x0, t->z1, t->a1, t->z2, t->a2);
        mlp::k_out_grad<<<(unsigned)((batch + 127) / 128), 128, 0, s>>>(batch, t->out, d_R, t->wp, t->z2, t->dout, t->dz2,
                                                                       t->row_loss);
        const size_t hs = (mlp::kHid * mlp::kLdHid + mlp::kRowsPerCta * mlp::kLdHid) * sizeof(__nv_bfloat16);
        mlp::k_hidden_grad<<<mlp::persistent_grid(batch), mlp::kFwdThreads, hs, s>>>(batch, t->dz2, t->w2t, t->z1, t->dz1);
        const size_t ws = (3 * mlp::kHid + mlp::kInPad) * mlp::kLdChunk * sizeof(__nv_bfloat16) +
                          mlp::kGradThreads * sizeof(float);
        mlp::k_weight_grad<<<(unsigned)chunks, mlp::kGradThreads, ws, s>>>(batch, t->x0, t->a1, t->a2, t->dz1, t->dz2,
                                                                          t->dout, t->row_loss, t->partial);
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
        if (h_grad) e = cudaMemcpyAsync(h_grad, t->grad, mlp::kParams * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&loss_sum, t->grad + mlp::kParams, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
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
