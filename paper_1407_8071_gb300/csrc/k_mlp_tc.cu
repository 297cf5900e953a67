// k_mlp_tc.cu -- the backward GEMMs of the proposal network's training step
// on the fifth-generation tensor cores (tcgen05, accumulators in tensor memory).
//
//   k_hidden_grad_tc   dz1 = (dz2 W2) * gelu'(z1): 128-row tiles of dz2 against
//                      W2^T, the GELU derivative in the epilogue (BF16 out);
//   k_weight_grad_tc   per chunk of 128 rows, the rows are the reduction
//                      dimension: dW2 = dz2^T a1 and dW1 = dz1^T x0, staged
//                      transposed into shared memory (K-major in the rows), plus,
//                      on the CUDA cores, dW3 = d_out^T a2, the bias sums and the
//                      chunk's loss; one partial gradient per chunk, summed in
//                      chunk order by the Adam kernel (deterministic).
// The forward of the training step is the filter's tensor-core forward in its
// training mode (k_proposal_tc.cu).  Every tensor-core wait is bounded; an
// expired one sets the trainer's error word and the kernel returns.
#include <cstdint>
#include <mutex>

#include "mlp_device.cuh"
#include "pf.h"
#include "pf_internal.h"
#include "tc_device.cuh"

namespace pf {
namespace tc {

constexpr int kGThreads = 256;
constexpr int kGRows = 128;

// ---------------------------------------------------------------------------
// dz1 = (dz2 W2) * gelu'(z1)
// ---------------------------------------------------------------------------
constexpr uint32_t kHgOffW = 0;                          // W2^T: 128 x 128
constexpr uint32_t kHgOffA = kHgOffW + 128 * 128 * 2;    // dz2 tile: 128 x 128
constexpr uint32_t kHgOffBar = kHgOffA + 128 * 128 * 2;
constexpr uint32_t kHgOffTmem = kHgOffBar + 8;
constexpr uint32_t kHgSmem = kHgOffTmem + 8;
constexpr uint32_t kHgTmemCols = 128;

__global__ void __launch_bounds__(kGThreads, 1)
    k_hidden_grad_tc(int64_t B, const __nv_bfloat16 *__restrict__ dz2, const __nv_bfloat16 *__restrict__ w2t,
                     const float *__restrict__ z1, __nv_bfloat16 *__restrict__ dz1, int32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar = smem_u32(smem + kHgOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kHgOffTmem);
    // W2^T [in][out] is the B operand (N = in, K = out), K-major
    const uint4 *wg = reinterpret_cast<const uint4 *>(w2t);
    for (int i = tid; i < 128 * 16; i += kGThreads) {
        const int n = i >> 4, g = i & 15;
        *reinterpret_cast<uint4 *>(smem + kHgOffW + cm_off(n, g, 128)) = wg[n * 16 + g];
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kHgTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int row = tid & (kGRows - 1), half = tid >> 7;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t id128 = idesc_bf16(128, 128);
    const int64_t n_tiles = (B + kGRows - 1) / kGRows;
    uint32_t phase = 0;
    bool expired = false;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t g = tile * kGRows + row;
        // this thread's half of its row of dz2 -> A (64 of the 128 columns)
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(dz2 + g * mlp::kHid) + 8 * half;
#pragma unroll
            for (int kg = 0; kg < 8; ++kg)
                *reinterpret_cast<uint4 *>(smem + kHgOffA + cm_off(row, 8 * half + kg, 128)) =
                    g < B ? src[kg] : make_uint4(0u, 0u, 0u, 0u);
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 8; ++k)
                umma(tmem, sdesc(sbase + kHgOffA + 256 * k, 128, 2048), sdesc(sbase + kHgOffW + 256 * k, 128, 2048),
                     id128, k > 0);
            umma_commit(bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) { expired = true; break; }
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(lane_base + c0, v);
            tc_wait_ld();
            if (g < B) {
                const float *zr = z1 + g * mlp::kHid + c0;
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    w[i] = mlp::pack_bf16(__uint_as_float(v[2 * i]) * mlp::gelu_grad(zr[2 * i]),
                                          __uint_as_float(v[2 * i + 1]) * mlp::gelu_grad(zr[2 * i + 1]));
                uint4 *dst = reinterpret_cast<uint4 *>(dz1 + g * mlp::kHid + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) dst[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
            }
        }
        tc_fence_before();
        __syncthreads();  // A is rewritten by the next tile
    }
    if (expired && tid == 0 && err) atomicOr(&err[0], kErrTimeout);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kHgTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradients of one chunk of 128 rows
// ---------------------------------------------------------------------------
constexpr uint32_t kWgOffA2 = 0;                        // dz2^T: 128 out x 128 rows
constexpr uint32_t kWgOffB2 = kWgOffA2 + 128 * 128 * 2;  // a1^T: 128 in x 128 rows
constexpr uint32_t kWgOffA1 = kWgOffB2 + 128 * 128 * 2;  // dz1^T: 128 out x 128 rows
constexpr uint32_t kWgOffB1 = kWgOffA1 + 128 * 128 * 2;  // x0^T: 64 in x 128 rows
constexpr uint32_t kWgOffRed = kWgOffB1 + 64 * 128 * 2;  // [kGThreads] floats
constexpr uint32_t kWgOffBar = kWgOffRed + kGThreads * 4;
constexpr uint32_t kWgOffTmem = kWgOffBar + 8;
constexpr uint32_t kWgSmem = kWgOffTmem + 8;
constexpr uint32_t kWgTmemCols = 256;  // dW2 in columns 0..127, dW1 in 128..191
static_assert(kWgOffBar % 8 == 0, "mbarrier alignment");

// Element (r, k) of a K-major operand with K = 128 (here k is the chunk row).
__device__ __forceinline__ uint32_t cm_elem(int r, int k) { return cm_off(r, k >> 3, 128) + (k & 7) * 2; }

__global__ void __launch_bounds__(kGThreads, 1)
    k_weight_grad_tc(int64_t B, const __nv_bfloat16 *__restrict__ x0s, const __nv_bfloat16 *__restrict__ a1s,
                     const __nv_bfloat16 *__restrict__ a2s, const __nv_bfloat16 *__restrict__ dz1,
                     const __nv_bfloat16 *__restrict__ dz2, const float *__restrict__ dout,
                     const float *__restrict__ row_loss, float *partial, int32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kGRows;
    const int n = (int)min((int64_t)kGRows, B - base);
    const uint32_t bar = smem_u32(smem + kWgOffBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kWgOffTmem);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    // transposed staging: consecutive threads read consecutive columns of a row (coalesced)
    for (int i = tid; i < kGRows * mlp::kHid; i += kGThreads) {
        const int r = i >> 7, c = i & 127;
        const bool ok = r < n;
        const int64_t src = (base + r) * mlp::kHid + c;
        const uint32_t off = cm_elem(c, r);
        *reinterpret_cast<__nv_bfloat16 *>(smem + kWgOffA2 + off) = ok ? dz2[src] : zero;
        *reinterpret_cast<__nv_bfloat16 *>(smem + kWgOffB2 + off) = ok ? a1s[src] : zero;
        *reinterpret_cast<__nv_bfloat16 *>(smem + kWgOffA1 + off) = ok ? dz1[src] : zero;
    }
    for (int i = tid; i < kGRows * mlp::kInPad; i += kGThreads) {
        const int r = i >> 6, c = i & 63;
        *reinterpret_cast<__nv_bfloat16 *>(smem + kWgOffB1 + cm_elem(c, r)) =
            r < n ? x0s[(base + r) * mlp::kInPad + c] : zero;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kWgTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sbase = smem_u32(smem);
    if (tid == 0) {
        tc_fence_after();
        const uint32_t id2 = idesc_bf16(128, 128), id1 = idesc_bf16(128, 64);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            umma(tmem, sdesc(sbase + kWgOffA2 + 256 * k, 128, 2048), sdesc(sbase + kWgOffB2 + 256 * k, 128, 2048), id2,
                 k > 0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            umma(tmem + 128, sdesc(sbase + kWgOffA1 + 256 * k, 128, 2048), sdesc(sbase + kWgOffB1 + 256 * k, 128, 2048),
                 id1, k > 0);
        umma_commit(bar);
    }
    float *pg = partial + (int64_t)blockIdx.x * (mlp::kParams + 1);
    // meanwhile, on the CUDA cores: dW3 [4][128] = d_out^T a2, the bias sums, b3 (rows in order)
    for (int j = tid; j < mlp::kOut * mlp::kHid; j += kGThreads) {
        const int o = j / mlp::kHid, in = j % mlp::kHid;
        float s = 0.0f;
        for (int r = 0; r < n; ++r)
            s = fmaf(dout[(base + r) * mlp::kOut + o], __bfloat162float(a2s[(base + r) * mlp::kHid + in]), s);
        pg[mlp::kOffW3 + j] = s;
    }
    for (int j = tid; j < mlp::kHid; j += kGThreads) {
        float s1 = 0.0f, s2 = 0.0f;
        for (int r = 0; r < n; ++r) {
            s1 += __bfloat162float(dz1[(base + r) * mlp::kHid + j]);
            s2 += __bfloat162float(dz2[(base + r) * mlp::kHid + j]);
        }
        pg[mlp::kOffB1 + j] = s1;
        pg[mlp::kOffB2 + j] = s2;
    }
    if (tid < mlp::kOut) {
        float s = 0.0f;
        for (int r = 0; r < n; ++r) s += dout[(base + r) * mlp::kOut + tid];
        pg[mlp::kOffB3 + tid] = s;
    }
    float *red = reinterpret_cast<float *>(smem + kWgOffRed);
    float l = 0.0f;
    for (int r = tid; r < n; r += kGThreads) l += row_loss[base + r];
    red[tid] = l;
    const bool ok = mbar_wait_bounded(bar, 0);
    const bool expired = __syncthreads_or(!ok);
    if (tid == 0) {
        float s = 0.0f;
        for (int i = 0; i < kGThreads; ++i) s += red[i];
        pg[mlp::kParams] = s;
    }
    if (!expired) {
        tc_fence_after();
        // TMEM lane o = output neuron o; the two warpgroups take halves of the columns
        const int o = tid & 127, half = tid >> 7;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
        for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(lane_base + c0, v);
            tc_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) pg[mlp::kOffW2 + o * mlp::kHid + c0 + i] = __uint_as_float(v[i]);
        }
        {
            uint32_t v[32];
            tmem_ld32(lane_base + 128 + 32 * half, v);
            tc_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int in = 32 * half + i;
                if (in < mlp::kIn) pg[mlp::kOffW1 + o * mlp::kIn + in] = __uint_as_float(v[i]);
            }
        }
    } else if (tid == 0 && err) {
        atomicOr(&err[0], kErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmemCols)
                     : "memory");
    }
}

cudaError_t grad_attrs()
{
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        e = cudaFuncSetAttribute(k_hidden_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHgSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_weight_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    });
    return e;
}

}  // namespace tc

cudaError_t launch_hidden_grad_tc(int64_t B, const __nv_bfloat16 *dz2, const __nv_bfloat16 *w2t, const float *z1,
                                  __nv_bfloat16 *dz1, int32_t *err, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const cudaError_t e = tc::grad_attrs();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n_tiles = (B + tc::kGRows - 1) / tc::kGRows;
    const int64_t grid = std::min<int64_t>(n_tiles, 2 * (int64_t)(sms > 0 ? sms : 1));
    tc::k_hidden_grad_tc<<<(unsigned)grid, tc::kGThreads, tc::kHgSmem, s>>>(B, dz2, w2t, z1, dz1, err);
    return cudaGetLastError();
}

cudaError_t launch_weight_grad_tc(int64_t B, const __nv_bfloat16 *x0s, const __nv_bfloat16 *a1s,
                                  const __nv_bfloat16 *a2s, const __nv_bfloat16 *dz1, const __nv_bfloat16 *dz2,
                                  const float *dout, const float *row_loss, float *partial, int32_t *err,
                                  cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const cudaError_t e = tc::grad_attrs();
    if (e != cudaSuccess) return e;
    const int64_t chunks = (B + tc::kGRows - 1) / tc::kGRows;
    tc::k_weight_grad_tc<<<(unsigned)chunks, tc::kGThreads, tc::kWgSmem, s>>>(B, x0s, a1s, a2s, dz1, dz2, dout,
                                                                            row_loss, partial, err);
    return cudaGetLastError();
}

}  // namespace pf
