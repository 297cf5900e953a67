// k_proposal_tc.cu -- the learned proposal's network forward on the
// fifth-generation tensor cores, fused with the construction of its input
// rows from the lattice state.
//
// One CTA of 512 threads per SM, persistent over tiles of 128 network rows
// (one row per (particle, observed node)), with four independent slots: each
// warpgroup of 128 threads carries its own tile through the three layers,
// with its own 128 TMEM columns (the four slots take all 512), its own 32 KB
// operand buffer and mbarrier, and named barrier 1 + slot, so a slot's
// epilogue runs while the others' MMAs do; the weights are staged once for
// all four.  Thread t works on row t % 128 of slot t / 128.  Per tile:
//   rows     every thread gathers its row (columns 0..31: the v patch and the
//            first w values; 32..63: the rest of the w patch and y; 5x5
//            patches mirrored at the edges) from the particle's state, rounds
//            it to BF16 and stores it as the A operand in the slot's buffer;
//   layer 1  the slot's first thread issues 4 tcgen05.mma (M 128, N 128,
//            K 16) into the slot's TMEM columns, commit -> mbarrier;
//   GELU     every thread loads its row of the accumulator (tcgen05.ld; warp
//            w reaches TMEM lanes 32 (w % 4) .. + 31), adds the bias, applies
//            GELU and stores BF16 as the next A operand over the first;
//   layer 2  8 MMAs into the same columns (every row of layer 1's read), GELU;
//   layer 3  8 MMAs with N 16 (W3 zero-padded from 4 to 16 rows) into
//            columns 0..15; every thread writes its row's 4 outputs + bias.
// Operands are K-major without swizzle: element (r, k) of a tile with K
// columns sits at (r / 8) (K / 8) 128 + (k / 8) 128 + (r % 8) 16 + (k % 8) 2
// bytes (8 x 16-byte core matrices; K-direction stride 128 B, row-group
// stride K * 16 B).  Every wait on the tensor cores is bounded (2 s by the
// global timer); on expiry the slot flags kErrTimeout in the context's error
// word and stops, and the CTA frees its TMEM once every slot has stopped.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lattice.cuh"
#include "mlp_device.cuh"
#include "pf.h"
#include "pf_internal.h"
#include "tc_device.cuh"

namespace pf {
namespace tc {

constexpr int kRows = 128;
constexpr int kSlots = 4;                     // tiles in flight per CTA, one warpgroup each
constexpr int kThreads = 128 * kSlots;        // a thread per row of its slot's tile
constexpr uint32_t kTmemCols = 128 * kSlots;  // 128 accumulator columns per slot: all 512 of the SM
constexpr uint32_t kOffW1 = 0;                          // 128 x 64
constexpr uint32_t kOffW2 = kOffW1 + 128 * 64 * 2;      // 128 x 128
constexpr uint32_t kOffW3 = kOffW2 + 128 * 128 * 2;     // 16 x 128
constexpr uint32_t kOffBuf = kOffW3 + 16 * 128 * 2;     // per slot: A (128 x 64), then H (128 x 128) over it
constexpr uint32_t kBufBytes = 128 * 128 * 2;
constexpr uint32_t kOffBias = kOffBuf + kSlots * kBufBytes;  // b1[128], b2[128], b3[4]
constexpr uint32_t kOffBar = kOffBias + (128 + 128 + 4) * 4; // an mbarrier per slot
constexpr uint32_t kOffTmem = kOffBar + 8 * kSlots;
constexpr uint32_t kSmemBytes = kOffTmem + 8;
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kOffBuf % 1024 == 0, "operand alignment");
static_assert(kSmemBytes <= 227 * 1024, "one CTA per SM");

// A slot's warpgroup synchronises on named barrier 1 + slot (barrier 0 is the
// CTA's); the OR form returns whether any of its threads passed `pred`.
__device__ __forceinline__ void slot_sync(int slot)
{
    asm volatile("bar.sync %0, 128;" ::"r"(1 + slot) : "memory");
}
__device__ __forceinline__ bool slot_any(int slot, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(1 + slot)
        : "memory");
    return r != 0;
}

// Bias + GELU on 32 accumulator columns [c0, c0 + 32) of row r, stored as BF16
// into the 128-wide A operand at `h`; with zs / as (training) also the
// pre-activations (FP32) and the BF16 activations of the row to global memory.
__device__ __forceinline__ void gelu_store(const uint32_t (&v)[32], const float *bias, int c0, int r, unsigned char *h,
                                           float *zs = nullptr, __nv_bfloat16 *as = nullptr)
{
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint32_t w[4];
        float z[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // two columns at once on the packed FP32 pipes
            const int c = g * 8 + 2 * i;
            const float2 zz = __fadd2_rn(make_float2(__uint_as_float(v[c]), __uint_as_float(v[c + 1])),
                                         make_float2(bias[c0 + c], bias[c0 + c + 1]));
            z[2 * i] = zz.x;
            z[2 * i + 1] = zz.y;
            const float2 gg = mlp::gelu_x2(zz);
            w[i] = mlp::pack_bf16(gg.x, gg.y);
        }
        *reinterpret_cast<uint4 *>(h + cm_off(r, (c0 >> 3) + g, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
        if (zs) {
            *reinterpret_cast<float4 *>(zs + c0 + g * 8) = make_float4(z[0], z[1], z[2], z[3]);
            *reinterpret_cast<float4 *>(zs + c0 + g * 8 + 4) = make_float4(z[4], z[5], z[6], z[7]);
            *reinterpret_cast<uint4 *>(as + c0 + g * 8) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Rows from an FP32 matrix (training, and the stateless forward) and, when x0 and
// z1 are given, the activations the backward pass needs.
struct TrainIO {
    const float *X;        // [R][51] input rows (null: rows from lattice states)
    int64_t R;
    __nv_bfloat16 *x0;     // [R][64] the BF16 input rows (zero-padded)
    float *z1, *z2;        // [R][128] pre-activations
    __nv_bfloat16 *a1, *a2;  // [R][128] BF16 activations
};

template <bool Train>
__global__ void __launch_bounds__(kThreads, 1)
    k_proposal_forward_tc(int32_t J, int32_t dx, int32_t dy, const float *__restrict__ x, int64_t P,
                          const int32_t *__restrict__ pfilt, const int32_t *__restrict__ obs_idx,
                          const float *__restrict__ obs, int32_t obs_stride, const __nv_bfloat16 *__restrict__ wp,
                          const float *__restrict__ theta, float *__restrict__ out, int32_t *err, TrainIO io)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, slot = tid >> 7, row = tid & (kRows - 1);
    const int64_t R = Train ? io.R : P * dy;
    const int64_t n_tiles = (R + kRows - 1) / kRows;
    float *bias = reinterpret_cast<float *>(smem + kOffBias);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffTmem);

    // weights (core-matrix layout) and biases, once per CTA for its four slots
    const uint4 *w1g = reinterpret_cast<const uint4 *>(wp);
    const uint4 *w2g = reinterpret_cast<const uint4 *>(wp + mlp::kPackW1);
    const uint4 *w3g = reinterpret_cast<const uint4 *>(wp + mlp::kPackW1 + mlp::kPackW2);
    for (int i = tid; i < 128 * 8; i += kThreads) {  // W1: 128 rows x 8 groups of 8
        const int n = i >> 3, g = i & 7;
        *reinterpret_cast<uint4 *>(smem + kOffW1 + cm_off(n, g, 64)) = w1g[n * 8 + g];
    }
    for (int i = tid; i < 128 * 16; i += kThreads) {  // W2: 128 rows x 16 groups
        const int n = i >> 4, g = i & 15;
        *reinterpret_cast<uint4 *>(smem + kOffW2 + cm_off(n, g, 128)) = w2g[n * 16 + g];
    }
    for (int i = tid; i < 16 * 16; i += kThreads) {  // W3: 8 packed rows, rows 8..15 zero
        const int n = i >> 4, g = i & 15;
        *reinterpret_cast<uint4 *>(smem + kOffW3 + cm_off(n, g, 128)) =
            n < mlp::kOutPad ? w3g[n * 16 + g] : make_uint4(0u, 0u, 0u, 0u);
    }
    for (int i = tid; i < 128; i += kThreads) {
        bias[i] = theta[mlp::kOffB1 + i];
        bias[128 + i] = theta[mlp::kOffB2 + i];
    }
    if (tid < 4) bias[256 + tid] = theta[mlp::kOffB3 + tid];
    if (tid < kSlots) mbar_init(smem_u32(smem + kOffBar + 8 * tid), 1);
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the slot's accumulator columns; warp w reaches TMEM lanes 32 (w % 4) .. + 31 (its rows)
    const uint32_t dcol = tmem + 128u * (uint32_t)slot;
    const uint32_t lane_base = dcol + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t bar = smem_u32(smem + kOffBar + 8 * slot);
    unsigned char *buf = smem + kOffBuf + (uint32_t)slot * kBufBytes;

    const uint32_t sbase = smem_u32(smem), sbuf = sbase + kOffBuf + (uint32_t)slot * kBufBytes;
    const uint32_t id128 = idesc_bf16(128, 128), id16 = idesc_bf16(128, 16);
    uint32_t phase = 0;
    bool expired = false;
    const int nn = J * J;
    // slot-major: with fewer tiles than SMs each CTA's first slot takes one, spread over the SMs
    for (int64_t tile = (int64_t)slot * gridDim.x + blockIdx.x; tile < n_tiles; tile += (int64_t)gridDim.x * kSlots) {
        const int64_t g = tile * kRows + row;
        // ---- the input row -> A (columns 0..31, then 32..63)
        const int64_t p = (!Train && g < R) ? g / dy : 0;
        const int j = (!Train && g < R) ? (int)(g - p * dy) : 0;
        const int nd = (!Train && g < R) ? obs_idx[j] : 0, ri = nd / J, ci = nd - ri * J;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) w[i] = 0u;
            if (Train && g < R) {  // an FP32 row of 51 inputs, zero-padded to 64
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = 32 * half + 2 * q;
                    w[q] = mlp::pack_bf16(c < mlp::kIn ? io.X[g * mlp::kIn + c] : 0.0f,
                                          c + 1 < mlp::kIn ? io.X[g * mlp::kIn + c + 1] : 0.0f);
                }
                if (io.x0)
#pragma unroll
                    for (int kg = 0; kg < 4; ++kg)
                        reinterpret_cast<uint4 *>(io.x0 + g * mlp::kInPad + 32 * half)[kg] =
                            make_uint4(w[4 * kg], w[4 * kg + 1], w[4 * kg + 2], w[4 * kg + 3]);
            } else if (!Train && g < R) {
                const float *xp = x + p * (int64_t)dx;
                float vals[32];
                if (half == 0) {  // v patch (25) and w patch elements 0..6
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int e = q < 25 ? q : q - 25;
                        const int k = mirror_index(ri + e / 5 - 2, J) * J + mirror_index(ci + e % 5 - 2, J);
                        vals[q] = xp[(q < 25 ? 0 : nn) + k];
                    }
                } else {  // w patch elements 7..24, y, zeros
#pragma unroll
                    for (int q = 0; q < 18; ++q) {
                        const int e = q + 7;
                        const int k = mirror_index(ri + e / 5 - 2, J) * J + mirror_index(ci + e % 5 - 2, J);
                        vals[q] = xp[nn + k];
                    }
                    vals[18] = obs[(obs_stride ? (int64_t)pfilt[p] * obs_stride : 0) + j];
#pragma unroll
                    for (int q = 19; q < 32; ++q) vals[q] = 0.0f;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) w[i] = mlp::pack_bf16(vals[2 * i], vals[2 * i + 1]);
            }
#pragma unroll
            for (int kg = 0; kg < 4; ++kg)
                *reinterpret_cast<uint4 *>(buf + cm_off(row, 4 * half + kg, 64)) =
                    make_uint4(w[4 * kg], w[4 * kg + 1], w[4 * kg + 2], w[4 * kg + 3]);
        }
        fence_proxy_async();
        tc_fence_before();
        slot_sync(slot);
        // ---- layer 1
        if (row == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                umma(dcol, sdesc(sbuf + 256 * k, 128, 1024), sdesc(sbase + kOffW1 + 256 * k, 128, 1024), id128, k > 0);
            umma_commit(bar);
        }
        bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (slot_any(slot, !ok)) { expired = true; break; }
        tc_fence_after();
        const bool save = Train && io.z1 && g < R;
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {  // H over A: layer 1's MMAs have read it
            uint32_t v[32];
            tmem_ld32(lane_base + c0, v);
            tc_wait_ld();
            gelu_store(v, bias, c0, row, buf, save ? io.z1 + g * mlp::kHid : nullptr,
                       save ? io.a1 + g * mlp::kHid : nullptr);
        }
        fence_proxy_async();
        tc_fence_before();
        slot_sync(slot);
        // ---- layer 2 (into the same columns: every thread has read layer 1's)
        if (row == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 8; ++k)
                umma(dcol, sdesc(sbuf + 256 * k, 128, 2048), sdesc(sbase + kOffW2 + 256 * k, 128, 2048), id128, k > 0);
            umma_commit(bar);
        }
        ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (slot_any(slot, !ok)) { expired = true; break; }
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {  // H again: layer 2's MMAs have read it
            uint32_t v[32];
            tmem_ld32(lane_base + c0, v);
            tc_wait_ld();
            gelu_store(v, bias + 128, c0, row, buf, save ? io.z2 + g * mlp::kHid : nullptr,
                       save ? io.a2 + g * mlp::kHid : nullptr);
        }
        fence_proxy_async();
        tc_fence_before();
        slot_sync(slot);
        // ---- layer 3 (N = 16; rows 4..15 of W3 are zero)
        if (row == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 8; ++k)
                umma(dcol, sdesc(sbuf + 256 * k, 128, 2048), sdesc(sbase + kOffW3 + 256 * k, 128, 2048), id16, k > 0);
            umma_commit(bar);
        }
        ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (slot_any(slot, !ok)) { expired = true; break; }
        tc_fence_after();
        {
            uint32_t v[4];
            tmem_ld4(lane_base, v);
            tc_wait_ld();
            if (g < R)
                reinterpret_cast<float4 *>(out)[g] =
                    make_float4(__uint_as_float(v[0]) + bias[256], __uint_as_float(v[1]) + bias[257],
                                __uint_as_float(v[2]) + bias[258], __uint_as_float(v[3]) + bias[259]);
        }
        tc_fence_before();
        slot_sync(slot);  // every row's output read before the next tile's layer 1 overwrites the columns
    }
    // a wait that expired: report it (the slot's threads left its loop together)
    if (expired && row == 0 && err) atomicOr(&err[0], kErrTimeout);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// The forward kernels' shared-memory size, set once per process.
cudaError_t forward_attrs()
{
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_proposal_forward_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(k_proposal_forward_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSmemBytes);
    });
    return attr_err;
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

}  // namespace tc

cudaError_t launch_proposal_forward_tc(int32_t J, int32_t dx, int32_t dy, const float *x, int64_t P,
                                       const int32_t *pfilt, const int32_t *obs_idx, const float *obs,
                                       int32_t obs_stride, const __nv_bfloat16 *wp, const float *theta, float *out,
                                       int32_t *err, cudaStream_t s)
{
    const int64_t R = P * dy;
    if (R <= 0) return cudaSuccess;
    const cudaError_t attr_err = tc::forward_attrs();
    if (attr_err != cudaSuccess) return attr_err;
    const int64_t n_tiles = (R + tc::kRows - 1) / tc::kRows;
    const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)tc::sm_count());
    tc::k_proposal_forward_tc<false><<<(unsigned)grid, tc::kThreads, tc::kSmemBytes, s>>>(
        J, dx, dy, x, P, pfilt, obs_idx, obs, obs_stride, wp, theta, out, err, tc::TrainIO{});
    return cudaGetLastError();
}

// The forward on FP32 input rows X [R][51] -> outputs [R][4] (training, and the
// stateless forward), with the BF16 inputs, the pre-activations and the BF16
// activations saved for the backward pass when x0 and z1 are given -- the same
// tensor-core kernel as the filter's forward.
cudaError_t launch_train_forward_tc(const float *X, int64_t R, const __nv_bfloat16 *wp, const float *theta, float *out,
                                    __nv_bfloat16 *x0, float *z1, __nv_bfloat16 *a1, float *z2, __nv_bfloat16 *a2,
                                    int32_t *err, cudaStream_t s)
{
    if (R <= 0) return cudaSuccess;
    const cudaError_t e = tc::forward_attrs();
    if (e != cudaSuccess) return e;
    const int64_t n_tiles = (R + tc::kRows - 1) / tc::kRows;
    const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)tc::sm_count());
    tc::k_proposal_forward_tc<true><<<(unsigned)grid, tc::kThreads, tc::kSmemBytes, s>>>(
        2, 8, 1, nullptr, 0, nullptr, nullptr, nullptr, 0, wp, theta, out, err, tc::TrainIO{X, R, x0, z1, z2, a1, a2});
    return cudaGetLastError();
}

}  // namespace pf

extern "C" {

pf_status pf_proposal_forward(int32_t J, int64_t P, const float *d_x, int32_t dy, const int32_t *h_obs_idx,
                              const float *d_y, const float *d_theta, float *d_out, void *stream)
{
    if (J < 2 || J > 44 || P < 0 || dy < 1 || !h_obs_idx) return PF_EINVAL;
    if (P > 0 && (!d_x || !d_y || !d_theta || !d_out)) return PF_EINVAL;
    if (((uintptr_t)d_out & 15u) != 0) return PF_EINVAL;  // float4 rows
    for (int j = 0; j < dy; ++j)
        if (h_obs_idx[j] < 0 || h_obs_idx[j] >= J * J) return PF_EINVAL;
    if (P == 0) return PF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16 *wp = nullptr;
    int32_t *idx = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&wp, (pf::mlp::kPackTotal + pf::mlp::kHid * pf::mlp::kHid) * 2, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&idx, (size_t)dy * sizeof(int32_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (wp) cudaFreeAsync(wp, s);
        return PF_ENOMEM;
    }
    e = cudaMemcpyAsync(idx, h_obs_idx, (size_t)dy * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = pf::launch_mlp_pack(d_theta, wp, wp + pf::mlp::kPackTotal, s);
    if (e == cudaSuccess)
        e = pf::launch_proposal_forward_tc(J, 2 * J * J, dy, d_x, P, nullptr, idx, d_y, 0, wp, d_theta, d_out,
                                           nullptr, s);
    cudaFreeAsync(idx, s);
    cudaFreeAsync(wp, s);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

}  // extern "C"
