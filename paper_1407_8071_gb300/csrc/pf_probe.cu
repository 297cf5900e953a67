// pf_probe.cu -- a self-test of the failure detection of bounded device waits.
//
// The tensor-core kernels wait on mbarriers that the tensor cores complete;
// each wait is bounded by the global timer and, when it runs out, sets an
// error word that the host reports as PF_ETIMEOUT.  pf_probe_bounded_wait
// runs the same bounded wait (a 20 ms limit instead of 2 s) on a barrier of
// its own with no other work in flight: completed first, the wait succeeds;
// left incomplete, only its limit ends it.  One thread, one CTA.
#include <cstdint>

#include "pf.h"
#include "pf_internal.h"
#include "tc_device.cuh"

namespace {

constexpr uint64_t kProbeLimitNs = 20000000ull;  // 20 ms

__device__ int32_t g_probe_err;

__global__ void k_probe_wait(int32_t arrive)
{
    __shared__ __align__(8) uint64_t bar_word;
    const uint32_t bar = pf::tc::smem_u32(&bar_word);
    pf::tc::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
    if (!pf::tc::mbar_wait_bounded<kProbeLimitNs>(bar, 0)) atomicOr(&g_probe_err, pf::kErrTimeout);
}

}  // namespace

extern "C" {

pf_status pf_probe_bounded_wait(int32_t arrive, void *stream)
{
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t zero = 0;
    int32_t word = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_probe_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_probe_wait<<<1, 1, 0, s>>>(arrive ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&word, g_probe_err, sizeof word, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        pf::set_global_error((std::string("pf_probe_bounded_wait: ") + cudaGetErrorString(e)).c_str());
        return PF_ECUDA;
    }
    if (word & pf::kErrTimeout) {
        pf::set_global_error("pf_probe_bounded_wait: the bounded device wait gave up after its 20 ms limit");
        return PF_ETIMEOUT;
    }
    return PF_OK;
}

}  // extern "C"
