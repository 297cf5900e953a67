// pf_noalloc.cu -- systematic resampling without any allocation.
//
// Some callers cannot allocate device memory at the moment they need to
// resample: applications whose host framework owns every device allocation
// and forbids others, and real-time loops with a fixed memory budget, where
// an allocation could fail or stall.  For them
// pf_systematic_resample_noalloc takes its scratch from one file-scope device
// array instead of from the caller or from cudaMalloc.
#include <cstdint>

#include "pf.h"
#include "pf_internal.h"

namespace {

constexpr int32_t kNoallocMaxFilters = PF_NOALLOC_MAX_FILTERS;
constexpr int64_t kNoallocMaxParticles = PF_NOALLOC_MAX_PARTICLES;

// Scratch of pf_systematic_resample for the largest problem accepted
// (about 3.3 MB; every GPU that loads the library holds it until exit):
// tile plan, per-tile and per-filter sums, the 64-bit prefix, the
// ancestor markers and each tile's first ancestor.
constexpr size_t kTilesMax = kNoallocMaxFilters + kNoallocMaxParticles / pf::kTile + 1;
constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kScratchBytes =
    a256(kTilesMax * sizeof(pf::TileDesc)) + a256(kNoallocMaxFilters * sizeof(pf::FilterDesc)) +
    a256(kTilesMax * pf::kTsCount * sizeof(double)) +
    a256(kTilesMax * sizeof(uint64_t)) + a256(kNoallocMaxFilters * pf::kFsCount * sizeof(double)) +
    a256(kNoallocMaxFilters * 2 * sizeof(uint64_t)) + a256(kNoallocMaxParticles * sizeof(uint64_t)) +
    a256(kNoallocMaxParticles * sizeof(int32_t)) + a256(2 * sizeof(int32_t)) + a256(kTilesMax * sizeof(int32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with that device current.  It is looked up on every
// call (cheap once the module is loaded, and it allocates nothing), so the
// address stays right across devices and after a cudaDeviceReset.
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" {

pf_status pf_systematic_resample_noalloc(int32_t M, const int32_t *h_N, const double *d_w, const double *d_u,
                                         int32_t *d_anc, void *stream)
{
    if (M < 1 || !h_N || !d_w || !d_u || !d_anc) return PF_EINVAL;
    int64_t total = 0;
    for (int32_t m = 0; m < M; ++m) {
        if (h_N[m] < 1) return PF_EINVAL;
        total += h_N[m];
    }
    if (M > kNoallocMaxFilters || total > kNoallocMaxParticles) {
        pf::set_global_error("pf_systematic_resample_noalloc: at most PF_NOALLOC_MAX_FILTERS filters and "
                             "PF_NOALLOC_MAX_PARTICLES particles in all");
        return PF_EINVAL;
    }
    void *scratch = nullptr;
    const cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        pf::set_global_error("pf_systematic_resample_noalloc: cudaGetSymbolAddress failed");
        return PF_ECUDA;
    }
    return pf_systematic_resample(M, h_N, d_w, d_u, d_anc, scratch, kScratchBytes, stream);
}

}  // extern "C"
