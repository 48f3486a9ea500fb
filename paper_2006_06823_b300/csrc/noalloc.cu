// lddmm_bl_project_noalloc: the band-limited projection for callers that cannot allocate
// device memory.
//
// The regular lddmm_bl_project takes its scratch (twiddle tables and the two stage
// buffers of the separable partial DFT) from CUDA's stream-ordered pool on every call.
// Some callers cannot let a library allocate: a host framework that owns all device
// memory through its own pool and forbids allocations behind its back, a service that
// must stay inside a memory budget reserved up front, or a latency-critical loop that
// cannot afford the allocator. This variant instead uses one file-scope device array of
// fixed size (kScratchBytes below), which every GPU that loads the library holds until
// the process exits. It computes exactly what lddmm_bl_project computes, with the same
// kernels.
#include "common.cuh"
#include "lddmm.h"

#include <mutex>
#include <string>

namespace lddmm {
namespace {

constexpr size_t kScratchBytes = size_t(24) << 20;  // 24 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device. The host-side symbol g_scratch is
// only a stand-in; the address must come from cudaGetSymbolAddress, taken once per device
// with that device current.
int scratch_address(void** out) {
    int dev = -1;
    LDDMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("bl_project_noalloc: device index out of range");
        return LDDMM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("bl_project_noalloc: cudaGetSymbolAddress: ") +
                      cudaGetErrorString(e));
            return LDDMM_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LDDMM_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace lddmm

using namespace lddmm;

extern "C" int lddmm_bl_project_noalloc(int nx, int ny, int nz, int K, const float* f, int ncomp,
                                        float* c, int precision, void* stream) {
    // the checks of lddmm_bl_project itself, so that both accept the same arguments
    int rc = check_grid(nx, ny, nz);
    if (rc) return rc;
    rc = check_band(nx, ny, nz, K);
    if (rc) return rc;
    rc = check_spectral_precision(precision);
    if (rc) return rc;
    if (!f || !c || ncomp < 1) {
        set_error("bl_project_noalloc: null pointer or ncomp < 1");
        return LDDMM_EINVAL;
    }
    const Grid g{nx, ny, nz};
    const long kh = K / 2;
    // stage X output and z-block partials share s1; stage Y output in s2
    const size_t tw_bytes = round256((size_t)twiddle_floats(g, K) * sizeof(float));
    const size_t s1_bytes = round256((size_t)ncomp * nz * (ny > K ? ny : K) * kh * sizeof(float2));
    const size_t s2_bytes = round256((size_t)ncomp * nz * K * kh * sizeof(float2));
    const size_t need = tw_bytes + s1_bytes + s2_bytes;
    if (need > kScratchBytes) {
        set_error("bl_project_noalloc: needs " + std::to_string(need) +
                  " bytes of scratch, more than its fixed " + std::to_string(kScratchBytes) +
                  " (about ncomp * nz * max(ny, K) * K * 4 bytes); use lddmm_bl_project");
        return LDDMM_EINVAL;
    }
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* p = static_cast<unsigned char*>(base);
    float* twm = reinterpret_cast<float*>(p);
    float2* s1 = reinterpret_cast<float2*>(p + tw_bytes);
    float2* s2 = reinterpret_cast<float2*>(p + tw_bytes + s1_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Twiddles tw;
    rc = twiddle_init(g, K, twm, tw, st);
    if (rc) return rc;
    return bl_project(g, tw, f, g.ntot(), ncomp, reinterpret_cast<float2*>(c), s1, s2, precision,
                      st);
}
