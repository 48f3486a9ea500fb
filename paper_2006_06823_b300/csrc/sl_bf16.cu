// BF16-storage form of the scalar SL transport D_t m = 0 (Table 1 row 1; Sec. 3.1, Eqs. 40-43),
// the mixed-precision variant of the state sweep: the departure offsets are computed in FP32
// as in lddmm_sl_transport, then optionally stored in BF16, and the transported field is kept
// in BF16 between steps; every interpolation is evaluated in FP32 (taps widened on load). The
// first step reads the FP32 input field and the last one writes the FP32 result. Bytes per
// voxel-step: 12 (FP32 offsets) or 6 (BF16) + 2 (tap) + 2 (store), against 20 for FP32 storage.
#include "common.cuh"
#include "lddmm.h"

#include <cuda_bf16.h>

#include <string>

namespace lddmm {
namespace {

__device__ __forceinline__ float clampD(float d) { return fminf(fmaxf(d, -1048576.f), 1048576.f); }

__device__ __forceinline__ int wrapi(int i, int n) {
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
}

__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldo(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ldo(const __nv_bfloat16* p) {
    return __bfloat162float(__ldcs(reinterpret_cast<const __nv_bfloat16*>(p)));
}
__device__ __forceinline__ void st(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// trilinear interpolation at (x, y, z) + (dx, dy, dz), periodic; the single-pair kernels' cell
// and weights, FP32 arithmetic on widened taps
template <typename TF>
__device__ __forceinline__ float lin_at(const TF* f, int nx, int ny, int nz, int x, int y, int z,
                                        float dx, float dy, float dz) {
    auto axis = [](int j, float D, int n, int mul, int& a0, int& a1, float& t) {
        D = clampD(D);
        const float fl = floorf(D);
        t = D - fl;
        const int i = wrapi(j + (int)fl, n);
        const int i1 = i + 1 == n ? 0 : i + 1;
        a0 = i * mul;
        a1 = i1 * mul;
    };
    int x0, x1, y0, y1, z0, z1;
    float tx, ty, tz;
    axis(x, dx, nx, 1, x0, x1, tx);
    axis(y, dy, ny, nx, y0, y1, ty);
    axis(z, dz, nz, nx * ny, z0, z1, tz);
    const float v000 = ld(f + z0 + y0 + x0), v001 = ld(f + z0 + y0 + x1);
    const float v010 = ld(f + z0 + y1 + x0), v011 = ld(f + z0 + y1 + x1);
    const float v100 = ld(f + z1 + y0 + x0), v101 = ld(f + z1 + y0 + x1);
    const float v110 = ld(f + z1 + y1 + x0), v111 = ld(f + z1 + y1 + x1);
    const float a00 = fmaf(tx, v001 - v000, v000), a01 = fmaf(tx, v011 - v010, v010);
    const float a10 = fmaf(tx, v101 - v100, v100), a11 = fmaf(tx, v111 - v110, v110);
    const float b0 = fmaf(ty, a01 - a00, a00), b1 = fmaf(ty, a11 - a10, a10);
    return fmaf(tz, b1 - b0, b0);
}

// departure offsets D = dt/2 (v(X*) + v(x)), X* = x + dts v(x), stored as TD
template <typename TD>
__global__ void __launch_bounds__(256)
k_char_store(Grid g, const float* __restrict__ vel, float dts, TD* __restrict__ D) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();
    const int i = (z * g.ny + y) * g.nx + x;
    const float V0 = __ldcs(vel + i), V1 = __ldcs(vel + n + i), V2 = __ldcs(vel + 2 * n + i);
    const float W0 = lin_at(vel, g.nx, g.ny, g.nz, x, y, z, dts * V0, dts * V1, dts * V2);
    const float W1 = lin_at(vel + n, g.nx, g.ny, g.nz, x, y, z, dts * V0, dts * V1, dts * V2);
    const float W2 = lin_at(vel + 2 * n, g.nx, g.ny, g.nz, x, y, z, dts * V0, dts * V1, dts * V2);
    const float h = 0.5f * dts;
    st(D + i, h * (W0 + V0));
    st(D + n + i, h * (W1 + V1));
    st(D + 2 * n + i, h * (W2 + V2));
}

// one step out = src o (x + D) over zt consecutive z planes per thread (the offsets of plane
// z + 1 are loaded while the taps of plane z are in flight)
template <typename TS, typename TD, typename TO>
__global__ void __launch_bounds__(256, 5)
k_gather_mixed(Grid g, const TS* __restrict__ src, const TD* __restrict__ D, TO* __restrict__ out,
               int zt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();
    const int plane = g.nx * g.ny;
    int z = blockIdx.z * zt;
    const int zend = min(z + zt, g.nz);
    if (z >= zend) return;
    int i = (z * g.ny + y) * g.nx + x;
    float d0 = ldo(D + i), d1 = ldo(D + n + i), d2 = ldo(D + 2 * n + i);
    for (;;) {
        const bool more = z + 1 < zend;
        const int ip = more ? i + plane : i;
        const float e0 = ldo(D + ip), e1 = ldo(D + n + ip), e2 = ldo(D + 2 * n + ip);
        st(out + i, lin_at(src, g.nx, g.ny, g.nz, x, y, z, d0, d1, d2));
        if (!more) break;
        ++z;
        i = ip;
        d0 = e0; d1 = e1; d2 = e2;
    }
}

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

template <typename TD>
int run(const Grid& g, int nt, const float* vel, const float* field, float dts, float* out,
        void* scratch, cudaStream_t st) {
    const long n = g.ntot();
    TD* D = static_cast<TD*>(scratch);
    __nv_bfloat16* b0 = reinterpret_cast<__nv_bfloat16*>(D + 3 * n);
    __nv_bfloat16* b1 = b0 + n;
    const dim3 blk(32, 8, 1);
    const int zt = 4;
    const dim3 grid(cdiv(g.nx, 32), cdiv(g.ny, 8), cdiv(g.nz, zt));
    const double dbytes = sizeof(TD) == 2 ? 6.0 : 12.0;
    {
        KTRACE(sizeof(TD) == 2 ? "sl_char_bf16" : "sl_char", st, (24.0 + dbytes) * n, 0);
        k_char_store<TD><<<dim3(cdiv(g.nx, 32), cdiv(g.ny, 8), g.nz), blk, 0, st>>>(g, vel, dts, D);
    }
    LDDMM_CHECK_LAUNCH();
    for (int j = 0; j < nt; ++j) {
        const bool first = j == 0, last = j == nt - 1;
        __nv_bfloat16* dst16 = (j & 1) ? b1 : b0;
        const __nv_bfloat16* src16 = (j & 1) ? b0 : b1;
        KTRACE("sl_gather_bf16", st, (dbytes + (first ? 4.0 : 2.0) + (last ? 4.0 : 2.0)) * n, 0);
        if (first && last)
            k_gather_mixed<float, TD, float><<<grid, blk, 0, st>>>(g, field, D, out, zt);
        else if (first)
            k_gather_mixed<float, TD, __nv_bfloat16><<<grid, blk, 0, st>>>(g, field, D, dst16, zt);
        else if (last)
            k_gather_mixed<__nv_bfloat16, TD, float><<<grid, blk, 0, st>>>(g, src16, D, out, zt);
        else
            k_gather_mixed<__nv_bfloat16, TD, __nv_bfloat16><<<grid, blk, 0, st>>>(g, src16, D, dst16, zt);
        LDDMM_CHECK_LAUNCH();
    }
    return LDDMM_OK;
}

}  // namespace
}  // namespace lddmm

using namespace lddmm;

extern "C" int lddmm_sl_transport_bf16(int nx, int ny, int nz, int nt, const float* vel,
                                       const float* field, int direction, int offsets_bf16,
                                       float* out, void* stream) {
    int rc = check_grid(nx, ny, nz);
    if (rc) return rc;
    if (!vel || !field || !out) {
        set_error("sl_transport_bf16: null pointer");
        return LDDMM_EINVAL;
    }
    if (nt < 1) { set_error("sl_transport_bf16: nt must be >= 1"); return LDDMM_EINVAL; }
    if (direction != 1 && direction != -1) {
        set_error("sl_transport_bf16: direction must be +1 or -1");
        return LDDMM_EINVAL;
    }
    if (offsets_bf16 != 0 && offsets_bf16 != 1) {
        set_error("sl_transport_bf16: offsets_bf16 must be 0 or 1");
        return LDDMM_EINVAL;
    }
    if (field == out) {
        set_error("sl_transport_bf16: field and out must not be the same buffer");
        return LDDMM_EINVAL;
    }
    const Grid g{nx, ny, nz};
    const long n = g.ntot();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // scratch: offsets (3 planes, FP32 or BF16) and two BF16 field planes, stream-ordered pool
    const size_t bytes = (size_t)n * (offsets_bf16 ? 6 : 12) + (size_t)n * 4 + 256;
    void* scratch = nullptr;
    LDDMM_CUDA(cudaMallocAsync(&scratch, bytes, st));
    const double dt = 1.0 / nt;
    const float dts = (float)(direction > 0 ? -dt : dt);
    rc = offsets_bf16 ? run<__nv_bfloat16>(g, nt, vel, field, dts, out, scratch, st)
                      : run<float>(g, nt, vel, field, dts, out, scratch, st);
    cudaFreeAsync(scratch, st);
    return rc;
}
