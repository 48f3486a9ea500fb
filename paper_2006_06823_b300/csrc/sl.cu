// Semi-Lagrangian kernels (Sec. 3): departure points (Eqs. 40-42), transport along them
// with trilinear or cubic B-spline interpolation, the Heun (SL-RK) step forms of Table 1,
// the warped source image with its gradient, and the periodic B-spline prefilter.
//
// Offsets D = X - x are stored per voxel in voxels (three planes). A query point is the
// grid index j plus D; the cell is j + floor(D) and the fraction D - floor(D), which keeps
// the fraction at the precision of the (small) offset. Indices wrap periodically. Offsets
// are clamped to +-2^20 voxels before use, so non-finite or huge inputs can never address
// memory outside the field.
#include "common.cuh"

#include <cuda_bf16.h>
#include "lddmm.h"

namespace lddmm {

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ float clampD(float d) { return fminf(fmaxf(d, -1048576.f), 1048576.f); }

__device__ __forceinline__ int wrapi(int i, int n) {
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
}

// Trilinear cell: corner offsets and fractions.
struct LinCell {
    int x0, x1, y0, y1, z0, z1;   // offsets within one component (< 2^31 voxels)
    float tx, ty, tz;
};

__device__ __forceinline__ void lin_axis(int j, float D, int n, int mul, int& a0, int& a1,
                                         float& t) {
    D = clampD(D);
    float fl = floorf(D);
    t = D - fl;
    int i = wrapi(j + (int)fl, n);
    int i1 = i + 1 == n ? 0 : i + 1;
    a0 = i * mul;
    a1 = i1 * mul;
}

__device__ __forceinline__ LinCell lin_cell(const Grid& g, int x, int y, int z, float dx, float dy,
                                            float dz) {
    LinCell c;
    lin_axis(x, dx, g.nx, 1, c.x0, c.x1, c.tx);
    lin_axis(y, dy, g.ny, g.nx, c.y0, c.y1, c.ty);
    lin_axis(z, dz, g.nz, g.nx * g.ny, c.z0, c.z1, c.tz);
    return c;
}

__device__ __forceinline__ float lin_eval(const float* __restrict__ f, const LinCell& c) {
    float v000 = __ldg(f + c.z0 + c.y0 + c.x0), v001 = __ldg(f + c.z0 + c.y0 + c.x1);
    float v010 = __ldg(f + c.z0 + c.y1 + c.x0), v011 = __ldg(f + c.z0 + c.y1 + c.x1);
    float v100 = __ldg(f + c.z1 + c.y0 + c.x0), v101 = __ldg(f + c.z1 + c.y0 + c.x1);
    float v110 = __ldg(f + c.z1 + c.y1 + c.x0), v111 = __ldg(f + c.z1 + c.y1 + c.x1);
    float a00 = fmaf(c.tx, v001 - v000, v000), a01 = fmaf(c.tx, v011 - v010, v010);
    float a10 = fmaf(c.tx, v101 - v100, v100), a11 = fmaf(c.tx, v111 - v110, v110);
    float b0 = fmaf(c.ty, a01 - a00, a00), b1 = fmaf(c.ty, a11 - a10, a10);
    return fmaf(c.tz, b1 - b0, b0);
}

// value and gradient (d/dx, d/dy, d/dz in voxel units) of the trilinear interpolant
__device__ __forceinline__ float lin_eval_grad(const float* __restrict__ f, const LinCell& c,
                                               float& gx, float& gy, float& gz) {
    float v000 = __ldg(f + c.z0 + c.y0 + c.x0), v001 = __ldg(f + c.z0 + c.y0 + c.x1);
    float v010 = __ldg(f + c.z0 + c.y1 + c.x0), v011 = __ldg(f + c.z0 + c.y1 + c.x1);
    float v100 = __ldg(f + c.z1 + c.y0 + c.x0), v101 = __ldg(f + c.z1 + c.y0 + c.x1);
    float v110 = __ldg(f + c.z1 + c.y1 + c.x0), v111 = __ldg(f + c.z1 + c.y1 + c.x1);
    float a00 = fmaf(c.tx, v001 - v000, v000), a01 = fmaf(c.tx, v011 - v010, v010);
    float a10 = fmaf(c.tx, v101 - v100, v100), a11 = fmaf(c.tx, v111 - v110, v110);
    float b0 = fmaf(c.ty, a01 - a00, a00), b1 = fmaf(c.ty, a11 - a10, a10);
    gz = b1 - b0;
    gy = fmaf(c.tz, (a11 - a10) - (a01 - a00), a01 - a00);
    float dx00 = v001 - v000, dx01 = v011 - v010, dx10 = v101 - v100, dx11 = v111 - v110;
    float e0 = fmaf(c.ty, dx01 - dx00, dx00), e1 = fmaf(c.ty, dx11 - dx10, dx10);
    gx = fmaf(c.tz, e1 - e0, e0);
    return fmaf(c.tz, b1 - b0, b0);
}

// Cubic B-spline cell: 4 taps per axis (i-1 .. i+2) and their weights.
struct CubCell {
    int ox[4], oy[4], oz[4];
    float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void cub_weights(float t, float w[4]) {
    float s = 1.f - t, t2 = t * t, t3 = t2 * t;
    w[0] = s * s * s * (1.f / 6.f);
    w[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
    w[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
    w[3] = t3 * (1.f / 6.f);
}
__device__ __forceinline__ void cub_dweights(float t, float w[4]) {
    float s = 1.f - t;
    w[0] = -0.5f * s * s;
    w[1] = (9.f * t * t - 12.f * t) * (1.f / 6.f);
    w[2] = (-9.f * t * t + 6.f * t + 3.f) * (1.f / 6.f);
    w[3] = 0.5f * t * t;
}

__device__ __forceinline__ void cub_axis(int j, float D, int n, int mul, int o[4], float& t) {
    D = clampD(D);
    float fl = floorf(D);
    t = D - fl;
    int i = wrapi(j + (int)fl - 1, n);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        o[q] = i * mul;
        i = i + 1 == n ? 0 : i + 1;
    }
}

__device__ __forceinline__ CubCell cub_cell(const Grid& g, int x, int y, int z, float dx, float dy,
                                            float dz, float tf[3]) {
    CubCell c;
    cub_axis(x, dx, g.nx, 1, c.ox, tf[0]);
    cub_axis(y, dy, g.ny, g.nx, c.oy, tf[1]);
    cub_axis(z, dz, g.nz, g.nx * g.ny, c.oz, tf[2]);
    cub_weights(tf[0], c.wx);
    cub_weights(tf[1], c.wy);
    cub_weights(tf[2], c.wz);
    return c;
}

__device__ __forceinline__ float cub_eval(const float* __restrict__ f, const CubCell& c) {
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float accy = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float* row = f + c.oz[r] + c.oy[q];
            float ax = c.wx[0] * __ldg(row + c.ox[0]);
            ax = fmaf(c.wx[1], __ldg(row + c.ox[1]), ax);
            ax = fmaf(c.wx[2], __ldg(row + c.ox[2]), ax);
            ax = fmaf(c.wx[3], __ldg(row + c.ox[3]), ax);
            accy = fmaf(c.wy[q], ax, accy);
        }
        acc = fmaf(c.wz[r], accy, acc);
    }
    return acc;
}

__device__ __forceinline__ float cub_eval_grad(const float* __restrict__ f, const CubCell& c,
                                               const float tf[3], float& gx, float& gy,
                                               float& gz) {
    float dwx[4], dwy[4], dwz[4];
    cub_dweights(tf[0], dwx);
    cub_dweights(tf[1], dwy);
    cub_dweights(tf[2], dwz);
    float v = 0.f;
    gx = gy = gz = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float vy = 0.f, vyd = 0.f, vxd = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float* row = f + c.oz[r] + c.oy[q];
            float s0 = __ldg(row + c.ox[0]), s1 = __ldg(row + c.ox[1]);
            float s2 = __ldg(row + c.ox[2]), s3 = __ldg(row + c.ox[3]);
            float ax = c.wx[0] * s0 + c.wx[1] * s1 + c.wx[2] * s2 + c.wx[3] * s3;
            float adx = dwx[0] * s0 + dwx[1] * s1 + dwx[2] * s2 + dwx[3] * s3;
            vy = fmaf(c.wy[q], ax, vy);
            vyd = fmaf(dwy[q], ax, vyd);
            vxd = fmaf(c.wy[q], adx, vxd);
        }
        v = fmaf(c.wz[r], vy, v);
        gz = fmaf(dwz[r], vy, gz);
        gy = fmaf(c.wz[r], vyd, gy);
        gx = fmaf(c.wz[r], vxd, gx);
    }
    return v;
}

// Interpolator front end: IP = 1 trilinear on samples, 3 cubic on spline coefficients.
template <int IP>
struct Interp;

template <>
struct Interp<1> {
    LinCell c;
    __device__ __forceinline__ Interp(const Grid& g, int x, int y, int z, float dx, float dy,
                                      float dz)
        : c(lin_cell(g, x, y, z, dx, dy, dz)) {}
    __device__ __forceinline__ float operator()(const float* f) const { return lin_eval(f, c); }
    __device__ __forceinline__ float grad(const float* f, float& gx, float& gy, float& gz) const {
        return lin_eval_grad(f, c, gx, gy, gz);
    }
};

template <>
struct Interp<3> {
    CubCell c;
    float tf[3];
    __device__ __forceinline__ Interp(const Grid& g, int x, int y, int z, float dx, float dy,
                                      float dz) {
        c = cub_cell(g, x, y, z, dx, dy, dz, tf);
    }
    __device__ __forceinline__ float operator()(const float* f) const { return cub_eval(f, c); }
    __device__ __forceinline__ float grad(const float* f, float& gx, float& gy, float& gz) const {
        return cub_eval_grad(f, c, tf, gx, gy, gz);
    }
};

#define VOXEL_PROLOGUE                                          \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;        \
    const int y = blockIdx.y * blockDim.y + threadIdx.y;        \
    const int z = blockIdx.z;                                   \
    if (x >= g.nx || y >= g.ny) return;                         \
    const long n = g.ntot();                                    \
    const int i = (z * g.ny + y) * g.nx + x;

// launch shape of a voxel kernel for SLArgs (autotuned block, 256 threads)
#define VOX_LAUNCH(a) dim3(cdiv((a).g.nx, (a).bx), cdiv((a).g.ny, (a).by), (a).g.nz), dim3((a).bx, (a).by, 1)

// z planes per thread of the pipelined 3-component kernels: the set value, or (0) the largest
// of 4, 2 that still leaves about two waves of 256-thread blocks on 148 SMs at five per SM.
static int zt_of(const SLArgs& a) {
    if (a.zt > 0) return a.zt;
    const long tiles = (long)cdiv(a.g.nx, a.bx) * cdiv(a.g.ny, a.by);
    for (int zt : {4, 2})
        if (tiles * cdiv(a.g.nz, zt) >= 2L * 148 * 5) return zt;
    return 1;
}

// ---------------------------------------------------------------- characteristics
template <int IP>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 3)
k_sl_char(Grid g, const float* __restrict__ vsrc, const float* __restrict__ vval,
                          float s0, float s1, float s2, float dts, float* __restrict__ D) {
    VOXEL_PROLOGUE
    float V0 = vval[i] * s0, V1 = vval[n + i] * s1, V2 = vval[2 * n + i] * s2;
    Interp<IP> it(g, x, y, z, dts * V0, dts * V1, dts * V2);  // X* = x + dts V
    float W0 = it(vsrc) * s0, W1 = it(vsrc + n) * s1, W2 = it(vsrc + 2 * n) * s2;
    const float h = 0.5f * dts;
    D[i] = h * (W0 + V0);
    D[n + i] = h * (W1 + V1);
    D[2 * n + i] = h * (W2 + V2);
}

// The same over zt consecutive z planes per thread (trilinear): the velocity of plane z + 1
// is loaded while the taps of plane z are in flight.
__global__ void __launch_bounds__(256, 5)
k_sl_char_zt(Grid g, const float* __restrict__ vsrc, const float* __restrict__ vval, float s0,
             float s1, float s2, float dts, float* __restrict__ D, int zt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();             // 3 n < 2^31 (checked at context creation)
    const int plane = g.nx * g.ny;
    int z = blockIdx.z * zt;
    const int zend = min(z + zt, g.nz);
    if (z >= zend) return;
    int i = (z * g.ny + y) * g.nx + x;
    float V0 = __ldcs(vval + i) * s0, V1 = __ldcs(vval + n + i) * s1, V2 = __ldcs(vval + 2 * n + i) * s2;
    const float h = 0.5f * dts;
    for (;;) {
        const bool more = z + 1 < zend;
        const int ip = more ? i + plane : i;
        const float U0 = __ldcs(vval + ip) * s0, U1 = __ldcs(vval + n + ip) * s1,
                    U2 = __ldcs(vval + 2 * n + ip) * s2;
        const Interp<1> it(g, x, y, z, dts * V0, dts * V1, dts * V2);   // X* = x + dts V
        const float W0 = it(vsrc) * s0, W1 = it(vsrc + n) * s1, W2 = it(vsrc + 2 * n) * s2;
        __stcs(D + i, h * (W0 + V0));
        __stcs(D + n + i, h * (W1 + V1));
        __stcs(D + 2 * n + i, h * (W2 + V2));
        if (!more) break;
        ++z;
        i = ip;
        V0 = U0; V1 = U1; V2 = U2;
    }
}

int sl_characteristics(const SLArgs& a, const float* vsrc, const float* vval, const float scale[3],
                       double dt_signed, float* D, cudaStream_t st) {
    KTRACE(a.interp == 3 ? "sl_char_cubic" : "sl_char", st, 36.0 * a.g.ntot(), 0);
    if (a.interp == 3)
        k_sl_char<3><<<VOX_LAUNCH(a), 0, st>>>(a.g, vsrc, vval, scale[0], scale[1],
                                                          scale[2], (float)dt_signed, D);
    else if (zt_of(a) > 1)
        k_sl_char_zt<<<dim3(cdiv(a.g.nx, a.bx), cdiv(a.g.ny, a.by), cdiv(a.g.nz, zt_of(a))),
                       dim3(a.bx, a.by, 1), 0, st>>>(a.g, vsrc, vval, scale[0], scale[1], scale[2],
                                                     (float)dt_signed, D, zt_of(a));
    else
        k_sl_char<1><<<VOX_LAUNCH(a), 0, st>>>(a.g, vsrc, vval, scale[0], scale[1],
                                                          scale[2], (float)dt_signed, D);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ---------------------------------------------------------------- gathers
// MODE 0: out = src o X; 1: * aux(x) (one plane); 2: + aux[c](x). NC components;
// launch bounds keep the trilinear kernel at <= 40 registers (8 warps x 6 CTAs per SM: the
// gathers are latency-bound, so resident warps matter more than registers).
template <int IP, int MODE, int NC>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 6)
k_sl_gather(Grid g, const float* __restrict__ src, const float* __restrict__ D,
            const float* __restrict__ aux, float* __restrict__ out) {
    VOXEL_PROLOGUE
    Interp<IP> it(g, x, y, z, __ldcs(D + i), __ldcs(D + n + i), __ldcs(D + 2 * n + i));
    float sc = MODE == 1 ? __ldcs(aux + i) : 1.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float v = it(src + c * n);
        if (MODE == 1) v *= sc;
        if (MODE == 2) v += __ldcs(aux + c * n + i);
        __stcs(out + c * n + i, v);
    }
}

// Trilinear 3-component gather, zt consecutive z planes per thread: the offsets (and aux) of
// plane z + 1 are loaded while the taps of plane z are in flight, so a thread keeps the two
// levels of its load chain (offsets -> taps) overlapped instead of serialised.
template <int IP, int MODE>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 5)
k_sl_gather_zt(Grid g, const float* __restrict__ src, const float* __restrict__ D,
               const float* __restrict__ aux, float* __restrict__ out, int zt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();             // 3 n < 2^31 (checked at context creation)
    const int plane = g.nx * g.ny;
    int z = blockIdx.z * zt;
    const int zend = min(z + zt, g.nz);
    if (z >= zend) return;
    int i = (z * g.ny + y) * g.nx + x;
    float d0 = __ldcs(D + i), d1 = __ldcs(D + n + i), d2 = __ldcs(D + 2 * n + i);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if (MODE == 1) a0 = __ldcs(aux + i);
    if (MODE == 2) {
        a0 = __ldcs(aux + i);
        a1 = __ldcs(aux + n + i);
        a2 = __ldcs(aux + 2 * n + i);
    }
    for (;;) {
        const bool more = z + 1 < zend;
        const int ip = more ? i + plane : i;
        // next plane's streams, issued before this plane's taps are consumed
        const float e0 = __ldcs(D + ip), e1 = __ldcs(D + n + ip), e2 = __ldcs(D + 2 * n + ip);
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
        if (MODE == 1) b0 = __ldcs(aux + ip);
        if (MODE == 2) {
            b0 = __ldcs(aux + ip);
            b1 = __ldcs(aux + n + ip);
            b2 = __ldcs(aux + 2 * n + ip);
        }
        const Interp<IP> it(g, x, y, z, d0, d1, d2);
        float v0 = it(src), v1 = it(src + n), v2 = it(src + 2 * n);
        if (MODE == 1) {
            v0 *= a0;
            v1 *= a0;
            v2 *= a0;
        }
        if (MODE == 2) {
            v0 += a0;
            v1 += a1;
            v2 += a2;
        }
        __stcs(out + i, v0);
        __stcs(out + n + i, v1);
        __stcs(out + 2 * n + i, v2);
        if (!more) break;
        ++z;
        i = ip;
        d0 = e0; d1 = e1; d2 = e2;
        a0 = b0; a1 = b1; a2 = b2;
    }
}

// The same for NC single fields (NC = 1: the cubic scalar gathers). The trilinear form fits in
// 32 registers, so eight 256-thread blocks (the full 64 warps) stay resident per SM: the
// gathers are latency-bound, and the extra warps raise the scalar transport by ~4%.
template <int IP, int MODE, int NC>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 8)
k_sl_gather_zt1(Grid g, const float* __restrict__ src, const float* __restrict__ D,
               const float* __restrict__ aux, float* __restrict__ out, int zt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();             // 3 n < 2^31 (checked at context creation)
    const int plane = g.nx * g.ny;
    int z = blockIdx.z * zt;
    const int zend = min(z + zt, g.nz);
    if (z >= zend) return;
    int i = (z * g.ny + y) * g.nx + x;
    float d0 = __ldcs(D + i), d1 = __ldcs(D + n + i), d2 = __ldcs(D + 2 * n + i);
    float a[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
        a[c] = MODE == 1 ? (c == 0 ? __ldcs(aux + i) : 0.f) : MODE == 2 ? __ldcs(aux + c * n + i) : 0.f;
    for (;;) {
        const bool more = z + 1 < zend;
        const int ip = more ? i + plane : i;
        // next plane's streams, issued before this plane's taps are consumed
        const float e0 = __ldcs(D + ip), e1 = __ldcs(D + n + ip), e2 = __ldcs(D + 2 * n + ip);
        float b[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            b[c] = MODE == 1 ? (c == 0 ? __ldcs(aux + ip) : 0.f) : MODE == 2 ? __ldcs(aux + c * n + ip) : 0.f;
        float v[NC];
        {
            const Interp<IP> it(g, x, y, z, d0, d1, d2);
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] = it(src + c * n);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (MODE == 1) v[c] *= a[0];
            if (MODE == 2) v[c] += a[c];
            __stcs(out + c * n + i, v[c]);
        }
        if (!more) break;
        ++z;
        i = ip;
        d0 = e0; d1 = e1; d2 = e2;
#pragma unroll
        for (int c = 0; c < NC; ++c) a[c] = b[c];
    }
}

// Trilinear gather, four consecutive x voxels per thread (nx % 4 == 0): float4 offset loads
// and stores, 4 x 8 independent gathers per component in flight.
template <int MODE, int NC>
__global__ void __launch_bounds__(256, 3)
k_sl_gather4(Grid g, const float* __restrict__ src, const float* __restrict__ D,
             const float* __restrict__ aux, float* __restrict__ out) {
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    const long n = g.ntot();
    const int i = (z * g.ny + y) * g.nx + x0;
    const float4 dx = __ldcs(reinterpret_cast<const float4*>(D + i));
    const float4 dy = __ldcs(reinterpret_cast<const float4*>(D + n + i));
    const float4 dz = __ldcs(reinterpret_cast<const float4*>(D + 2 * n + i));
    LinCell cl[4];
    cl[0] = lin_cell(g, x0 + 0, y, z, dx.x, dy.x, dz.x);
    cl[1] = lin_cell(g, x0 + 1, y, z, dx.y, dy.y, dz.y);
    cl[2] = lin_cell(g, x0 + 2, y, z, dx.z, dy.z, dz.z);
    cl[3] = lin_cell(g, x0 + 3, y, z, dx.w, dy.w, dz.w);
    float4 sc = make_float4(1.f, 1.f, 1.f, 1.f);
    if (MODE == 1) sc = __ldcs(reinterpret_cast<const float4*>(aux + i));
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        const float* f = src + c * n;
        float4 r = make_float4(lin_eval(f, cl[0]), lin_eval(f, cl[1]), lin_eval(f, cl[2]),
                               lin_eval(f, cl[3]));
        if (MODE == 1) {
            r.x *= sc.x; r.y *= sc.y; r.z *= sc.z; r.w *= sc.w;
        }
        if (MODE == 2) {
            const float4 a = __ldcs(reinterpret_cast<const float4*>(aux + c * n + i));
            r.x += a.x; r.y += a.y; r.z += a.z; r.w += a.w;
        }
        __stcs(reinterpret_cast<float4*>(out + c * n + i), r);
    }
}

static inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }


template <int IP, int MODE>
static void launch_gather_nc(const SLArgs& a, const float* src, const float* D, const float* aux,
                             int ncomp, float* out, cudaStream_t st) {
    const long n = a.g.ntot();
    const bool vec4 = IP == 1 && (a.g.nx & 3) == 0 && aligned16(src) && aligned16(D) &&
                      aligned16(out) && (aux == nullptr || aligned16(aux));
    const dim3 g4(cdiv(a.g.nx / 4, 16), cdiv(a.g.ny, 16), a.g.nz), b4(16, 16, 1);
    for (int c0 = 0; c0 < ncomp;) {
        int left = ncomp - c0;
        const float* s = src + c0 * n;
        const float* x = MODE == 2 ? aux + c0 * n : aux;
        float* o = out + c0 * n;
        if (IP == 1 && left < 3 && zt_of(a) > 1) {
            // single fields on grids that fill the GPU: one voxel per thread, z-pipelined
            const int zt = zt_of(a);
            k_sl_gather_zt1<IP, MODE, 1><<<dim3(cdiv(a.g.nx, a.bx), cdiv(a.g.ny, a.by), cdiv(a.g.nz, zt)),
                                           dim3(a.bx, a.by, 1), 0, st>>>(a.g, s, D, x, o, zt);
            c0 += 1;
        } else if (vec4 && left < 3) {
            // single fields: four voxels per thread (the 3-component form keeps one voxel per
            // thread, which holds more gathers in flight per register)
            k_sl_gather4<MODE, 1><<<g4, b4, 0, st>>>(a.g, s, D, x, o);
            c0 += 1;
        } else if (left >= 3) {
            const int zt = zt_of(a);
            if (zt > 1)
                k_sl_gather_zt<IP, MODE><<<dim3(cdiv(a.g.nx, a.bx), cdiv(a.g.ny, a.by), cdiv(a.g.nz, zt)),
                                            dim3(a.bx, a.by, 1), 0, st>>>(a.g, s, D, x, o, zt);
            else
                k_sl_gather<IP, MODE, 3><<<VOX_LAUNCH(a), 0, st>>>(a.g, s, D, x, o);
            c0 += 3;
        } else {
            const int zt = zt_of(a);
            if (IP == 3 && zt > 1)   // (trilinear single fields take the four-voxel kernel)
                k_sl_gather_zt1<IP, MODE, 1><<<dim3(cdiv(a.g.nx, a.bx), cdiv(a.g.ny, a.by), cdiv(a.g.nz, zt)),
                                               dim3(a.bx, a.by, 1), 0, st>>>(a.g, s, D, x, o, zt);
            else
                k_sl_gather<IP, MODE, 1><<<VOX_LAUNCH(a), 0, st>>>(a.g, s, D, x, o);
            c0 += 1;
        }
    }
}

template <int MODE>
static int launch_gather(const SLArgs& a, const float* src, const float* D, const float* aux,
                         int ncomp, float* out, cudaStream_t st) {
    static const char* names[2][2][3] = {
        {{"sl_gather", "sl_gather_scale", "sl_gather_add"},
         {"sl_gather_cubic", "sl_gather_scale_cubic", "sl_gather_add_cubic"}},
        {{"sl_gather3", "sl_gather3_scale", "sl_gather3_add"},
         {"sl_gather3_cubic", "sl_gather3_scale_cubic", "sl_gather3_add_cubic"}}};
    KTRACE(names[ncomp == 3][a.interp == 3][MODE], st,
           (double)a.g.ntot() * (12.0 + 8.0 * ncomp + (MODE == 1 ? 4.0 : MODE == 2 ? 4.0 * ncomp : 0.0)), 0);
    if (a.interp == 3)
        launch_gather_nc<3, MODE>(a, src, D, aux, ncomp, out, st);
    else
        launch_gather_nc<1, MODE>(a, src, D, aux, ncomp, out, st);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int sl_gather(const SLArgs& a, const float* src, const float* D, int ncomp, float* out,
              cudaStream_t st) {
    return launch_gather<0>(a, src, D, nullptr, ncomp, out, st);
}
int sl_gather_scale(const SLArgs& a, const float* src, const float* D, const float* gam,
                    int ncomp, float* out, cudaStream_t st) {
    return launch_gather<1>(a, src, D, gam, ncomp, out, st);
}
int sl_gather_add(const SLArgs& a, const float* src, const float* D, const float* add, int ncomp,
                  float* out, cudaStream_t st) {
    return launch_gather<2>(a, src, D, add, ncomp, out, st);
}

// ---------------------------------------------------------------- stationary factors
// Backward Heun step of -D_t u = u d folds into u^j(x) = u^{j+1}(X+) gam(x).
template <int IP>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 3)
k_prep_adjoint(Grid g, const float* __restrict__ dsrc,
                               const float* __restrict__ dval, const float* __restrict__ Dp,
                               float dt, float* __restrict__ gam) {
    VOXEL_PROLOGUE
    Interp<IP> it(g, x, y, z, Dp[i], Dp[n + i], Dp[2 * n + i]);
    float dX = it(dsrc);
    float d = dval[i];
    gam[i] = 1.f + 0.5f * dt * (dX + (1.f + dt * dX) * d);
}

int sl_prep_adjoint(const SLArgs& a, const float* dsrc, const float* dval, const float* Dp,
                    double dt, float* gam, cudaStream_t st) {
    KTRACE("sl_prep_adjoint", st, 24.0 * a.g.ntot(), 0);
    if (a.interp == 3)
        k_prep_adjoint<3><<<VOX_LAUNCH(a), 0, st>>>(a.g, dsrc, dval, Dp, (float)dt, gam);
    else
        k_prep_adjoint<1><<<VOX_LAUNCH(a), 0, st>>>(a.g, dsrc, dval, Dp, (float)dt, gam);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// Deformation state source term with stationary v: W = dt/2 (v(X) + v(x)).
template <int IP>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 3)
k_prep_source(Grid g, const float* __restrict__ vsrc,
                              const float* __restrict__ vval, const float* __restrict__ D,
                              float dt, float* __restrict__ W) {
    VOXEL_PROLOGUE
    Interp<IP> it(g, x, y, z, D[i], D[n + i], D[2 * n + i]);
    for (int c = 0; c < 3; ++c) W[c * n + i] = 0.5f * dt * (it(vsrc + c * n) + vval[c * n + i]);
}

int sl_prep_source(const SLArgs& a, const float* vsrc, const float* vval, const float* D,
                   double dt, float* W, cudaStream_t st) {
    KTRACE("sl_prep_source", st, 48.0 * a.g.ntot(), 0);
    if (a.interp == 3)
        k_prep_source<3><<<VOX_LAUNCH(a), 0, st>>>(a.g, vsrc, vval, D, (float)dt, W);
    else
        k_prep_source<1><<<VOX_LAUNCH(a), 0, st>>>(a.g, vsrc, vval, D, (float)dt, W);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ---------------------------------------------------------------- block reduction
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of a double over a (possibly 2-D) block; thread 0 gets the result.
__device__ double block_sum_d(double v) {
    __shared__ double part[32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    v = warp_sum_d(v);
    if ((t & 31) == 0) part[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t < 32) {
        r = t < (nthreads >> 5) ? part[t] : 0.0;
        r = warp_sum_d(r);
    }
    return r;
}

// ---------------------------------------------------------------- warped source image
// m1 = I0 o (x - u1 to_vox); G = grad(I0 interpolant) there in physical units;
// rho = -(2/sigma2) r G with r = m1 - I1. One partial sum of r^2 per block (grid-stride).
template <int IP>
__global__ void k_warp_image(Grid g, const float* __restrict__ I0src, const float* __restrict__ u1,
                             float t0, float t1, float t2, const float* __restrict__ I1,
                             float coef, float* __restrict__ m1, float* __restrict__ G,
                             float* __restrict__ rho, double* __restrict__ partials) {
    const long n = g.ntot();
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        int x = (int)(i % g.nx);
        long r_ = i / g.nx;
        int y = (int)(r_ % g.ny);
        int z = (int)(r_ / g.ny);
        Interp<IP> it(g, x, y, z, -u1[i] * t0, -u1[n + i] * t1, -u1[2 * n + i] * t2);
        float gx, gy, gz;
        float m = it.grad(I0src, gx, gy, gz);
        gx *= t0;
        gy *= t1;
        gz *= t2;
        float r = m - I1[i];
        acc += (double)r * r;
        if (m1) m1[i] = m;
        if (G) {
            G[i] = gx;
            G[n + i] = gy;
            G[2 * n + i] = gz;
        }
        if (rho) {
            float s = coef * r;
            rho[i] = s * gx;
            rho[n + i] = s * gy;
            rho[2 * n + i] = s * gz;
        }
    }
    double s = block_sum_d(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

int sl_warp_image(const SLArgs& a, const float* I0src, const float* u1, const float to_vox[3],
                  const float* I1, double sigma2, float* m1, float* G, float* rho,
                  double* partials, cudaStream_t st) {
    float coef = (float)(-2.0 / sigma2);
    KTRACE("warp_image", st, a.g.ntot() * (24.0 + (m1 ? 4.0 : 0.0) + (G ? 12.0 : 0.0) + (rho ? 12.0 : 0.0)), 0);
    if (a.interp == 3)
        k_warp_image<3><<<kReduceBlocks, 256, 0, st>>>(a.g, I0src, u1, to_vox[0], to_vox[1],
                                                       to_vox[2], I1, coef, m1, G, rho, partials);
    else
        k_warp_image<1><<<kReduceBlocks, 256, 0, st>>>(a.g, I0src, u1, to_vox[0], to_vox[1],
                                                       to_vox[2], I1, coef, m1, G, rho, partials);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ---------------------------------------------------------------- compositions (state-eq. variant)
// out = mul(x) * src o (x - U(x) to_vox): m_j = I0 o phi_j and lambda_j = J_j lambda(1) o psi_j
// with phi_j = id - iota(u~_j), psi_j = id - iota(nu~_j) (U physical, mul may be null).
template <int IP>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 4)
k_compose(Grid g, const float* __restrict__ src, const float* __restrict__ U, float t0, float t1,
          float t2, const float* __restrict__ mul, float* __restrict__ out) {
    VOXEL_PROLOGUE
    Interp<IP> it(g, x, y, z, -U[i] * t0, -U[n + i] * t1, -U[2 * n + i] * t2);
    const float f = it(src);
    out[i] = mul ? mul[i] * f : f;
}

int sl_compose(const SLArgs& a, const float* src, const float* U, const float to_vox[3],
               const float* mul, float* out, cudaStream_t st) {
    KTRACE("sl_compose", st, a.g.ntot() * (20.0 + (mul ? 4.0 : 0.0)), 0);
    if (a.interp == 3)
        k_compose<3><<<VOX_LAUNCH(a), 0, st>>>(a.g, src, U, to_vox[0], to_vox[1], to_vox[2], mul, out);
    else
        k_compose<1><<<VOX_LAUNCH(a), 0, st>>>(a.g, src, U, to_vox[0], to_vox[1], to_vox[2], mul, out);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// dlambda(1) = -(2/sigma2) dm1 with dm1 = -G . du1
__global__ void k_state_dlam1(long n, const float* __restrict__ G, const float* __restrict__ du,
                              float coef, float* __restrict__ out) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = coef * (G[i] * du[i] + G[n + i] * du[n + i] + G[2 * n + i] * du[2 * n + i]);
}

int state_dlam1(const Grid& g, const float* G, const float* du1, double sigma2, float* out,
                cudaStream_t st) {
    long n = g.ntot();
    KTRACE("state_dlam1", st, 28.0 * n, 6.0 * n);
    k_state_dlam1<<<cdiv(n, 256), 256, 0, st>>>(n, G, du1, (float)(2.0 / sigma2), out);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ---------------------------------------------------------------- incremental state
// The nine Jacobian entries Du[3a + b] = d u_a / d x_b of voxel i: FP32 planes [9][n], or the
// packed BF16 form [n] x 8 entries (one 16-byte load) followed by the plane of entry 8.
__device__ __forceinline__ void load_jac9(const float* __restrict__ Du, int n, int i, float j[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) j[k] = __ldcs(Du + k * n + i);
}
__device__ __forceinline__ void load_jac9(const __nv_bfloat16* __restrict__ Du, int n, int i, float j[9]) {
    const uint4 p = __ldcs(reinterpret_cast<const uint4*>(Du) + i);
    const unsigned w[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        j[2 * k] = __uint_as_float(w[k] << 16);
        j[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
    j[8] = __bfloat162float(Du[8 * n + i]);
}

// D~_t du~ = dv~ - D~u~ * dv~ (Table 1 row 7): F = dv - (Du) dv, Heun along X.
template <int IP, typename TJ>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 4)
k_inc_defstate(Grid g, const float* __restrict__ U, const float* __restrict__ D,
                               const float* __restrict__ Fold, const TJ* __restrict__ Du,
                               const float* __restrict__ dv, float dt, float* __restrict__ out,
                               float* __restrict__ Fnew) {
    VOXEL_PROLOGUE
    float w0 = dv[i], w1 = dv[n + i], w2 = dv[2 * n + i];
    float F[3], J[9];
    load_jac9(Du, (int)n, i, J);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float j0 = J[3 * c], j1 = J[3 * c + 1], j2 = J[3 * c + 2];
        F[c] = (c == 0 ? w0 : c == 1 ? w1 : w2) - (j0 * w0 + j1 * w1 + j2 * w2);
    }
    Interp<IP> it(g, x, y, z, D[i], D[n + i], D[2 * n + i]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        out[c * n + i] = it(U + c * n) + 0.5f * dt * (it(Fold + c * n) + F[c]);
        Fnew[c * n + i] = F[c];
    }
}

// The same step over zt consecutive z planes per thread (trilinear), the offsets of plane
// z + 1 loaded while the taps of plane z are in flight.
template <int IP, typename TJ>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 4)
k_inc_defstate_zt(Grid g, const float* __restrict__ U, const float* __restrict__ D,
                  const float* __restrict__ Fold, const TJ* __restrict__ Du,
                  const float* __restrict__ dv, float dt, float* __restrict__ out,
                  float* __restrict__ Fnew, int zt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int n = (int)g.ntot();             // 3 n < 2^31 (checked at context creation)
    const int plane = g.nx * g.ny;
    int z = blockIdx.z * zt;
    const int zend = min(z + zt, g.nz);
    if (z >= zend) return;
    int i = (z * g.ny + y) * g.nx + x;
    float d0 = __ldcs(D + i), d1 = __ldcs(D + n + i), d2 = __ldcs(D + 2 * n + i);
    const float h = 0.5f * dt;
    for (;;) {
        const bool more = z + 1 < zend;
        const int ip = more ? i + plane : i;
        const float e0 = __ldcs(D + ip), e1 = __ldcs(D + n + ip), e2 = __ldcs(D + 2 * n + ip);
        const Interp<IP> it(g, x, y, z, d0, d1, d2);
        const float w0 = __ldcs(dv + i), w1 = __ldcs(dv + n + i), w2 = __ldcs(dv + 2 * n + i);
        float J[9];
        load_jac9(Du, n, i, J);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float j0 = J[3 * a], j1 = J[3 * a + 1], j2 = J[3 * a + 2];
            const float F = (a == 0 ? w0 : a == 1 ? w1 : w2) - (j0 * w0 + j1 * w1 + j2 * w2);
            __stcs(out + a * n + i, it(U + a * n) + h * (it(Fold + a * n) + F));
            __stcs(Fnew + a * n + i, F);
        }
        if (!more) break;
        ++z;
        i = ip;
        d0 = e0; d1 = e1; d2 = e2;
    }
}

int sl_inc_defstate(const SLArgs& a, const float* U, const float* D, const float* Fold,
                    const void* Du, bool du_bf16, const float* dv, double dt, float* out,
                    float* Fnew, cudaStream_t st) {
    const double bytes = (du_bf16 ? 90.0 : 108.0) * a.g.ntot();
    const char* name = a.interp == 3 ? (du_bf16 ? "sl_inc_defstate_cubic_jbf16" : "sl_inc_defstate_cubic")
                                     : (du_bf16 ? "sl_inc_defstate_jbf16" : "sl_inc_defstate");
    KTRACE(name, st, bytes, 0);
    const auto* j32 = static_cast<const float*>(Du);
    const auto* j16 = static_cast<const __nv_bfloat16*>(Du);
    // the cubic step keeps one voxel per thread: at 128 registers the pipelined form measured
    // slower (1041 against 906 us at 192x224x192), while the cubic gathers gain from it
    if (a.interp == 1 && zt_of(a) > 1) {
        const int zt = zt_of(a);
        const dim3 grid(cdiv(a.g.nx, a.bx), cdiv(a.g.ny, a.by), cdiv(a.g.nz, zt)), block(a.bx, a.by, 1);
        if (du_bf16)
            k_inc_defstate_zt<1, __nv_bfloat16><<<grid, block, 0, st>>>(a.g, U, D, Fold, j16, dv, (float)dt, out, Fnew, zt);
        else
            k_inc_defstate_zt<1, float><<<grid, block, 0, st>>>(a.g, U, D, Fold, j32, dv, (float)dt, out, Fnew, zt);
    } else if (a.interp == 3) {
        if (du_bf16)
            k_inc_defstate<3, __nv_bfloat16><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, j16, dv, (float)dt, out, Fnew);
        else
            k_inc_defstate<3, float><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, j32, dv, (float)dt, out, Fnew);
    } else {
        if (du_bf16)
            k_inc_defstate<1, __nv_bfloat16><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, j16, dv, (float)dt, out, Fnew);
        else
            k_inc_defstate<1, float><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, j32, dv, (float)dt, out, Fnew);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

template <typename TJ>
__global__ void k_defstate_rhs(long n, const TJ* __restrict__ Du, const float* __restrict__ dv,
                               float* __restrict__ F) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float w0 = dv[i], w1 = dv[n + i], w2 = dv[2 * n + i];
    float J[9];
    load_jac9(Du, (int)n, (int)i, J);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float j0 = J[3 * c], j1 = J[3 * c + 1], j2 = J[3 * c + 2];
        F[c * n + i] = (c == 0 ? w0 : c == 1 ? w1 : w2) - (j0 * w0 + j1 * w1 + j2 * w2);
    }
}

int defstate_rhs(const Grid& g, const void* Du, bool du_bf16, const float* dv, float* F,
                 cudaStream_t st) {
    long n = g.ntot();
    KTRACE("defstate_rhs", st, (du_bf16 ? 42.0 : 60.0) * n, 24.0 * n);
    if (du_bf16)
        k_defstate_rhs<<<cdiv(n, 256), 256, 0, st>>>(n, static_cast<const __nv_bfloat16*>(Du), dv, F);
    else
        k_defstate_rhs<<<cdiv(n, 256), 256, 0, st>>>(n, static_cast<const float*>(Du), dv, F);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// FP32 Jacobian planes of `nodes` nodes ([node][9][n]) -> the packed BF16 form read by
// load_jac9 (per node: [n] x entries 0..7 as one 16-byte word, then the plane of entry 8;
// node stride jac_bf16_stride(n) elements), each entry rounded to nearest even.
__global__ void k_pack_jac_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                long n, int nodes, long stride) {
    const long total = n * nodes;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long node = t / n, i = t - node * n;
        const float* src = in + node * 9 * n + i;
        __nv_bfloat16* dst = out + node * stride;
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned lo = __bfloat16_as_ushort(__float2bfloat16_rn(__ldcs(src + (2 * k) * n)));
            const unsigned hi = __bfloat16_as_ushort(__float2bfloat16_rn(__ldcs(src + (2 * k + 1) * n)));
            w[k] = lo | (hi << 16);
        }
        reinterpret_cast<uint4*>(dst)[i] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[8 * n + i] = __float2bfloat16_rn(__ldcs(src + 8 * n));
    }
}

long jac_bf16_stride(long n) { return (9 * n + 7) & ~7L; }

int pack_jac_bf16(const float* in, void* out, long n, int nodes, cudaStream_t st) {
    KTRACE("to_bf16", st, 54.0 * n * nodes, 0);
    const long total = n * nodes;
    k_pack_jac_bf16<<<(int)std::min<long>(cdiv(total, 256), 16 * 148), 256, 0, st>>>(
        in, static_cast<__nv_bfloat16*>(out), n, nodes, jac_bf16_stride(n));
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_defstate_drho1(long n, const float* __restrict__ G, const float* __restrict__ du,
                                 float coef, float* __restrict__ drho) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g0 = G[i], g1 = G[n + i], g2 = G[2 * n + i];
    float dm = -(g0 * du[i] + g1 * du[n + i] + g2 * du[2 * n + i]);
    float s = coef * dm;
    drho[i] = s * g0;
    drho[n + i] = s * g1;
    drho[2 * n + i] = s * g2;
}

int defstate_drho1(const Grid& g, const float* G, const float* du1, double sigma2, float* drho,
                   cudaStream_t st) {
    long n = g.ntot();
    KTRACE("defstate_drho1", st, 36.0 * n, 10.0 * n);
    k_defstate_drho1<<<cdiv(n, 256), 256, 0, st>>>(n, G, du1, (float)(-2.0 / sigma2), drho);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// acc_b (+)= w sum_a Du[a*3+b] R_a   ((D u)^T R, the D~u~ * rho~ term before projection)
template <typename TJ>
__global__ void k_accum_JT(long n, const TJ* __restrict__ Du, const float* __restrict__ R,
                           float w, float* __restrict__ acc, int init) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float r0 = R[i], r1 = R[n + i], r2 = R[2 * n + i];
    float J[9];
    load_jac9(Du, (int)n, (int)i, J);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float s = J[b] * r0 + J[3 + b] * r1 + J[6 + b] * r2;
        acc[b * n + i] = init ? w * s : fmaf(w, s, acc[b * n + i]);
    }
}

int accum_JT(const Grid& g, const void* Du, bool du_bf16, const float* R, float w, float* acc,
             int init, cudaStream_t st) {
    long n = g.ntot();
    KTRACE("accum_JT", st, n * ((du_bf16 ? 42.0 : 60.0) + (init ? 0.0 : 12.0)), 21.0 * n);
    if (du_bf16)
        k_accum_JT<<<cdiv(n, 256), 256, 0, st>>>(n, static_cast<const __nv_bfloat16*>(Du), R, w, acc, init);
    else
        k_accum_JT<<<cdiv(n, 256), 256, 0, st>>>(n, static_cast<const float*>(Du), R, w, acc, init);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// acc_b = sum_j w_j sum_a Du_j[a*3+b] R_j[a] over the nodes j = nt .. 0 in one pass (the
// trapezoid weights: w_end at j = 0 and j = nt, w_mid between). The sum runs in the order of
// the node-by-node form above (node nt first, then one fmaf per node downwards), so both give
// the same bits, while the accumulator is written once instead of read and written per node.
template <typename TJ>
__global__ void __launch_bounds__(256)
k_accum_JT_nodes(long n, int nt, const TJ* __restrict__ Du, long du_stride,
                 const float* __restrict__ R, float w_end, float w_mid, float* __restrict__ acc) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a[3];
#pragma unroll 2
    for (int j = nt; j >= 0; --j) {
        const float* Rj = R + (long)j * 3 * n;
        const float r0 = __ldcs(Rj + i), r1 = __ldcs(Rj + n + i), r2 = __ldcs(Rj + 2 * n + i);
        float J[9];
        load_jac9(Du + (long)j * du_stride, (int)n, (int)i, J);
        const float w = (j == 0 || j == nt) ? w_end : w_mid;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float s = J[b] * r0 + J[3 + b] * r1 + J[6 + b] * r2;
            a[b] = j == nt ? w * s : fmaf(w, s, a[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) acc[b * n + i] = a[b];
}

int accum_JT_nodes(const Grid& g, const void* Du, bool du_bf16, const float* R, int nt,
                   float w_end, float w_mid, float* acc, cudaStream_t st) {
    long n = g.ntot();
    if (nt < 1) { set_error("accum_JT_nodes: nt must be >= 1"); return LDDMM_EINVAL; }
    KTRACE("accum_JT_nodes", st, n * ((nt + 1) * (du_bf16 ? 30.0 : 48.0) + 12.0),
           21.0 * n * (nt + 1));
    if (du_bf16)
        k_accum_JT_nodes<<<cdiv(n, 256), 256, 0, st>>>(n, nt, static_cast<const __nv_bfloat16*>(Du),
                                                       jac_bf16_stride(n), R, w_end, w_mid, acc);
    else
        k_accum_JT_nodes<<<cdiv(n, 256), 256, 0, st>>>(n, nt, static_cast<const float*>(Du), 9 * n, R,
                                                       w_end, w_mid, acc);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// J = det(I - Du) per voxel from the nine planes Du[3a + b] = d u_a / d x_b (physical), with
// per-block minimum and maximum (FP64) into pmin / pmax (kReduceBlocks each).
__global__ void __launch_bounds__(256)
k_jacdet(long n, const float* __restrict__ Du, float* __restrict__ J, double* __restrict__ pmin,
         double* __restrict__ pmax) {
    double mn = 1e300, mx = -1e300;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double a[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) a[r][c] = (r == c ? 1.0 : 0.0) - (double)Du[(3 * r + c) * n + i];
        const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
        if (J) J[i] = (float)det;
        mn = fmin(mn, det);
        mx = fmax(mx, det);
    }
    __shared__ double smin[256], smax[256];
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pmin[blockIdx.x] = smin[0];
        pmax[blockIdx.x] = smax[0];
    }
}

int jacobian_det(const Grid& g, const float* Du, float* J, double* pmin, double* pmax, cudaStream_t st) {
    const long n = g.ntot();
    KTRACE("jacobian_det", st, n * (36.0 + (J ? 4.0 : 0.0)), n * 40.0);
    k_jacdet<<<kReduceBlocks, 256, 0, st>>>(n, Du, J, pmin, pmax);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_fill_field(float* out, float v, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

int fill_field(float* out, float v, long n, cudaStream_t st) {
    KTRACE("fill_field", st, 4.0 * n, 0);
    k_fill_field<<<cdiv(n, 256), 256, 0, st>>>(out, v, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_scale_field(float* out, const float* in, float a, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * in[i];
}

int scale_field(float* out, const float* in, float a, long n, cudaStream_t st) {
    KTRACE("scale_field", st, 8.0 * n, n);
    k_scale_field<<<cdiv(n, 256), 256, 0, st>>>(out, in, a, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_sum_sq_diff(const float* a, const float* b, long n, double* partials) {
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        double d = (double)a[i] - (double)b[i];
        acc += d * d;
    }
    double s = block_sum_d(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

int sum_sq_diff(const float* a, const float* b, long n, double* partials, double* out,
                cudaStream_t st) {
    {
        KTRACE("sum_sq_diff", st, 8.0 * n, 3.0 * n);
        k_sum_sq_diff<<<kReduceBlocks, 256, 0, st>>>(a, b, n, partials);
    }
    LDDMM_CHECK_LAUNCH();
    return finalize_sum(partials, kReduceBlocks, out, st);
}

// ---------------------------------------------------------------- B-spline prefilter
// Periodic cubic B-spline coefficients along one axis: the cyclic system
// (c_{j-1} + 4 c_j + c_{j+1}) / 6 = f_j is solved by the causal / anti-causal recursive
// filter pair with pole zp = sqrt(3) - 2 (Unser, Aldroubi and Eden's B-spline transform),
// each started from its exact periodic initial value (a full-period geometric sum).
__device__ __forceinline__ void prefilter_line(float* f, long stride, int L) {
    const float zp = -0.2679491924311228f;
    float zk = 1.f, s = 0.f;
    for (int k = 0; k < L; ++k) {
        int j = k == 0 ? 0 : L - k;
        s = fmaf(zk, f[(long)j * stride], s);
        zk *= zp;
    }
    const float zL = zk;
    float prev = s / (1.f - zL);
    f[0] = prev;
    for (int j = 1; j < L; ++j) {
        prev = fmaf(zp, prev, f[(long)j * stride]);
        f[(long)j * stride] = prev;
    }
    zk = 1.f;
    s = 0.f;
    for (int k = 0; k < L; ++k) {
        int j = k == 0 ? L - 1 : k - 1;
        s = fmaf(zk, f[(long)j * stride], s);
        zk *= zp;
    }
    float cm = -zp / (1.f - zL) * s;
    f[(long)(L - 1) * stride] = 6.f * cm;
    for (int j = L - 2; j >= 0; --j) {
        cm = zp * (cm - f[(long)j * stride]);
        f[(long)j * stride] = 6.f * cm;
    }
}

// x lines through shared memory: the CTA stages `rows` rows with all of its threads (a flat,
// unrolled copy, so that many loads are in flight), one thread filters one row, and all
// threads write the rows back. Rows are padded to nx + 1 floats (no bank conflicts).
constexpr int PFX_THREADS = 256;

__global__ void __launch_bounds__(PFX_THREADS)
k_prefilter_x(const float* __restrict__ in, float* __restrict__ out, long nrows, int nx, int rows) {
    extern __shared__ float sm[];
    const int ld = nx + 1;
    const long row0 = (long)blockIdx.x * rows;
    const int nr = (int)min((long)rows, nrows - row0);
    const int tot = nr * nx;
    const float* src = in + row0 * nx;
#pragma unroll 4
    for (int e = threadIdx.x; e < tot; e += PFX_THREADS) {
        const int r = e / nx;
        sm[r * ld + (e - r * nx)] = __ldcs(src + e);
    }
    __syncthreads();
    if ((int)threadIdx.x < nr) prefilter_line(sm + threadIdx.x * ld, 1, nx);
    __syncthreads();
    float* dst = out + row0 * nx;
#pragma unroll 4
    for (int e = threadIdx.x; e < tot; e += PFX_THREADS) {
        const int r = e / nx;
        dst[e] = sm[r * ld + (e - r * nx)];
    }
}

// y or z lines in place in global memory: thread per line, consecutive threads along x.
__global__ void k_prefilter_strided(float* f, long nlines, int nx, long outer_stride, long stride,
                                    int L) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlines) return;
    long x = t % nx, o = t / nx;
    prefilter_line(f + o * outer_stride + x, stride, L);
}

// out = B-spline coefficients of ncomp fields `in` (out may alias in).
int bspline_prefilter(const Grid& g, const float* in, int ncomp, float* out, cudaStream_t st) {
    const long n = g.ntot();
    // rows per CTA: up to one per thread, fewer when the staged rows would not fit
    int rows = PFX_THREADS;
    while (rows > 32 && (long)rows * (g.nx + 1) * 4 > 100 * 1024) rows -= 32;
    if ((long)rows * (g.nx + 1) * 4 > 220 * 1024) {
        set_error("bspline_prefilter: nx too large");
        return LDDMM_EINVAL;
    }
    size_t smem = (size_t)rows * (g.nx + 1) * 4;
    static bool attr = false;
    if (!attr) {
        LDDMM_CUDA(cudaFuncSetAttribute(k_prefilter_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024));
        attr = true;
    }
    for (int c = 0; c < ncomp; ++c) {
        const float* src = in + c * n;
        float* dst = out + c * n;
        long nrows = (long)g.ny * g.nz;
        {
            KTRACE("prefilter_x", st, 8.0 * n, 8.0 * n);
            k_prefilter_x<<<cdiv(nrows, rows), PFX_THREADS, smem, st>>>(src, dst, nrows, g.nx, rows);
        }
        LDDMM_CHECK_LAUNCH();
        // y lines: for each z, x -> start z*nx*ny + x, stride nx
        long ly = (long)g.nx * g.nz;
        {
            KTRACE("prefilter_yz", st, 8.0 * n, 8.0 * n);
            k_prefilter_strided<<<cdiv(ly, 128), 128, 0, st>>>(dst, ly, g.nx, (long)g.nx * g.ny,
                                                              g.nx, g.ny);
        }
        LDDMM_CHECK_LAUNCH();
        // z lines: for each y, x -> start y*nx + x, stride nx*ny
        long lz = (long)g.nx * g.ny;
        {
            KTRACE("prefilter_yz", st, 8.0 * n, 8.0 * n);
            k_prefilter_strided<<<cdiv(lz, 128), 128, 0, st>>>(dst, lz, g.nx, g.nx,
                                                              (long)g.nx * g.ny, g.nz);
        }
        LDDMM_CHECK_LAUNCH();
    }
    return LDDMM_OK;
}

// ---------------------------------------------------------------- image variant
// Incremental state, D~_t dm~ = -grad~ m~ * dv~ (Table 1 row 5): F = -Gm . dv,
// out = U o X + dt/2 (Fold o X + Fnew).
template <int IP>
__global__ void __launch_bounds__(256, IP == 3 ? 2 : 3)
k_inc_image(Grid g, const float* __restrict__ U, const float* __restrict__ D,
                            const float* __restrict__ Fold, const float* __restrict__ Gm,
                            const float* __restrict__ dv, float dt, float* __restrict__ out,
                            float* __restrict__ Fnew) {
    VOXEL_PROLOGUE
    float F = -(Gm[i] * dv[i] + Gm[n + i] * dv[n + i] + Gm[2 * n + i] * dv[2 * n + i]);
    Interp<IP> it(g, x, y, z, D[i], D[n + i], D[2 * n + i]);
    out[i] = it(U) + 0.5f * dt * (it(Fold) + F);
    Fnew[i] = F;
}

int sl_inc_image(const SLArgs& a, const float* U, const float* D, const float* Fold,
                 const float* Gm, const float* dv, double dt, float* out, float* Fnew,
                 cudaStream_t st) {
    KTRACE(a.interp == 3 ? "sl_inc_image_cubic" : "sl_inc_image", st, 52.0 * a.g.ntot(), 0);
    if (a.interp == 3)
        k_inc_image<3><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, Gm, dv, (float)dt, out,
                                                            Fnew);
    else
        k_inc_image<1><<<VOX_LAUNCH(a), 0, st>>>(a.g, U, D, Fold, Gm, dv, (float)dt, out,
                                                            Fnew);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_image_rhs(long n, const float* __restrict__ Gm, const float* __restrict__ dv,
                            float* __restrict__ F) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) F[i] = -(Gm[i] * dv[i] + Gm[n + i] * dv[n + i] + Gm[2 * n + i] * dv[2 * n + i]);
}

int image_rhs(const Grid& g, const float* Gm, const float* dv, float* F, cudaStream_t st) {
    long n = g.ntot();
    KTRACE("image_rhs", st, 28.0 * n, 6.0 * n);
    k_image_rhs<<<cdiv(n, 256), 256, 0, st>>>(n, Gm, dv, F);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// acc_b (+)= w s(x) Gm_b(x)   (the lambda~ * grad~ m~ term before projection)
__global__ void k_accum_sv(long n, const float* __restrict__ s, const float* __restrict__ Gm,
                           float w, float* __restrict__ acc, int init) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = w * s[i];
#pragma unroll
    for (int b = 0; b < 3; ++b)
        acc[b * n + i] = init ? v * Gm[b * n + i] : fmaf(v, Gm[b * n + i], acc[b * n + i]);
}

// four voxels per thread (n % 4 == 0, 16-byte aligned planes): 16-byte loads and stores
__global__ void k_accum_sv4(long n4, long n, const float4* __restrict__ s, const float* __restrict__ Gm,
                            float w, float* __restrict__ acc, int init) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const float4 sv = __ldcs(s + i);
    const float4 v = make_float4(w * sv.x, w * sv.y, w * sv.z, w * sv.w);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float4 gm = __ldcs(reinterpret_cast<const float4*>(Gm + b * n) + i);
        float4* a = reinterpret_cast<float4*>(acc + b * n) + i;
        float4 r;
        if (init) {
            r = make_float4(v.x * gm.x, v.y * gm.y, v.z * gm.z, v.w * gm.w);
        } else {
            const float4 o = *a;
            r = make_float4(fmaf(v.x, gm.x, o.x), fmaf(v.y, gm.y, o.y), fmaf(v.z, gm.z, o.z),
                            fmaf(v.w, gm.w, o.w));
        }
        *a = r;
    }
}

int accum_sv(const Grid& g, const float* s, const float* Gm, float w, float* acc, int init,
             cudaStream_t st) {
    long n = g.ntot();
    KTRACE("accum_sv", st, n * (28.0 + (init ? 0.0 : 12.0)), 7.0 * n);
    const bool al = ((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(Gm) |
                      reinterpret_cast<uintptr_t>(acc)) & 15) == 0;
    if ((n & 3) == 0 && al)
        k_accum_sv4<<<cdiv(n / 4, 256), 256, 0, st>>>(n / 4, n, reinterpret_cast<const float4*>(s), Gm,
                                                      w, acc, init);
    else
        k_accum_sv<<<cdiv(n, 256), 256, 0, st>>>(n, s, Gm, w, acc, init);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// acc_b = sum_{j=nt..0} w_j s_j(x) Gm_{j,b}(x) in one pass over the nodes (s_j at S + n j, Gm_j at
// Gm + 3 n j; w_j = w_end at j = 0 and nt, w_mid between), in the order and with the roundings
// of accum_sv node by node from j = nt down, so both give the same bits.
__global__ void __launch_bounds__(256)
k_accum_sv_nodes(long n, int nt, const float* __restrict__ S, const float* __restrict__ Gm,
                 float w_end, float w_mid, float* __restrict__ acc) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a[3];
#pragma unroll 2
    for (int j = nt; j >= 0; --j) {
        const float w = (j == 0 || j == nt) ? w_end : w_mid;
        const float v = w * __ldcs(S + (long)j * n + i);
        const float* G = Gm + (long)j * 3 * n;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float gm = __ldcs(G + b * n + i);
            a[b] = j == nt ? v * gm : fmaf(v, gm, a[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) acc[b * n + i] = a[b];
}

// four voxels per thread (n % 4 == 0, 16-byte aligned planes)
__global__ void __launch_bounds__(256)
k_accum_sv4_nodes(long n4, long n, int nt, const float* __restrict__ S, const float* __restrict__ Gm,
                  float w_end, float w_mid, float* __restrict__ acc) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    float4 a[3];
#pragma unroll 2
    for (int j = nt; j >= 0; --j) {
        const float w = (j == 0 || j == nt) ? w_end : w_mid;
        const float4 sv = __ldcs(reinterpret_cast<const float4*>(S + (long)j * n) + i);
        const float4 v = make_float4(w * sv.x, w * sv.y, w * sv.z, w * sv.w);
        const float* G = Gm + (long)j * 3 * n;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float4 gm = __ldcs(reinterpret_cast<const float4*>(G + b * n) + i);
            if (j == nt)
                a[b] = make_float4(v.x * gm.x, v.y * gm.y, v.z * gm.z, v.w * gm.w);
            else
                a[b] = make_float4(fmaf(v.x, gm.x, a[b].x), fmaf(v.y, gm.y, a[b].y),
                                   fmaf(v.z, gm.z, a[b].z), fmaf(v.w, gm.w, a[b].w));
        }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) reinterpret_cast<float4*>(acc + b * n)[i] = a[b];
}

int accum_sv_nodes(const Grid& g, const float* S, const float* Gm, int nt, float w_end, float w_mid,
                   float* acc, cudaStream_t st) {
    long n = g.ntot();
    if (nt < 1) { set_error("accum_sv_nodes: nt must be >= 1"); return LDDMM_EINVAL; }
    KTRACE("accum_sv_nodes", st, n * ((nt + 1) * 16.0 + 12.0), 7.0 * n * (nt + 1));
    const bool al = ((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(Gm) |
                      reinterpret_cast<uintptr_t>(acc)) & 15) == 0;
    if ((n & 3) == 0 && al)
        k_accum_sv4_nodes<<<cdiv(n / 4, 256), 256, 0, st>>>(n / 4, n, nt, S, Gm, w_end, w_mid, acc);
    else
        k_accum_sv_nodes<<<cdiv(n, 256), 256, 0, st>>>(n, nt, S, Gm, w_end, w_mid, acc);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// lambda(1) = coef (m1 - I1)
__global__ void k_axpy_diff(long n, const float* a, const float* b, float coef, float* out) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = coef * (a[i] - b[i]);
}

int scaled_diff(const Grid& g, const float* a, const float* b, float coef, float* out,
                cudaStream_t st) {
    long n = g.ntot();
    KTRACE("scaled_diff", st, 12.0 * n, 2.0 * n);
    k_axpy_diff<<<cdiv(n, 256), 256, 0, st>>>(n, a, b, coef, out);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

}  // namespace lddmm
