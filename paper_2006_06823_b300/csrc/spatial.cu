// Spatial-domain form (Sec. 2.1 with SL-RK integration in Omega, Sec. 3): the velocity and
// every transported quantity are fields on the image grid. The band-limited machinery is
// replaced by the identity for pi and iota, while L = (Id - alpha Laplacian)^s, its inverse
// (the PCG preconditioner, Eqs. 13-14) and the spectral derivatives of the fields (grad m,
// D u, div v) go through full-grid FFTs (cuFFT, the plain library transform). Everything
// else -- characteristics, gathers, incremental steps, accumulations -- is the same kernels.
// The same transforms restrict the images of a band-limited context to the half grid for the
// coarse level of the two-level preconditioner.
#include <cufft.h>

#include <algorithm>
#include <string>

#include "common.cuh"

namespace lddmm {

namespace {

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

#define LDDMM_CUFFT(expr)                                                               \
    do {                                                                                \
        cufftResult r__ = (expr);                                                       \
        if (r__ != CUFFT_SUCCESS) {                                                     \
            set_error(std::string(#expr) + ": cuFFT error " + std::to_string((int)r__)); \
            return LDDMM_ECUDA;                                                         \
        }                                                                               \
    } while (0)

// signed integer wavenumber of index i on n points (numpy's fftfreq order)
__device__ __forceinline__ int wavenum(int i, int n) { return i <= n / 2 - (n % 2 == 0) ? i : i - n; }

// Spectrum [nz][ny][nxh] of one component (R2C layout, nxh = nx/2 + 1).
// mode 1: s *= wL w(k) / n; mode -1: s *= 1 / (w(k) n), w(k) = (1 + alpha |k|^2)^s.
__global__ void k_spec_L(cufftComplex* spec, int nx, int ny, int nz, float wL, double alpha, int sexp,
                         int mode, double inv_n) {
    const int nxh = nx / 2 + 1;
    const long tot = (long)nz * ny * nxh;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxh);
        const int iy = (int)((i / nxh) % ny);
        const int iz = (int)(i / ((long)nxh * ny));
        const double kx = ix, ky = wavenum(iy, ny), kz = wavenum(iz, nz);
        const double b = 1.0 + alpha * (kx * kx + ky * ky + kz * kz);
        double w = 1.0;
        for (int q = 0; q < sexp; ++q) w *= b;
        const float f = (float)(mode > 0 ? wL * w * inv_n : inv_n / w);
        cufftComplex v = spec[i];
        spec[i] = make_float2(v.x * f, v.y * f);
    }
}

// acc (=, +=) i k_axis spec / n, the Nyquist wavenumber of that axis contributing zero
__global__ void k_spec_deriv(const cufftComplex* spec, cufftComplex* acc, int nx, int ny, int nz,
                             int axis, int accumulate, double inv_n) {
    const int nxh = nx / 2 + 1;
    const long tot = (long)nz * ny * nxh;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxh);
        const int iy = (int)((i / nxh) % ny);
        const int iz = (int)(i / ((long)nxh * ny));
        int k, n;
        if (axis == 0) { k = ix; n = nx; }
        else if (axis == 1) { k = wavenum(iy, ny); n = ny; }
        else { k = wavenum(iz, nz); n = nz; }
        if (n % 2 == 0 && (k == n / 2 || k == -n / 2)) k = 0;
        const float f = (float)(k * inv_n);
        const cufftComplex v = spec[i];
        const float2 d = make_float2(-f * v.y, f * v.x);
        if (accumulate) {
            const cufftComplex a = acc[i];
            acc[i] = make_float2(a.x + d.x, a.y + d.y);
        } else {
            acc[i] = d;
        }
    }
}

__global__ void k_axpy_f32(float* out, float a, const float* y, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fmaf(a, y[i], out[i]);
}

__global__ void k_maxabs_f32(const float* a, long n, double* partials) {
    __shared__ double sm[256];
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        s = fmax(s, fabs((double)a[i]));
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void k_finalize_max(const double* partials, int n, double* out) {
    __shared__ double sm[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, partials[i]);
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// Coarse half spectrum [nzc][nyc][nxc/2 + 1] from the fine one: modes with 2|k_a| < n_a (the
// half grid's n) copied with the factor scale (1/n_fine: mean-normalised coefficients, which
// the unnormalised C2R then synthesises), every other mode zero.
__global__ void k_spec_restrict(const cufftComplex* __restrict__ fs, int nxf, int nyf, int nzf,
                                cufftComplex* __restrict__ cs, int nxc, int nyc, int nzc, float scale) {
    const int nxhc = nxc / 2 + 1, nxhf = nxf / 2 + 1;
    const long tot = (long)nzc * nyc * nxhc;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxhc);
        const int iy = (int)((i / nxhc) % nyc);
        const int iz = (int)(i / ((long)nxhc * nyc));
        const int kx = ix, ky = wavenum(iy, nyc), kz = wavenum(iz, nzc);
        cufftComplex v = make_float2(0.f, 0.f);
        if (2 * kx < nxc && 2 * abs(ky) < nyc && 2 * abs(kz) < nzc) {
            const int fy = ky < 0 ? ky + nyf : ky, fz = kz < 0 ? kz + nzf : kz;
            const cufftComplex f = fs[((long)fz * nyf + fy) * nxhf + kx];
            v = make_float2(f.x * scale, f.y * scale);
        }
        cs[i] = v;
    }
}

inline int spec_grid(const Grid& g) {
    const long tot = (long)g.nz * g.ny * (g.nx / 2 + 1);
    return (int)std::min<long>(cdiv(tot, 256), 4L * kReduceBlocks);
}

}  // namespace

struct SpatialFFT {
    Grid g;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
    cufftComplex* spec = nullptr;   // one component's half spectrum
    cufftComplex* acc = nullptr;    // divergence accumulator / derivative output
};

int spatial_fft_create(const Grid& g, cudaStream_t st, SpatialFFT** out) {
    *out = nullptr;
    auto* f = new SpatialFFT;
    f->g = g;
    const long nspec = (long)g.nz * g.ny * (g.nx / 2 + 1);
    auto fail = [&](int code) {
        spatial_fft_destroy(f);
        return code;
    };
    if (cufftPlan3d(&f->r2c, g.nz, g.ny, g.nx, CUFFT_R2C) != CUFFT_SUCCESS) {
        set_error("cufftPlan3d (R2C) failed");
        return fail(LDDMM_ECUDA);
    }
    f->have_r2c = true;
    if (cufftPlan3d(&f->c2r, g.nz, g.ny, g.nx, CUFFT_C2R) != CUFFT_SUCCESS) {
        set_error("cufftPlan3d (C2R) failed");
        return fail(LDDMM_ECUDA);
    }
    f->have_c2r = true;
    if (cufftSetStream(f->r2c, st) != CUFFT_SUCCESS || cufftSetStream(f->c2r, st) != CUFFT_SUCCESS) {
        set_error("cufftSetStream failed");
        return fail(LDDMM_ECUDA);
    }
    if (cudaMalloc(&f->spec, nspec * sizeof(cufftComplex)) != cudaSuccess ||
        cudaMalloc(&f->acc, nspec * sizeof(cufftComplex)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of the FFT buffers failed");
        return fail(LDDMM_ENOMEM);
    }
    *out = f;
    return LDDMM_OK;
}

void spatial_fft_destroy(SpatialFFT* f) {
    if (!f) return;
    if (f->have_r2c) cufftDestroy(f->r2c);
    if (f->have_c2r) cufftDestroy(f->c2r);
    cudaFree(f->spec);
    cudaFree(f->acc);
    delete f;
}

int spatial_apply_L(SpatialFFT* f, float* out, const float* x, float wL, float a, const float* y,
                    int ncomp, double alpha, int s, int mode, cudaStream_t st) {
    const Grid& g = f->g;
    const long n = g.ntot();
    for (int c = 0; c < ncomp; ++c) {
        LDDMM_CUFFT(cufftExecR2C(f->r2c, const_cast<float*>(x + c * n), f->spec));
        {
            KTRACE("spatial_L", st, 16.0 * n, 8.0 * n);
            k_spec_L<<<spec_grid(g), 256, 0, st>>>(f->spec, g.nx, g.ny, g.nz, wL, alpha, s, mode,
                                                  1.0 / (double)n);
        }
        LDDMM_CHECK_LAUNCH();
        // out may alias x: the spectrum is complete before the inverse writes out
        LDDMM_CUFFT(cufftExecC2R(f->c2r, f->spec, out + c * n));
        if (mode > 0 && y && a != 0.f) {
            KTRACE("spatial_axpy", st, 12.0 * n, 2.0 * n);
            k_axpy_f32<<<cdiv(n, 256), 256, 0, st>>>(out + c * n, a, y + c * n, n);
            LDDMM_CHECK_LAUNCH();
        }
    }
    return LDDMM_OK;
}

int spatial_deriv(SpatialFFT* f, const float* in, int ncomp, int axis, float* out, long fstride,
                  cudaStream_t st) {
    const Grid& g = f->g;
    const long n = g.ntot();
    if (axis == 3) {  // divergence of three fields into one
        for (int c = 0; c < 3; ++c) {
            LDDMM_CUFFT(cufftExecR2C(f->r2c, const_cast<float*>(in + c * n), f->spec));
            KTRACE("spatial_deriv", st, 16.0 * n, 4.0 * n);
            k_spec_deriv<<<spec_grid(g), 256, 0, st>>>(f->spec, f->acc, g.nx, g.ny, g.nz, c, c > 0,
                                                      1.0 / (double)n);
            LDDMM_CHECK_LAUNCH();
        }
        LDDMM_CUFFT(cufftExecC2R(f->c2r, f->acc, out));
        return LDDMM_OK;
    }
    for (int c = 0; c < ncomp; ++c) {
        LDDMM_CUFFT(cufftExecR2C(f->r2c, const_cast<float*>(in + c * n), f->spec));
        {
            KTRACE("spatial_deriv", st, 16.0 * n, 4.0 * n);
            k_spec_deriv<<<spec_grid(g), 256, 0, st>>>(f->spec, f->acc, g.nx, g.ny, g.nz, axis, 0,
                                                      1.0 / (double)n);
        }
        LDDMM_CHECK_LAUNCH();
        LDDMM_CUFFT(cufftExecC2R(f->c2r, f->acc, out + c * fstride));
    }
    return LDDMM_OK;
}

int spectral_restrict_half(const Grid& gf, const float* const* in, const Grid& gc, float* const* out,
                           int nimg, cudaStream_t st) {
    if (gf.nx != 2 * gc.nx || gf.ny != 2 * gc.ny || gf.nz != 2 * gc.nz) {
        set_error("spectral_restrict_half: the coarse grid must be half the fine grid");
        return LDDMM_EINVAL;
    }
    SpatialFFT *ff = nullptr, *fc = nullptr;
    int rc = spatial_fft_create(gf, st, &ff);
    if (rc == LDDMM_OK) rc = spatial_fft_create(gc, st, &fc);
    for (int i = 0; rc == LDDMM_OK && i < nimg; ++i) {
        cufftResult r = cufftExecR2C(ff->r2c, const_cast<float*>(in[i]), ff->spec);
        if (r != CUFFT_SUCCESS) {
            set_error("cufftExecR2C (restriction): cuFFT error " + std::to_string((int)r));
            rc = LDDMM_ECUDA;
            break;
        }
        {
            KTRACE("spec_restrict", st, 16.0 * gc.ntot(), 2.0 * gc.ntot());
            k_spec_restrict<<<spec_grid(gc), 256, 0, st>>>(ff->spec, gf.nx, gf.ny, gf.nz, fc->spec, gc.nx,
                                                          gc.ny, gc.nz, (float)(1.0 / (double)gf.ntot()));
        }
        if (cudaGetLastError() != cudaSuccess) {
            set_error("k_spec_restrict launch failed");
            rc = LDDMM_ECUDA;
            break;
        }
        r = cufftExecC2R(fc->c2r, fc->spec, out[i]);
        if (r != CUFFT_SUCCESS) {
            set_error("cufftExecC2R (restriction): cuFFT error " + std::to_string((int)r));
            rc = LDDMM_ECUDA;
        }
    }
    // the plans and spectra are released only after the work queued on them has finished
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == LDDMM_OK) {
        set_error("spectral_restrict_half: stream synchronisation failed");
        rc = LDDMM_ECUDA;
    }
    spatial_fft_destroy(ff);
    spatial_fft_destroy(fc);
    return rc;
}

int max_abs_f32(const float* a, long n, double* partials, double* out, cudaStream_t st) {
    {
        KTRACE("maxabs_f32", st, 4.0 * n, n);
        k_maxabs_f32<<<kReduceBlocks, 256, 0, st>>>(a, n, partials);
    }
    LDDMM_CHECK_LAUNCH();
    {
        KTRACE("finalize", st, 8.0 * kReduceBlocks, kReduceBlocks);
        k_finalize_max<<<1, 256, 0, st>>>(partials, kReduceBlocks, out);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

}  // namespace lddmm
