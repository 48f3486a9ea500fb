// Spatial-domain form (Sec. 2.1 with SL-RK integration in Omega, Sec. 3): the velocity and
// every transported quantity are fields on the image grid. The band-limited machinery is
// replaced by the identity for pi and iota, while L = (Id - alpha Laplacian)^s, its inverse
// (the PCG preconditioner, Eqs. 13-14) and the spectral derivatives of the fields (grad m,
// D u, div v) go through full-grid FFTs. Everything else -- characteristics, gathers,
// incremental steps, accumulations -- is the same kernels. The same transforms restrict the
// images of a band-limited context to the half grid for the coarse level of the two-level
// preconditioner.
//
// The FFTs are the library's own: a real-to-half-complex 3-D transform (spectrum
// [nz][ny][nx/2 + 1], unnormalised, e^{-i k.x} forward and e^{+i k.x} inverse) as three passes
// of batched 1-D complex transforms in shared memory, one line per group of threads: the x pass
// turns rows of real samples into their nx/2 + 1 leading bins (the inverse rebuilds the other
// half from Hermitian symmetry and keeps the real part), the y and z passes transform columns of
// the half spectrum in place, a CTA holding 16 consecutive kx columns so that loads and stores
// stay coalesced. A 1-D transform of length n = R1 R2 ... Rm is a Stockham autosort sequence of
// radix-R stages (R = 4, 2, 3, 5, 7, or a remaining prime factor as a direct small DFT), each
// butterfly scaling its R inputs by the twiddles exp(-2 pi i r (j mod Ns) / (Ns R)) and writing
// its small DFT to the positions (j div Ns) Ns R + (j mod Ns) + s Ns; twiddles come from a
// table of exp(-2 pi i k / n) evaluated in FP64 per axis length.

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace lddmm {

namespace {

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

using cplx = float2;

#define TRY_FFT(expr)                   \
    do {                                \
        int rc__ = (expr);              \
        if (rc__ != LDDMM_OK) return rc__; \
    } while (0)

// signed integer wavenumber of index i on n points (numpy's fftfreq order)
__device__ __forceinline__ int wavenum(int i, int n) { return i <= n / 2 - (n % 2 == 0) ? i : i - n; }

// Spectrum [nz][ny][nxh] of one component (R2C layout, nxh = nx/2 + 1).
// mode 1: s *= wL w(k) / n; mode -1: s *= 1 / (w(k) n), w(k) = (1 + alpha |k|^2)^s.
__global__ void k_spec_L(cplx* spec, int nx, int ny, int nz, float wL, double alpha, int sexp,
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
        cplx v = spec[i];
        spec[i] = make_float2(v.x * f, v.y * f);
    }
}

// acc (=, +=) i k_axis spec / n, the Nyquist wavenumber of that axis contributing zero
__global__ void k_spec_deriv(const cplx* spec, cplx* acc, int nx, int ny, int nz,
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
        const cplx v = spec[i];
        const float2 d = make_float2(-f * v.y, f * v.x);
        if (accumulate) {
            const cplx a = acc[i];
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
__global__ void k_spec_restrict(const cplx* __restrict__ fs, int nxf, int nyf, int nzf,
                                cplx* __restrict__ cs, int nxc, int nyc, int nzc, float scale) {
    const int nxhc = nxc / 2 + 1, nxhf = nxf / 2 + 1;
    const long tot = (long)nzc * nyc * nxhc;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxhc);
        const int iy = (int)((i / nxhc) % nyc);
        const int iz = (int)(i / ((long)nxhc * nyc));
        const int kx = ix, ky = wavenum(iy, nyc), kz = wavenum(iz, nzc);
        cplx v = make_float2(0.f, 0.f);
        if (2 * kx < nxc && 2 * abs(ky) < nyc && 2 * abs(kz) < nzc) {
            const int fy = ky < 0 ? ky + nyf : ky, fz = kz < 0 ? kz + nzf : kz;
            const cplx f = fs[((long)fz * nyf + fy) * nxhf + kx];
            v = make_float2(f.x * scale, f.y * scale);
        }
        cs[i] = v;
    }
}

inline int spec_grid(const Grid& g) {
    const long tot = (long)g.nz * g.ny * (g.nx / 2 + 1);
    return (int)std::min<long>(cdiv(tot, 256), 4L * kReduceBlocks);
}

// ------------------------------------------------------------------ 1-D FFTs in shared memory
constexpr int kMaxStages = 16;
constexpr int kMaxRadix = 1024;   // a prime factor (direct DFT) up to the largest axis
constexpr int kFftThreads = 256;
constexpr int kColTile = 16;      // kx columns per CTA in the y and z passes

struct Plan1D {
    int n, nst;
    int radix[kMaxStages];
};

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One radix-R butterfly of a Stockham stage: inputs in[j + r m] (r < R) scaled by the
// twiddles exp(-+2 pi i r k / (Ns R)), their R-point DFT written to out[base + s Ns].
template <int R>
__device__ __forceinline__ void bfly(const cplx* in, cplx* out, int j, int m, int k, int step,
                                     int base, int Ns, int n, const cplx* tw, int sign) {
    cplx v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cplx x = in[j + r * m];
        if (r > 0 && k > 0) {
            cplx t = tw[r * k * step];
            if (sign > 0) t.y = -t.y;
            x = cmul(x, t);
        }
        v[r] = x;
    }
    const int wr = n / R;
#pragma unroll
    for (int sidx = 0; sidx < R; ++sidx) {
        cplx acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            cplx t = tw[((r * sidx) % R) * wr];
            if (sign > 0) t.y = -t.y;
            const cplx q = cmul(v[r], t);
            acc.x += q.x;
            acc.y += q.y;
        }
        out[base + sidx * Ns] = acc;
    }
}

// the same for a prime factor R > 7 (direct DFT, one output at a time)
__device__ void bfly_generic(const cplx* in, cplx* out, int R, int j, int m, int k, int step,
                             int base, int Ns, int n, const cplx* tw, int sign) {
    const int wr = n / R;
    for (int sidx = 0; sidx < R; ++sidx) {
        cplx acc = make_float2(0.f, 0.f);
        for (int r = 0; r < R; ++r) {
            cplx x = in[j + r * m];
            if (r > 0 && k > 0) {
                cplx t = tw[r * k * step];
                if (sign > 0) t.y = -t.y;
                x = cmul(x, t);
            }
            cplx t = tw[((r * sidx) % R) * wr];
            if (sign > 0) t.y = -t.y;
            const cplx q = cmul(x, t);
            acc.x += q.x;
            acc.y += q.y;
        }
        out[base + sidx * Ns] = acc;
    }
}

// Transforms `lines` lines of length n held in smem buffer a (line l at a + l * lds), ping-
// ponging with b; returns the buffer holding the result. tw: exp(-2 pi i k / n), k < n (smem);
// sign -1 forward (e^{-i}), +1 inverse (conjugate twiddles). All threads of the CTA take part.
__device__ cplx* fft_lines(cplx* a, cplx* b, int lines, int lds, const Plan1D& P, const cplx* tw,
                           int sign) {
    const int n = P.n;
    int Ns = 1;
    for (int st = 0; st < P.nst; ++st) {
        const int R = P.radix[st];
        const int m = n / R;             // butterflies per line
        const int step = n / (Ns * R);   // twiddle index step for (r, k): r k step < n
        for (int w = threadIdx.x; w < lines * m; w += blockDim.x) {
            const int l = w / m, j = w - l * m;
            const int k = j % Ns;
            const cplx* in = a + (long)l * lds;
            cplx* out = b + (long)l * lds;
            const int base = (j / Ns) * Ns * R + k;
            switch (R) {
                case 2: bfly<2>(in, out, j, m, k, step, base, Ns, n, tw, sign); break;
                case 3: bfly<3>(in, out, j, m, k, step, base, Ns, n, tw, sign); break;
                case 4: bfly<4>(in, out, j, m, k, step, base, Ns, n, tw, sign); break;
                case 5: bfly<5>(in, out, j, m, k, step, base, Ns, n, tw, sign); break;
                case 7: bfly<7>(in, out, j, m, k, step, base, Ns, n, tw, sign); break;
                default: bfly_generic(in, out, R, j, m, k, step, base, Ns, n, tw, sign); break;
            }
        }
        __syncthreads();
        cplx* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// x pass, forward: rows of nx reals -> bins 0 .. nx/2 of each row (spec row stride nxh)
__global__ void __launch_bounds__(kFftThreads)
k_fft_rows_r2c(const float* __restrict__ in, cplx* __restrict__ spec, long rows, int rows_per_cta,
               Plan1D P, const cplx* __restrict__ twg) {
    extern __shared__ float4 smem4[];
    const int n = P.n, nxh = n / 2 + 1;
    cplx* tw = reinterpret_cast<cplx*>(smem4);
    cplx* a = tw + n;
    cplx* b = a + (long)rows_per_cta * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const long r0 = (long)blockIdx.x * rows_per_cta;
    const int lines = (int)std::min<long>(rows_per_cta, rows - r0);
    for (int e = threadIdx.x; e < lines * n; e += blockDim.x)
        a[e] = make_float2(in[r0 * n + e], 0.f);
    __syncthreads();
    const cplx* res = fft_lines(a, b, lines, n, P, tw, -1);
    for (int e = threadIdx.x; e < lines * nxh; e += blockDim.x) {
        const int l = e / nxh, k = e - l * nxh;
        spec[(r0 + l) * nxh + k] = res[(long)l * n + k];
    }
}

// x pass, inverse: bins 0 .. nx/2 of each row -> nx reals (the other bins from Hermitian
// symmetry, the real part of the inverse transform)
__global__ void __launch_bounds__(kFftThreads)
k_fft_rows_c2r(const cplx* __restrict__ spec, float* __restrict__ out, long rows, int rows_per_cta,
               Plan1D P, const cplx* __restrict__ twg) {
    extern __shared__ float4 smem4[];
    const int n = P.n, nxh = n / 2 + 1;
    cplx* tw = reinterpret_cast<cplx*>(smem4);
    cplx* a = tw + n;
    cplx* b = a + (long)rows_per_cta * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const long r0 = (long)blockIdx.x * rows_per_cta;
    const int lines = (int)std::min<long>(rows_per_cta, rows - r0);
    for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
        const int l = e / n, k = e - l * n;
        cplx v;
        if (k < nxh) {
            v = spec[(r0 + l) * nxh + k];
        } else {
            v = spec[(r0 + l) * nxh + (n - k)];
            v.y = -v.y;
        }
        a[e] = v;
    }
    __syncthreads();
    const cplx* res = fft_lines(a, b, lines, n, P, tw, +1);
    for (int e = threadIdx.x; e < lines * n; e += blockDim.x) out[r0 * n + e] = res[e].x;
}

// y or z pass in place on the half spectrum: lines of length n at element stride `estride`;
// the CTA takes kColTile consecutive columns c (stride 1, c < ncol) of line group g (stride
// gstride): element e of column c is at g * gstride + c + e * estride
__global__ void __launch_bounds__(kFftThreads)
k_fft_cols(cplx* __restrict__ spec, int ncol, long estride, long gstride, Plan1D P,
           const cplx* __restrict__ twg, int sign) {
    extern __shared__ float4 smem4[];
    const int n = P.n, lds = n + 1;   // padded line stride: the column loads spread over banks
    cplx* tw = reinterpret_cast<cplx*>(smem4);
    cplx* a = tw + n;
    cplx* b = a + (long)kColTile * lds;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const int c0 = blockIdx.x * kColTile;
    const int cols = min(kColTile, ncol - c0);
    cplx* base = spec + (long)blockIdx.y * gstride + c0;
    // a[c][e] <- column c0 + c, element e (consecutive threads take consecutive columns)
    for (int t = threadIdx.x; t < kColTile * n; t += blockDim.x) {
        const int c = t % kColTile, e = t / kColTile;
        if (c < cols) a[(long)c * lds + e] = base[(long)e * estride + c];
    }
    __syncthreads();
    const cplx* res = fft_lines(a, b, cols, lds, P, tw, sign);
    for (int t = threadIdx.x; t < kColTile * n; t += blockDim.x) {
        const int c = t % kColTile, e = t / kColTile;
        if (c < cols) base[(long)e * estride + c] = res[(long)c * lds + e];
    }
}

// twiddle table exp(-2 pi i k / n), k < n, evaluated in FP64
__global__ void k_fft_twiddles(cplx* tw, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sv, cv;
    sincospi(-2.0 * (double)k / (double)n, &sv, &cv);
    tw[k] = make_float2((float)cv, (float)sv);
}

bool make_plan(int n, Plan1D& P) {
    P.n = n;
    P.nst = 0;
    int m = n;
    auto take = [&](int r) {
        while (m % r == 0 && P.nst < kMaxStages) {
            P.radix[P.nst++] = r;
            m /= r;
        }
    };
    take(4);
    take(2);
    take(3);
    take(5);
    take(7);
    for (int p = 11; m > 1 && p <= kMaxRadix; p += 2) take(p);
    return m == 1;
}

}  // namespace

struct SpatialFFT {
    Grid g;
    Plan1D px, py, pz;
    cplx *twx = nullptr, *twy = nullptr, *twz = nullptr;   // twiddle tables per axis
    int rows_per_cta = 1;
    cplx* spec = nullptr;   // one component's half spectrum
    cplx* acc = nullptr;    // divergence accumulator / derivative output
};

namespace {

size_t rows_smem(const SpatialFFT* f) {
    return sizeof(cplx) * ((size_t)f->g.nx + 2 * (size_t)f->rows_per_cta * f->g.nx);
}
size_t cols_smem(int n) { return sizeof(cplx) * ((size_t)n + 2 * (size_t)kColTile * (n + 1)); }

// spec <- forward transform of the real field x (unnormalised)
int fft_r2c(const SpatialFFT* f, const float* x, cplx* spec, cudaStream_t st) {
    const Grid& g = f->g;
    const int nxh = g.nx / 2 + 1;
    const long rows = (long)g.nz * g.ny;
    {
        KTRACE("fft_x", st, 4.0 * g.ntot() + 8.0 * rows * nxh, 0);
        k_fft_rows_r2c<<<cdiv(rows, f->rows_per_cta), kFftThreads, rows_smem(f), st>>>(
            x, spec, rows, f->rows_per_cta, f->px, f->twx);
    }
    LDDMM_CHECK_LAUNCH();
    {
        KTRACE("fft_y", st, 16.0 * rows * nxh, 0);
        k_fft_cols<<<dim3(cdiv(nxh, kColTile), g.nz), kFftThreads, cols_smem(g.ny), st>>>(
            spec, nxh, nxh, (long)g.ny * nxh, f->py, f->twy, -1);
    }
    LDDMM_CHECK_LAUNCH();
    {
        KTRACE("fft_z", st, 16.0 * rows * nxh, 0);
        k_fft_cols<<<dim3(cdiv(nxh, kColTile), g.ny), kFftThreads, cols_smem(g.nz), st>>>(
            spec, nxh, (long)g.ny * nxh, nxh, f->pz, f->twz, -1);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// out <- inverse transform of the Hermitian half spectrum (unnormalised); spec is overwritten
int fft_c2r(const SpatialFFT* f, cplx* spec, float* out, cudaStream_t st) {
    const Grid& g = f->g;
    const int nxh = g.nx / 2 + 1;
    const long rows = (long)g.nz * g.ny;
    {
        KTRACE("fft_z", st, 16.0 * rows * nxh, 0);
        k_fft_cols<<<dim3(cdiv(nxh, kColTile), g.ny), kFftThreads, cols_smem(g.nz), st>>>(
            spec, nxh, (long)g.ny * nxh, nxh, f->pz, f->twz, +1);
    }
    LDDMM_CHECK_LAUNCH();
    {
        KTRACE("fft_y", st, 16.0 * rows * nxh, 0);
        k_fft_cols<<<dim3(cdiv(nxh, kColTile), g.nz), kFftThreads, cols_smem(g.ny), st>>>(
            spec, nxh, nxh, (long)g.ny * nxh, f->py, f->twy, +1);
    }
    LDDMM_CHECK_LAUNCH();
    {
        KTRACE("fft_x", st, 8.0 * rows * nxh + 4.0 * g.ntot(), 0);
        k_fft_rows_c2r<<<cdiv(rows, f->rows_per_cta), kFftThreads, rows_smem(f), st>>>(
            spec, out, rows, f->rows_per_cta, f->px, f->twx);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

}  // namespace

int spatial_fft_create(const Grid& g, cudaStream_t st, SpatialFFT** out) {
    *out = nullptr;
    auto* f = new SpatialFFT;
    f->g = g;
    const long nspec = (long)g.nz * g.ny * (g.nx / 2 + 1);
    auto fail = [&](int code) {
        spatial_fft_destroy(f);
        return code;
    };
    if (!make_plan(g.nx, f->px) || !make_plan(g.ny, f->py) || !make_plan(g.nz, f->pz)) {
        set_error("spatial form: every grid size must factor into primes up to " +
                  std::to_string(kMaxRadix));
        return fail(LDDMM_EINVAL);
    }
    // rows per CTA of the x pass: as many as fit twice in 48 KB with the twiddles (at least 1)
    f->rows_per_cta = std::max(1, std::min(16, (int)((48 * 1024 / sizeof(cplx) - g.nx) / (2 * g.nx))));
    const size_t need_cols = std::max(cols_smem(g.ny), cols_smem(g.nz));
    if (rows_smem(f) > 200 * 1024 || need_cols > 200 * 1024) {
        set_error("spatial form: an axis is too long for the shared-memory transforms");
        return fail(LDDMM_EINVAL);
    }
    if (cudaMalloc(&f->spec, nspec * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&f->acc, nspec * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&f->twx, g.nx * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&f->twy, g.ny * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&f->twz, g.nz * sizeof(cplx)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of the FFT buffers failed");
        return fail(LDDMM_ENOMEM);
    }
    k_fft_twiddles<<<cdiv(g.nx, 256), 256, 0, st>>>(f->twx, g.nx);
    k_fft_twiddles<<<cdiv(g.ny, 256), 256, 0, st>>>(f->twy, g.ny);
    k_fft_twiddles<<<cdiv(g.nz, 256), 256, 0, st>>>(f->twz, g.nz);
    count_launches(3);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("FFT twiddle tables: launch failed");
        return fail(LDDMM_ECUDA);
    }
    for (auto fn : {reinterpret_cast<const void*>(k_fft_rows_r2c), reinterpret_cast<const void*>(k_fft_rows_c2r),
                    reinterpret_cast<const void*>(k_fft_cols)}) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
            cudaGetLastError();
            set_error("FFT kernels: shared-memory attribute refused");
            return fail(LDDMM_ECUDA);
        }
    }
    *out = f;
    return LDDMM_OK;
}

void spatial_fft_destroy(SpatialFFT* f) {
    if (!f) return;
    cudaFree(f->spec);
    cudaFree(f->acc);
    cudaFree(f->twx);
    cudaFree(f->twy);
    cudaFree(f->twz);
    delete f;
}

int spatial_apply_L(SpatialFFT* f, float* out, const float* x, float wL, float a, const float* y,
                    int ncomp, double alpha, int s, int mode, cudaStream_t st) {
    const Grid& g = f->g;
    const long n = g.ntot();
    for (int c = 0; c < ncomp; ++c) {
        TRY_FFT(fft_r2c(f, x + c * n, f->spec, st));
        {
            KTRACE("spatial_L", st, 16.0 * n, 8.0 * n);
            k_spec_L<<<spec_grid(g), 256, 0, st>>>(f->spec, g.nx, g.ny, g.nz, wL, alpha, s, mode,
                                                  1.0 / (double)n);
        }
        LDDMM_CHECK_LAUNCH();
        // out may alias x: the spectrum is complete before the inverse writes out
        TRY_FFT(fft_c2r(f, f->spec, out + c * n, st));
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
            TRY_FFT(fft_r2c(f, in + c * n, f->spec, st));
            KTRACE("spatial_deriv", st, 16.0 * n, 4.0 * n);
            k_spec_deriv<<<spec_grid(g), 256, 0, st>>>(f->spec, f->acc, g.nx, g.ny, g.nz, c, c > 0,
                                                      1.0 / (double)n);
            LDDMM_CHECK_LAUNCH();
        }
        TRY_FFT(fft_c2r(f, f->acc, out, st));
        return LDDMM_OK;
    }
    for (int c = 0; c < ncomp; ++c) {
        TRY_FFT(fft_r2c(f, in + c * n, f->spec, st));
        {
            KTRACE("spatial_deriv", st, 16.0 * n, 4.0 * n);
            k_spec_deriv<<<spec_grid(g), 256, 0, st>>>(f->spec, f->acc, g.nx, g.ny, g.nz, axis, 0,
                                                      1.0 / (double)n);
        }
        LDDMM_CHECK_LAUNCH();
        TRY_FFT(fft_c2r(f, f->acc, out + c * fstride, st));
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
        rc = fft_r2c(ff, in[i], ff->spec, st);
        if (rc != LDDMM_OK) break;
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
        rc = fft_c2r(fc, fc->spec, out[i], st);
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
