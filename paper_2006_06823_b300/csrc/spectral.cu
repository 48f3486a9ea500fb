// Band-limited projection pi and inclusion iota (Sec. 2.2) as separable partial DFTs.
//
// pi(f)_k = (1/N) sum_x f(x) e^{-i k.x} is computed axis by axis:
//   stage X  A[row][kx]    = sum_jx f[row][jx] e^{-i kx 2pi jx/nx},  kx = 0..K/2-1 only:
//                            f is real, so the kx < 0 half is the conjugate mirror;
//   stage Y  B[z][jy][kx]  = sum_y A[z][y][kx] e^{-i ky 2pi y/ny},   all retained ky;
//   stage Z  c[jz][jy][jx] = (1/N) sum_z B[z][jy][kx] e^{-i kz 2pi z/nz}, plus the mirror.
// iota runs the same three stages backwards (Z, Y on the kx >= 0 half, then X producing
// the real field as Re(T[0]) + 2 Re sum_{kx>0} T[kx] e^{i kx x}).
//
// Stage X touches the full grid and carries almost all of the work: it is a GEMM with
// M = rows (ncomp*nz*ny), N = K (cos and sin of K/2 modes), K-dim = nx. Here it runs as a
// register-blocked FP32 SIMT contraction with the twiddles staged in shared memory; the
// Y and Z stages operate on L2-resident intermediates.
#include "common.cuh"
#include "lddmm.h"

#include <algorithm>

namespace lddmm {

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Split of iota's Y stage into blocks of nyb positions (2 nyb <= 256 columns, nyb a multiple of
// 8 so that N = 2 nyb is a multiple of 16); false if ny has no such split.
static bool iota_y_blocks(int ny, int* nblk, int* nyb) {
    for (int b = (2 * ny + 255) / 256; b <= kMaxIotaYBlocks; ++b)
        if (ny % (8 * b) == 0) {
            *nblk = b;
            *nyb = ny / b;
            return true;
        }
    return false;
}

// The Y stages run on the tensor cores when both precision forms fit: W rows 2K (pi) and the
// (cos, sin) pairs of iota's positions, K-major operand rows of ny and K floats (16-B
// aligned rows), even row counts for the complex completion.
static bool tc_y_possible(const Grid& g, int K) {
    int nb, nyb;
    if ((K % 8) != 0 || (g.ny % 4) != 0 || !iota_y_blocks(g.ny, &nb, &nyb)) return false;
    const void* aligned = reinterpret_cast<const void*>(uintptr_t(256));
    return tc_rowgemm_supported(2 * K, g.ny, 2, aligned, g.ny, 2) &&
           tc_rowgemm_supported(2 * nyb, K, 2, aligned, K, 3, -1, nb) &&
           tc_rowgemm_supported(K, g.nx, 2, aligned, g.nx, 1);
}

static long ytables_floats(const Grid& g, int K) {
    if (!tc_y_possible(g, K)) return 0;
    int nb, nyb;
    iota_y_blocks(g.ny, &nb, &nyb);
    long f = 2L * K * g.ny * 2;   // W matrices of pi Y and iota Y
    f += 2 * ((tc_wimage_bytes(2 * K, g.ny) + 255) / 4 + nb * ((tc_wimage_bytes(2 * nyb, K) + 255) / 4));
    return f + 64 * (2 + 2 * nb);
}

long twiddle_floats(const Grid& g, int K) {
    // tables, W_pi and W_io, then the two tensor-core operand images (64-float aligned)
    long f = 2L * K * ((long)g.nx + g.ny + g.nz) + 2L * K * g.nx;
    f = (f + 63) & ~63L;
    f += 2 * ((tc_wimage_bytes(K, g.nx) + 255) / 4 + (tc_wimage_bytes(g.nx, K) + 255) / 4);
    f = (f + 63) & ~63L;
    f += 2L * K * (2L * g.ny + g.nz);  // mpy, miy, mpz (float2)
    f = (f + 63) & ~63L;
    f += ytables_floats(g, K);
    return f + 64;
}

// [q][p] complex contraction matrix from a twiddle table: M[q][p] = cos + i sgn sin at
// (mode, position) = (p, q) (mode_is_p) or (q, p); mode slot 0 zero when zero_mode0.
__global__ void k_build_cmat(const float* cosT, const float* sinT, int len, int P, int Q,
                             float sgn, int mode_is_p, int zero_mode0, float2* M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * Q) return;
    const int q = i / P, pp = i - q * P;
    const int m = mode_is_p ? pp : q, x = mode_is_p ? q : pp;
    const long o = (long)m * len + x;
    M[i] = (zero_mode0 && m == 0) ? make_float2(0.f, 0.f) : make_float2(cosT[o], sgn * sinT[o]);
}

// Y-stage matrices of the tensor-core path from the y twiddle table (slot jy: wavenumber
// jy - K/2): wpy[2 jy + {0, 1}][y] = {cos, sin}, wiy[2 y + {0, 1}][jy] = {cos, sin} (0 at jy = 0)
__global__ void k_build_wy(const float* cyT, const float* syT, int K, int ny, float* wpy, float* wiy) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * K * ny) return;
    {
        const int n = i / ny, y = i - n * ny, jy = n >> 1;
        const long o = (long)jy * ny + y;
        wpy[i] = (n & 1) ? syT[o] : cyT[o];
    }
    {
        const int n = i / K, jy = i - n * K, y = n >> 1;
        const long o = (long)jy * ny + y;
        wiy[i] = jy == 0 ? 0.f : ((n & 1) ? syT[o] : cyT[o]);
    }
}

// x-stage matrices of the tensor-core path from the x twiddle table (slot h + kx = wavenumber kx)
__global__ void k_build_w(const float* cxT, const float* sxT, int K, int nx, float* wpi, float* wio) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * nx) return;
    const int h = K / 2;
    // W_pi[n][jx]
    {
        int n = i / nx, jx = i - n * nx;
        int kx = n >> 1;
        long o = (long)(h + kx) * nx + jx;
        wpi[i] = (kx < h) ? ((n & 1) ? -sxT[o] : cxT[o]) : 0.f;
    }
    // W_io[x][j]
    {
        int x = i / K, j = i - x * K;
        int kx = j >> 1;
        long o = (long)(h + kx) * nx + x;
        float w = kx == 0 ? 1.f : 2.f;
        wio[i] = (kx < h) ? ((j & 1) ? -w * sxT[o] : w * cxT[o]) : 0.f;
    }
}

__global__ void k_twiddle(float* cosT, float* sinT, int K, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * n) return;
    int slot = i / n, j = i - slot * n;
    long k = slot - K / 2;
    long r = ((k * j) % n + n) % n;  // exact phase reduction
    double s, c;
    sincospi(2.0 * (double)r / (double)n, &s, &c);
    cosT[i] = (float)c;
    sinT[i] = (float)s;
}

int twiddle_init(const Grid& g, int K, float* mem, Twiddles& tw, cudaStream_t st) {
    const int ns[3] = {g.nx, g.ny, g.nz};
    const float* ptrs[6];
    float* p = mem;
    for (int a = 0; a < 3; ++a) {
        int n = ns[a];
        {
            KTRACE("twiddle", st, 8.0 * K * n, 0);
            k_twiddle<<<cdiv((long)K * n, 256), 256, 0, st>>>(p, p + (long)K * n, K, n);
        }
        LDDMM_CHECK_LAUNCH();
        ptrs[2 * a] = p;
        ptrs[2 * a + 1] = p + (long)K * n;
        p += 2L * K * n;
    }
    tw.K = K;
    tw.cx = ptrs[0]; tw.sx = ptrs[1];
    tw.cy = ptrs[2]; tw.sy = ptrs[3];
    tw.cz = ptrs[4]; tw.sz = ptrs[5];
    float* wpi = p;
    float* wio = p + (long)K * g.nx;
    {
        KTRACE("twiddle", st, 16.0 * K * g.nx, 0);
        k_build_w<<<cdiv((long)K * g.nx, 256), 256, 0, st>>>(ptrs[0], ptrs[1], K, g.nx, wpi, wio);
    }
    LDDMM_CHECK_LAUNCH();
    tw.wpi = wpi;
    tw.wio = wio;
    long off = (p - mem) + 2L * K * g.nx;
    off = (off + 63) & ~63L;
    unsigned char* img = reinterpret_cast<unsigned char*>(mem + off);
    const long bpi = (tc_wimage_bytes(K, g.nx) + 255) & ~255L;
    const long bio = (tc_wimage_bytes(g.nx, K) + 255) & ~255L;
    for (int prec = 0; prec < 2; ++prec) {
        unsigned char* img_pi = img + prec * (bpi + bio);
        unsigned char* img_io = img_pi + bpi;
        int rc = tc_build_wimage(wpi, K, g.nx, prec, img_pi, st);
        if (rc) return rc;
        rc = tc_build_wimage(wio, g.nx, K, prec, img_io, st);
        if (rc) return rc;
        tw.wpi_img[prec] = img_pi;
        tw.wio_img[prec] = img_io;
    }
    {
        long moff = (long)(img + 2 * (bpi + bio) - reinterpret_cast<unsigned char*>(mem)) / 4;
        moff = (moff + 63) & ~63L;
        float2* m = reinterpret_cast<float2*>(mem + moff);
        float2* mpy = m;
        float2* miy = mpy + (long)K * g.ny;
        float2* mpz = miy + (long)K * g.ny;
        KTRACE("twiddle", st, 24.0 * K * (2.0 * g.ny + g.nz), 0);
        k_build_cmat<<<cdiv((long)K * g.ny, 256), 256, 0, st>>>(tw.cy, tw.sy, g.ny, K, g.ny, -1.f, 1, 0, mpy);
        k_build_cmat<<<cdiv((long)K * g.ny, 256), 256, 0, st>>>(tw.cy, tw.sy, g.ny, g.ny, K, 1.f, 0, 1, miy);
        k_build_cmat<<<cdiv((long)K * g.nz, 256), 256, 0, st>>>(tw.cz, tw.sz, g.nz, K, g.nz, -1.f, 1, 0, mpz);
        LDDMM_CHECK_LAUNCH();
        count_launches(2);
        tw.mpy = mpy;
        tw.miy = miy;
        tw.mpz = mpz;
        moff += 2L * K * (2L * g.ny + g.nz);
        moff = (moff + 63) & ~63L;
        // Y stages on the tensor cores: W matrices, then their operand images
        tw.tc_y = tc_y_possible(g, K);
        tw.iy_blocks = tw.iy_nyb = 0;
        if (tw.tc_y) {
            int nb, nyb;
            iota_y_blocks(g.ny, &nb, &nyb);
            tw.iy_blocks = nb;
            tw.iy_nyb = nyb;
            float* wpy = mem + moff;
            float* wiy = wpy + 2L * K * g.ny;
            {
                KTRACE("twiddle", st, 32.0 * K * g.ny, 0);
                k_build_wy<<<cdiv(2L * K * g.ny, 256), 256, 0, st>>>(tw.cy, tw.sy, K, g.ny, wpy, wiy);
            }
            LDDMM_CHECK_LAUNCH();
            long boff = moff + 4L * K * g.ny;
            boff = (boff + 63) & ~63L;
            unsigned char* b = reinterpret_cast<unsigned char*>(mem + boff);
            const long bpy = (tc_wimage_bytes(2 * K, g.ny) + 255) & ~255L;
            const long biy = (tc_wimage_bytes(2 * nyb, K) + 255) & ~255L;
            for (int prec = 0; prec < 2; ++prec) {
                int rc = tc_build_wimage(wpy, 2 * K, g.ny, prec, b, st);
                if (rc) return rc;
                tw.wpy_img[prec] = b;
                b += bpy;
                for (int blk = 0; blk < nb; ++blk) {
                    rc = tc_build_wimage(wiy + 2L * blk * nyb * K, 2 * nyb, K, prec, b, st);
                    if (rc) return rc;
                    tw.wiy_img[prec][blk] = b;
                    b += biy;
                }
            }
        }
    }
    return LDDMM_OK;
}

long spectral_scratch_elems(const Grid& g, int K, int ncomp) {
    long kh = K / 2;
    long a = (long)ncomp * g.nz * g.ny * kh;      // stage X output / iota stage Y output
    long b = (long)ncomp * g.nz * K * kh;         // stage Y output / iota stage Z output
    long c = (long)ncomp * K * K * K;             // B-spline-divided input cube
    return std::max(a, std::max(b, c));
}

// ------------------------------------------------------------------------ pi, stage X
// CTA: ROWS rows x all KH modes. Thread (row group rg, mode pair p): rows rg + 16 i
// (i = 0..3) and modes 2p, 2p+1 -> 16 accumulators. Shared memory: rows padded to
// ldr = round4(nx) + 4 floats (conflict-free float4 reads across row groups), twiddles
// as (cos, sin) pairs at [jx][kx] so a thread reads both of its modes with one float4.
constexpr int PX_ROWS = 64;

template <int KHP>
__global__ void __launch_bounds__(KHP * 8)
k_pi_x(const float* __restrict__ f, long fstride, long rows_per_comp, int ncomp, int nx,
       int KH, int K, const float* __restrict__ cosT, const float* __restrict__ sinT,
       float2* __restrict__ A) {
    constexpr int NT = KHP * 8;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int nxp = (nx + 3) & ~3;
    const int ldr = nxp + 4;
    float* frow = sm;                                             // PX_ROWS * ldr
    float2* tw = reinterpret_cast<float2*>(sm + PX_ROWS * ldr);  // nxp * KHP
    const int tid = threadIdx.x;

    for (int e = tid; e < nxp * KHP; e += NT) {
        int jx = e / KHP, kx = e - jx * KHP;
        float2 v = make_float2(0.f, 0.f);
        if (jx < nx && kx < KH) {
            long o = (long)(K / 2 + kx) * nx + jx;
            v = make_float2(cosT[o], sinT[o]);
        }
        tw[e] = v;
    }
    const long rows = rows_per_comp * ncomp;
    const long row0 = (long)blockIdx.x * PX_ROWS;
    const bool contiguous = fstride == rows_per_comp * nx;
    if (contiguous && (nx & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
        // the CTA's rows are one contiguous chunk: every 16-byte copy in flight at once
        const int q4 = nx >> 2;
        const float* base = f + row0 * nx;
        for (int e = tid; e < PX_ROWS * q4; e += NT) {
            int r = e / q4, qq = e - r * q4;
            float* dst = &frow[r * ldr + 4 * qq];
            if (row0 + r < rows) {
                unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa),
                             "l"(base + (long)e * 4));
            } else {
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
        for (int r = 0; r < PX_ROWS; ++r) {
            long row = row0 + r;
            const float* src = nullptr;
            if (row < rows) {
                long comp = row / rows_per_comp;
                src = f + comp * fstride + (row - comp * rows_per_comp) * nx;
            }
            for (int x = tid; x < nxp; x += NT)
                frow[r * ldr + x] = (src && x < nx) ? __ldcs(src + x) : 0.f;
        }
    }
    __syncthreads();

    const int p = tid % (KHP / 2);
    const int rg = tid / (KHP / 2);  // 0..15
    float re[4][2], im[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) re[i][q] = im[i][q] = 0.f;

    for (int jx = 0; jx < nxp; jx += 4) {
        float4 fr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            fr[i] = *reinterpret_cast<const float4*>(&frow[(rg + 16 * i) * ldr + jx]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 t = *reinterpret_cast<const float4*>(&tw[(jx + q) * KHP + 2 * p]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v = q == 0 ? fr[i].x : q == 1 ? fr[i].y : q == 2 ? fr[i].z : fr[i].w;
                re[i][0] = fmaf(v, t.x, re[i][0]);
                im[i][0] = fmaf(-v, t.y, im[i][0]);
                re[i][1] = fmaf(v, t.z, re[i][1]);
                im[i][1] = fmaf(-v, t.w, im[i][1]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        long row = row0 + rg + 16 * i;
        if (row >= rows) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int kx = 2 * p + q;
            if (kx < KH) A[row * KH + kx] = make_float2(re[i][q], im[i][q]);
        }
    }
}

// 8-byte asynchronous global -> shared copy; zero fill when !ok (source size 0)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}

// ------------------------------------------- Y and Z stages: batched twiddle contractions
// Out[split][s][p][col] = sum_{q in split's range} M[q][p] In[s][q][col] for every slab s and
// column col < C, with M a prebuilt complex matrix (Twiddles::mpy / miy / mpz). The columns of
// all slabs form one GEMM dimension N = nslab * C. CTA tile: PT = 16 RPT rows p x NT columns,
// q in chunks of 32 through double-buffered shared memory (cp.async prefetch of the next
// chunk during the current one). Thread (rg, cg): rows RPT rg .. RPT rg + RPT - 1 and columns
// cg + 16 j (j < NT/16), so that for each j the 16 threads of a row group touch 16
// consecutive columns: one shared-memory wavefront per read and 128-byte global stores. The
// per-thread load positions do not change with q, so the index arithmetic (including the
// slab division) is done once.
constexpr int CG_QT = 32;

template <int RPT, int NT>
__global__ void __launch_bounds__(256)
k_cgemm_tw(const float2* __restrict__ M, int P, int Q, int C, int N, const float2* __restrict__ In,
           long inS, long inQ, float2* __restrict__ Out, long outS, long outP, long outSplit) {
    constexpr int PT = 16 * RPT;
    constexpr int CPT = NT / 16;         // columns per thread
    constexpr int IROWS = 256 / NT;      // q rows of the input tile loaded per pass
    constexpr int MROWS = 256 / PT;      // q rows of the matrix tile loaded per pass
    __shared__ __align__(16) float2 Ms[2][CG_QT][PT];
    __shared__ __align__(16) float2 Is[2][CG_QT][NT];
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const int n0 = blockIdx.x * NT;
    const int p0 = blockIdx.y * PT;
    const int qsplit = gridDim.z;
    const int qlen = (Q + qsplit - 1) / qsplit;
    const int qb = blockIdx.z * qlen, qe = min(Q, qb + qlen);
    // load positions: matrix tile column pl (rows ql0 + MROWS r), input tile column nl (rows
    // qi0 + IROWS r)
    const int pl = tid % PT, ql0 = tid / PT;
    const bool pok = p0 + pl < P;
    const int nl = tid % NT, qi0 = tid / NT;
    const int nload = n0 + nl;
    const bool nok = nload < N;
    const int sl = nok ? nload / C : 0;
    const float2* inp = In + (long)sl * inS + (nload - sl * C);
    // asynchronous copy of the chunk starting at q0 into buffer b (zero fill outside)
    auto issue = [&](int b, int q0) {
#pragma unroll
        for (int r = 0; r < CG_QT / MROWS; ++r) {
            const int ql = ql0 + MROWS * r, q = q0 + ql;
            const bool ok = pok && q < qe;
            cp_async8(&Ms[b][ql][pl], ok ? M + (long)q * P + p0 + pl : M, ok);
        }
#pragma unroll
        for (int r = 0; r < CG_QT / IROWS; ++r) {
            const int ql = qi0 + IROWS * r, q = q0 + ql;
            const bool ok = nok && q < qe;
            cp_async8(&Is[b][ql][nl], ok ? inp + (long)q * inQ : In, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    float ar[RPT][CPT], ai[RPT][CPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) ar[i][j] = ai[i][j] = 0.f;
    // one q step: the thread's RPT matrix entries (broadcast reads) times its CPT inputs
    auto step = [&](int b, int ql) {
        float2 mv[RPT];
#pragma unroll
        for (int i = 0; i < RPT; i += 2) {
            const float4 m4 = *reinterpret_cast<const float4*>(&Ms[b][ql][RPT * rg + i]);
            mv[i] = make_float2(m4.x, m4.y);
            mv[i + 1] = make_float2(m4.z, m4.w);
        }
        float2 iv[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) iv[j] = Is[b][ql][cg + 16 * j];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                ar[i][j] = fmaf(mv[i].x, iv[j].x, fmaf(-mv[i].y, iv[j].y, ar[i][j]));
                ai[i][j] = fmaf(mv[i].x, iv[j].y, fmaf(mv[i].y, iv[j].x, ai[i][j]));
            }
    };
    if (qb < qe) issue(0, qb);
    for (int q0 = qb, b = 0; q0 < qe; q0 += CG_QT, b ^= 1) {
        if (q0 + CG_QT < qe) {
            issue(b ^ 1, q0 + CG_QT);   // buffer b ^ 1 was last read before the previous barrier
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const int qn = min(CG_QT, qe - q0);
        if (qn == CG_QT) {
#pragma unroll
            for (int ql = 0; ql < CG_QT; ++ql) step(b, ql);
        } else {
            for (int ql = 0; ql < qn; ++ql) step(b, ql);
        }
        __syncthreads();
    }
    float2* out = Out + (long)blockIdx.z * outSplit;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const int n = n0 + cg + 16 * j;
        if (n >= N) continue;
        const int s = n / C;
        float2* o = out + (long)s * outS + (n - s * C);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int p = p0 + RPT * rg + i;
            if (p < P) o[(long)p * outP] = make_float2(ar[i][j], ai[i][j]);
        }
    }
}

// Launches k_cgemm_tw: 64 x 32 CTA tiles (4 x 2 per thread) when P fills 64-row tiles, else
// 32 x 64 (2 x 4), or 32 x 32 when 64-column tiles would leave SMs idle. Static shared memory
// stays within 48 KB (two buffers of (PT + NT) x 32 complex).
static int cgemm_tw(const float2* M, int P, int Q, int C, long nslab, const float2* In, long inS,
                    long inQ, float2* Out, long outS, long outP, int qsplit, long outSplit,
                    const char* name, double bytes, cudaStream_t st) {
    const long N = nslab * C;
    if (N > 0x7fffffffL) {
        set_error("spectral: too many columns in a Y/Z stage");
        return LDDMM_EINVAL;
    }
    KTRACE(name, st, bytes, 8.0 * P * (double)Q * N);
    const unsigned nt64 = (unsigned)((N + 63) / 64), nt32 = (unsigned)((N + 31) / 32);
    if (P > 48) {
        dim3 grid(nt32, (P + 63) / 64, qsplit);
        k_cgemm_tw<4, 32><<<grid, 256, 0, st>>>(M, P, Q, C, (int)N, In, inS, inQ, Out, outS, outP, outSplit);
    } else if ((long)nt64 * ((P + 31) / 32) * qsplit >= 2 * 148) {
        dim3 grid(nt64, (P + 31) / 32, qsplit);
        k_cgemm_tw<2, 64><<<grid, 256, 0, st>>>(M, P, Q, C, (int)N, In, inS, inQ, Out, outS, outP, outSplit);
    } else {
        dim3 grid(nt32, (P + 31) / 32, qsplit);
        k_cgemm_tw<2, 32><<<grid, 256, 0, st>>>(M, P, Q, C, (int)N, In, inS, inQ, Out, outS, outP, outSplit);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// Sum of the z-block partials, 1/N normalisation, Hermitian mirror and zero slots.
__global__ void k_pi_z_fin(const float2* __restrict__ part, int ncomp, int K, int KH, int zsplit,
                           float inv_n, float2* __restrict__ c) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)ncomp * K * K * KH;
    if (i >= total) return;
    int kx = (int)(i % KH);
    long t = i / KH;
    int jy = (int)(t % K);
    t /= K;
    int jz = (int)(t % K);
    int comp = (int)(t / K);
    float re = 0.f, im = 0.f;
    if (jz >= 1 && jy >= 1) {
        const long stride = (long)ncomp * K * K * KH;
        const float2* p = part + (((long)comp * K + jz) * K + jy) * KH + kx;
        for (int sp = 0; sp < zsplit; ++sp) {
            float2 v = p[sp * stride];
            re += v.x;
            im += v.y;
        }
        re *= inv_n;
        im *= inv_n;
    }
    float2* cc = c + (long)comp * K * K * K;
    const int h = K / 2;
    cc[((long)jz * K + jy) * K + h + kx] = make_float2(re, im);
    if (kx >= 1) {
        if (jz >= 1 && jy >= 1)
            cc[((long)(K - jz) * K + (K - jy)) * K + h - kx] = make_float2(re, -im);
        else
            cc[((long)jz * K + jy) * K + h - kx] = make_float2(0.f, 0.f);
    } else {
        cc[((long)jz * K + jy) * K + 0] = make_float2(0.f, 0.f);
    }
}

template <int KHP>
static int launch_pi_x(const Grid& g, const Twiddles& tw, const float* f, long fstride, int ncomp,
                       float2* A, cudaStream_t st) {
    const int KH = tw.K / 2;
    const int nxp = (g.nx + 3) & ~3;
    size_t smem = (size_t)PX_ROWS * (nxp + 4) * 4 + (size_t)nxp * KHP * 8;
    if (smem > 227 * 1024) {
        set_error("bl_project: nx too large for the x stage");
        return LDDMM_EINVAL;
    }
    static bool attr_set = false;
    if (!attr_set) {
        LDDMM_CUDA(cudaFuncSetAttribute(k_pi_x<KHP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024));
        attr_set = true;
    }
    long rows = (long)g.nz * g.ny * ncomp;
    KTRACE("pi_x", st, rows * g.nx * 4.0 + rows * KH * 8.0, rows * g.nx * KH * 4.0);
    k_pi_x<KHP><<<cdiv(rows, PX_ROWS), KHP * 8, smem, st>>>(
        f, fstride, (long)g.nz * g.ny, ncomp, g.nx, KH, tw.K, tw.cx, tw.sx, A);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

static int check_spectral_shape(const Grid& g, int K) {
    if (g.nx < 2 || g.ny < 2 || g.nz < 2 || K < 4 || (K & 1) || K > 64 || K > g.nx ||
        K > g.ny || K > g.nz || g.nx > 1024 || g.ny > 1024) {
        set_error("spectral: need even 4 <= K <= min(64, nx, ny, nz) and nx, ny <= 1024");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

#define KHP_DISPATCH(KH, FN, ...)                                   \
    ((KH) <= 2 ? FN<2>(__VA_ARGS__) : (KH) <= 4 ? FN<4>(__VA_ARGS__) \
     : (KH) <= 8 ? FN<8>(__VA_ARGS__) : (KH) <= 16 ? FN<16>(__VA_ARGS__) : FN<32>(__VA_ARGS__))

int bl_project(const Grid& g, const Twiddles& tw, const float* f, long fstride, int ncomp,
               float2* c, float2* s1, float2* s2, int precision, cudaStream_t st) {
    int rc = check_spectral_shape(g, tw.K);
    if (rc) return rc;
    const int K = tw.K, KH = K / 2;
    const long rows = (long)ncomp * g.nz * g.ny;
    const long nslab = (long)ncomp * g.nz;
    const int tp = precision == LDDMM_PREC_BF16X3 ? 1 : 0;
    const bool tcx = precision != LDDMM_PREC_FP32_SIMT && fstride == (long)g.nz * g.ny * g.nx &&
                     tc_rowgemm_supported(K, g.nx, rows, f, g.nx);
    const bool tcy = tcx && tw.tc_y && (reinterpret_cast<uintptr_t>(s1) & 15) == 0;
    if (tcy) {
        // stage X on the tensor cores, stored transposed per (comp, z) slab:
        // A[comp, z][2 kx + re/im][y], the K-major rows of the tensor-core Y stage; W as the
        // MMA's A operand (128 input rows per instruction) where it fits
        if (tc_rowgemm_t_supported(K, g.nx, rows, f, g.nx))
            rc = tc_rowgemm_t(f, rows, g.nx, g.nx, tw.wpi_img[tp], K, tp, reinterpret_cast<float*>(s1), g.ny,
                              K, "pi_x_tc", rows * g.nx * 4.0 + rows * K * 4.0, st);
        else
            rc = tc_rowgemm_ex(f, rows, g.nx, g.nx, tw.wpi_img[tp], K, tp, 1, reinterpret_cast<float*>(s1),
                               g.ny, 0, K, 0, 0, 0, 1, "pi_x_tc", rows * g.nx * 4.0 + rows * K * 4.0, st);
    } else if (tcx) {
        // stage X on the tensor cores: A[row][0..K) = (Re, Im) pairs of kx = 0..K/2-1
        rc = tc_rowgemm(f, rows, g.nx, g.nx, tw.wpi_img[tp], K, tp, reinterpret_cast<float*>(s1), rows, 0, K,
                        "pi_x_tc", rows * g.nx * 4.0 + rows * K * 4.0, st);
    } else {
        rc = KHP_DISPATCH(KH, launch_pi_x, g, tw, f, fstride, ncomp, s1, st);
    }
    if (rc) return rc;
    // stage Y: B[comp, z][jy][kx] = sum_y e^{-i ky y} A[comp, z][y][kx]
    if (tcy) {
        // rows (comp, z, kx, re/im) of ny floats against W[2 jy + {cos, sin}][y]
        rc = tc_rowgemm_ex(reinterpret_cast<const float*>(s1), nslab * K, g.ny, g.ny, tw.wpy_img[tp],
                           2 * K, tp, 2, reinterpret_cast<float*>(s2), K, 0, 2 * K, K, 0, KH, 1, "pi_y_tc",
                           (double)nslab * K * g.ny * 4.0 + (double)nslab * K * KH * 8.0, st);
        if (rc) return rc;
    } else {
        rc = cgemm_tw(tw.mpy, K, g.ny, KH, nslab, s1, (long)g.ny * KH, KH, s2, (long)K * KH, KH, 1, 0,
                      "pi_y", (double)nslab * (g.ny + K) * KH * 8.0, st);
        if (rc) return rc;
    }
    // stage Z: z-block partial sums part[split][comp][jz][col] into s1 (free after stage Y)
    const int zsplit = std::max(1, std::min(8, g.nz / K));
    {
        const long ncol = (long)K * KH;
        rc = cgemm_tw(tw.mpz, K, g.nz, (int)ncol, ncomp, s2, g.nz * ncol, ncol, s1, K * ncol, ncol, zsplit,
                      (long)ncomp * K * ncol, "pi_z",
                      (double)ncomp * g.nz * ncol * 8.0 + (double)zsplit * ncomp * K * ncol * 8.0, st);
        if (rc) return rc;
    }
    long total = (long)ncomp * K * K * KH;
    {
        KTRACE("pi_z_fin", st, (double)zsplit * total * 8.0 + (double)ncomp * K * K * K * 8.0, 0);
        k_pi_z_fin<<<cdiv(total, 256), 256, 0, st>>>(s1, ncomp, K, KH, zsplit,
                                                     (float)(1.0 / (double)g.ntot()), c);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ------------------------------------------------- iota stage Z (GEMM over all planes)
// T1[comp][z][j] = sum_{jz>=1} Ez[z][jz] * m(k) c[comp][jz][jy][K/2+kx],  j = jy*KH + kx,
// with m(k) the derivative / divergence multiplier and 1/B^(k) for B-spline coefficients.
// CTA tile: 32 planes x 32 columns; thread: ZPT planes x 2 columns (2 ZPT complex
// accumulators), 16 x 32 / ZPT threads. The stage is small and latency-bound, so fewer planes
// per thread (more resident warps) is faster.
constexpr int Z2_ZT = 32, Z2_JT = 32;
constexpr int IOTA_Z_ZPT = 1;

template <int ZPT>
__global__ void __launch_bounds__((Z2_JT / 2) * (Z2_ZT / ZPT))
k_iota_z2(const float2* __restrict__ c, int nz, int ny, int nx, int K, int KH, int deriv_axis,
          int bspline, const float* __restrict__ cxT, const float* __restrict__ cyT,
          const float* __restrict__ czT, const float* __restrict__ szT, float2* __restrict__ T1,
          int kmajor) {
    constexpr int NTH = (Z2_JT / 2) * (Z2_ZT / ZPT);
    __shared__ float4 cs4[32 * Z2_JT / 2];   // [jz][Z2_JT] float2 (K <= 64 -> 2 passes if K > 32)
    __shared__ float4 es4[32 * Z2_ZT / 2];   // [jz][Z2_ZT] float2
    float2* cs = reinterpret_cast<float2*>(cs4);
    float2* es = reinterpret_cast<float2*>(es4);
    const int comp = blockIdx.z;
    const int z0 = blockIdx.x * Z2_ZT, j0 = blockIdx.y * Z2_JT;
    const int KK = K * KH, h = K / 2;
    const int tid = threadIdx.x, jq = tid % (Z2_JT / 2), zq = tid / (Z2_JT / 2);
    float ar[ZPT][2], ai[ZPT][2];
#pragma unroll
    for (int a = 0; a < ZPT; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) ar[a][b] = ai[a][b] = 0.f;
    const long kk3 = (long)K * K * K;
    for (int jzb = 0; jzb < K; jzb += 32) {
        const int nj = min(32, K - jzb);
        __syncthreads();
        for (int e = tid; e < 32 * Z2_JT; e += NTH) {
            const int jzl = e / Z2_JT, jj = e - jzl * Z2_JT;
            const int jz = jzb + jzl, j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (jzl < nj && jz >= 1 && j < KK) {
                // column j: (jy, kx) = (j / KH, j % KH), or kx-major (kx, jy) = (j / K, j % K)
                // for the K-major store, so that a tile's columns are consecutive jy
                const int jy = kmajor ? j % K : j / KH;
                const int kx = kmajor ? j / K : j - jy * KH;
                if (jy >= 1) {
                    const long o = ((long)jz * K + jy) * K + h + kx;
                    const float kxf = (float)kx, kyf = (float)(jy - h), kzf = (float)(jz - h);
                    float vr, vi;
                    if (deriv_axis == 3) {
                        const float2 a0 = c[o], a1 = c[kk3 + o], a2 = c[2 * kk3 + o];
                        vr = -(kxf * a0.y + kyf * a1.y + kzf * a2.y);
                        vi = kxf * a0.x + kyf * a1.x + kzf * a2.x;
                    } else {
                        const float2 w = c[comp * kk3 + o];
                        if (deriv_axis < 0) {
                            vr = w.x;
                            vi = w.y;
                        } else {
                            const float k = deriv_axis == 0 ? kxf : deriv_axis == 1 ? kyf : kzf;
                            vr = -k * w.y;
                            vi = k * w.x;
                        }
                    }
                    if (bspline) {
                        const float b = 27.f / ((2.f + cxT[(long)(h + kx) * nx + 1]) *
                                                (2.f + cyT[(long)jy * ny + 1]) *
                                                (2.f + czT[(long)jz * nz + 1]));
                        vr *= b;
                        vi *= b;
                    }
                    v = make_float2(vr, vi);
                }
            }
            cs[e] = v;
        }
        for (int e = tid; e < 32 * Z2_ZT; e += NTH) {
            const int jzl = e / Z2_ZT, zz = e - jzl * Z2_ZT;
            const int jz = jzb + jzl, z = z0 + zz;
            es[e] = (jzl < nj && z < nz) ? make_float2(czT[(long)jz * nz + z], szT[(long)jz * nz + z])
                                         : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int jzl = 0; jzl < nj; ++jzl) {
            const float4 cv = *reinterpret_cast<const float4*>(&cs[jzl * Z2_JT + 2 * jq]);
            float2 ev[ZPT];
#pragma unroll
            for (int a = 0; a < ZPT; ++a) ev[a] = es[jzl * Z2_ZT + ZPT * zq + a];
            const float2 cw[2] = {make_float2(cv.x, cv.y), make_float2(cv.z, cv.w)};
#pragma unroll
            for (int a = 0; a < ZPT; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    // (e.x + i e.y)(c.x + i c.y)
                    ar[a][b] = fmaf(ev[a].x, cw[b].x, fmaf(-ev[a].y, cw[b].y, ar[a][b]));
                    ai[a][b] = fmaf(ev[a].x, cw[b].y, fmaf(ev[a].y, cw[b].x, ai[a][b]));
                }
        }
    }
#pragma unroll
    for (int a = 0; a < ZPT; ++a) {
        const int z = z0 + ZPT * zq + a;
        if (z >= nz) continue;
        if (kmajor) {
            // T1[comp][z][kx][re, im][jy] (floats): the K-major rows the tensor-core Y stage
            // reads; the warp's columns are consecutive jy of one kx (128-byte stores)
            float* dst = reinterpret_cast<float*>(T1) + ((long)comp * nz + z) * 2 * KK;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int j = j0 + 2 * jq + b;
                if (j < KK) {
                    const int kx = j / K, jy = j - kx * K;
                    dst[(2 * kx) * K + jy] = ar[a][b];
                    dst[(2 * kx + 1) * K + jy] = ai[a][b];
                }
            }
        } else {
            float2* dst = T1 + ((long)comp * nz + z) * KK + j0 + 2 * jq;
#pragma unroll
            for (int b = 0; b < 2; ++b)
                if (j0 + 2 * jq + b < KK) dst[b] = make_float2(ar[a][b], ai[a][b]);
        }
    }
}

static int launch_iota_zy2(const Grid& g, const Twiddles& tw, const float2* c, int nout,
                           int deriv_axis, int bspline, float2* T1, float2* T2, int tp,
                           bool tc_y, cudaStream_t st) {
    const int K = tw.K, KH = K / 2, KK = K * KH;
    {
        dim3 grid(cdiv(g.nz, Z2_ZT), cdiv(KK, Z2_JT), nout);
        KTRACE("iota_z", st, (double)(deriv_axis == 3 ? 3 : nout) * K * K * KH * 8.0 +
                                 (double)nout * g.nz * KK * 8.0,
               (double)nout * g.nz * KK * K * 8.0);
        k_iota_z2<IOTA_Z_ZPT><<<grid, (Z2_JT / 2) * (Z2_ZT / IOTA_Z_ZPT), 0, st>>>(
            c, g.nz, g.ny, g.nx, K, KH, deriv_axis, bspline, tw.cx, tw.cy, tw.cz, tw.sz, T1,
            tc_y ? 1 : 0);
    }
    LDDMM_CHECK_LAUNCH();
    // stage Y: T2[plane][y][kx] = sum_{jy >= 1} e^{+i ky y} T1[plane][jy][kx]
    const long nplanes = (long)nout * g.nz;
    if (tc_y) {
        // on the tensor cores: rows (plane, kx, re/im) of K floats against W[2y + {cos, sin}][jy],
        // the positions y in iy_blocks column blocks of one launch
        const int nyb = tw.iy_nyb;
        return tc_rowgemm_ex(reinterpret_cast<const float*>(T1), nplanes * K, K, K, tw.wiy_img[tp][0],
                             2 * nyb, tp, 3, reinterpret_cast<float*>(T2), K, 0, 2 * nyb, g.ny, 0, KH,
                             tw.iy_blocks, "iota_y_tc",
                             (double)nplanes * K * K * 4.0 + (double)nplanes * g.ny * KH * 8.0, st);
    }
    return cgemm_tw(tw.miy, g.ny, K, KH, nplanes, T1, (long)K * KH, KH, T2, (long)g.ny * KH, KH, 1, 0,
                    "iota_y", (double)nplanes * (K + g.ny) * KH * 8.0, st);
}

// ---------------------------------------------------------------------- iota, stage X
// f[row][x] = Re T[row][0] + 2 sum_{kx>=1} Re(T[row][kx] e^{i kx 2pi x/nx}).
// CTA: IX_ROWS rows x all x. Warp tile: 16 rows x 32 x; lane -> (row lane rl = lane/8,
// x group xl = lane%8), thread rows {16 i + 4 wr + rl}, x = 4 (8 wx + xl) .. +3.
constexpr int IX_ROWS = 64;

template <int KHP>
__global__ void __launch_bounds__(256)
k_iota_x(const float2* __restrict__ T, long rows_per_comp, int ncomp, int nx, int KH, int K,
         const float* __restrict__ cosT, const float* __restrict__ sinT, float* __restrict__ f,
         long fstride) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int nxp = (nx + 31) & ~31;
    float* tc = sm;                       // KHP * nxp
    float* ts = tc + KHP * nxp;           // KHP * nxp
    float2* co = reinterpret_cast<float2*>(ts + KHP * nxp);  // IX_ROWS * (KHP + 1)
    const int ldc = KHP + 1;
    const int tid = threadIdx.x;
    const long rows = rows_per_comp * ncomp;
    const long row0 = (long)blockIdx.x * IX_ROWS;

    for (int e = tid; e < KHP * nxp; e += 256) {
        int kx = e / nxp, x = e - kx * nxp;
        float c = 0.f, s = 0.f;
        if (kx < KH && x < nx) {
            long o = (long)(K / 2 + kx) * nx + x;
            float w = kx == 0 ? 1.f : 2.f;
            c = w * cosT[o];
            s = w * sinT[o];
        }
        tc[e] = c;
        ts[e] = s;
    }
    for (int e = tid; e < IX_ROWS * KHP; e += 256) {
        int r = e / KHP, kx = e - r * KHP;
        long row = row0 + r;
        float2 v = make_float2(0.f, 0.f);
        if (row < rows && kx < KH) {
            v = T[row * KH + kx];
            if (kx == 0) v.y = 0.f;
        }
        co[r * ldc + kx] = v;
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int rl = lane >> 3, xl = lane & 7;
    const int wtiles_x = nxp / 32;
    const int wtiles = 4 * wtiles_x;  // 4 row blocks of 16 rows
    for (int wt = warp; wt < wtiles; wt += 8) {
        const int wr = wt % 4, wx = wt / 4;
        const int x0 = 4 * (8 * wx + xl);
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
        for (int kx = 0; kx < KHP; ++kx) {
            float4 c4 = *reinterpret_cast<const float4*>(&tc[kx * nxp + x0]);
            float4 s4 = *reinterpret_cast<const float4*>(&ts[kx * nxp + x0]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 ab = co[(16 * i + 4 * wr + rl) * ldc + kx];
                acc[i][0] = fmaf(ab.x, c4.x, fmaf(-ab.y, s4.x, acc[i][0]));
                acc[i][1] = fmaf(ab.x, c4.y, fmaf(-ab.y, s4.y, acc[i][1]));
                acc[i][2] = fmaf(ab.x, c4.z, fmaf(-ab.y, s4.z, acc[i][2]));
                acc[i][3] = fmaf(ab.x, c4.w, fmaf(-ab.y, s4.w, acc[i][3]));
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            long row = row0 + 16 * i + 4 * wr + rl;
            if (row >= rows) continue;
            long comp = row / rows_per_comp;
            float* dst = f + comp * fstride + (row - comp * rows_per_comp) * nx;
            if (x0 + 3 < nx && (nx & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                __stcs(reinterpret_cast<float4*>(dst + x0),
                       make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (x0 + q < nx) dst[x0 + q] = acc[i][q];
            }
        }
    }
}

template <int KHP>
static int launch_iota_x(const Grid& g, const Twiddles& tw, const float2* T, int ncomp, float* f,
                         long fstride, cudaStream_t st) {
    const int nxp = (g.nx + 31) & ~31;
    size_t smem = (size_t)2 * KHP * nxp * 4 + (size_t)IX_ROWS * (KHP + 1) * 8;
    if (smem > 227 * 1024) {
        set_error("bl_include: nx too large for the x stage");
        return LDDMM_EINVAL;
    }
    static bool attr_set = false;
    if (!attr_set) {
        LDDMM_CUDA(cudaFuncSetAttribute(k_iota_x<KHP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set = true;
    }
    long rows = (long)g.nz * g.ny * ncomp;
    KTRACE("iota_x", st, rows * (tw.K / 2) * 8.0 + rows * g.nx * 4.0, rows * g.nx * (tw.K / 2) * 4.0);
    k_iota_x<KHP><<<cdiv(rows, IX_ROWS), 256, smem, st>>>(T, (long)g.nz * g.ny, ncomp, g.nx,
                                                         tw.K / 2, tw.K, tw.cx, tw.sx, f, fstride);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int bl_include(const Grid& g, const Twiddles& tw, const float2* c, int ncomp, float* f,
               long fstride, int deriv_axis, int bspline, float2* s1, float2* s2,
               int precision, cudaStream_t st) {
    int rc = check_spectral_shape(g, tw.K);
    if (rc) return rc;
    if (deriv_axis < -1 || deriv_axis > 3 || (deriv_axis == 3 && ncomp != 3)) {
        set_error("bl_include: deriv_axis must be -1..2, or 3 (divergence) with ncomp = 3");
        return LDDMM_EINVAL;
    }
    const int K = tw.K, KH = K / 2;
    const int nout = deriv_axis == 3 ? 1 : ncomp;
    const long rows = (long)nout * g.nz * g.ny;
    const bool tcx = precision != LDDMM_PREC_FP32_SIMT && tc_rowgemm_supported(g.nx, K, rows, s1, K);
    const bool tcy = tcx && tw.tc_y && (reinterpret_cast<uintptr_t>(s2) & 15) == 0;
    const int tp = precision == LDDMM_PREC_BF16X3 ? 1 : 0;
    // stage Z into s2, stage Y into s1
    int rc2 = launch_iota_zy2(g, tw, c, nout, deriv_axis, bspline ? 1 : 0, s2, s1, tp, tcy, st);
    if (rc2) return rc2;
    if (tcx) {
        // stage X on the tensor cores: f[row][x] = sum_j T[row][j] W_io[x][j]
        return tc_rowgemm(reinterpret_cast<const float*>(s1), rows, K, K, tw.wio_img[tp], g.nx, tp, f,
                          (long)g.nz * g.ny, fstride, g.nx, "iota_x_tc",
                          rows * K * 4.0 + rows * g.nx * 4.0, st);
    }
    return KHP_DISPATCH(KH, launch_iota_x, g, tw, s1, nout, f, fstride, st);
}

// ------------------------------------------------------------------------ cube kernels
__global__ void k_cube_axpby(float2* out, float a, const float2* x, float b, const float2* y,
                             long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 r = make_float2(0.f, 0.f);
    if (x) { float2 v = x[i]; r.x = a * v.x; r.y = a * v.y; }
    if (y) { float2 v = y[i]; r.x = fmaf(b, v.x, r.x); r.y = fmaf(b, v.y, r.y); }
    out[i] = r;
}

int cube_axpby(float2* out, float a, const float2* x, float b, const float2* y, long n,
               cudaStream_t st) {
    KTRACE("cube_axpby", st, 24.0 * n, 4.0 * n);
    k_cube_axpby<<<cdiv(n, 256), 256, 0, st>>>(out, a, x, b, y, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_cube_L(float2* out, const float2* x, float wL, float a, const float2* y, int K,
                         long n, double alpha, int s, int mode) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int jx = (int)(i % K), jy = (int)((i / K) % K), jz = (int)((i / ((long)K * K)) % K);
    const int h = K / 2;
    float2 r = make_float2(0.f, 0.f);
    if (jx >= 1 && jy >= 1 && jz >= 1) {
        double k2 = (double)(jx - h) * (jx - h) + (double)(jy - h) * (jy - h) +
                    (double)(jz - h) * (jz - h);
        double base = 1.0 + alpha * k2, w = 1.0;
        for (int e = 0; e < s; ++e) w *= base;
        float f = (float)(mode > 0 ? w : 1.0 / w) * wL;
        float2 v = x[i];
        r = make_float2(f * v.x, f * v.y);
        if (y && mode > 0) {
            float2 u = y[i];
            r.x = fmaf(a, u.x, r.x);
            r.y = fmaf(a, u.y, r.y);
        }
    }
    out[i] = r;
}

int cube_apply_L(float2* out, const float2* x, float wL, float a, const float2* y, int K,
                 int ncomp, double alpha, int s, int mode, cudaStream_t st) {
    long n = (long)ncomp * K * K * K;
    KTRACE("cube_L", st, 24.0 * n, 4.0 * n);
    k_cube_L<<<cdiv(n, 256), 256, 0, st>>>(out, x, wL, a, y, K, n, alpha, s, mode);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

__global__ void k_cube_hermitian(float2* c, int K, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long kk = (long)K * K * K;
    long comp = i / kk;
    long r = i - comp * kk;
    int jx = (int)(r % K), jy = (int)((r / K) % K), jz = (int)(r / ((long)K * K));
    if (jx == 0 || jy == 0 || jz == 0) { c[i] = make_float2(0.f, 0.f); return; }
    long m = comp * kk + ((long)(K - jz) * K + (K - jy)) * K + (K - jx);
    if (m < i) return;  // the lower index of each pair does the work
    float2 a = c[i], b = c[m];
    float2 h = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    c[i] = h;
    c[m] = make_float2(h.x, -h.y);
}

int cube_hermitian(float2* c, int K, int ncomp, cudaStream_t st) {
    long n = (long)ncomp * K * K * K;
    KTRACE("cube_hermitian", st, 16.0 * n, 0);
    k_cube_hermitian<<<cdiv(n, 256), 256, 0, st>>>(c, K, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// --------------------------------------------------------- coarse band (two-level PCG)
// Coarse band S_c = {|k|_inf <= Kc/2 - 1} of a band-K cube: fine slot j holds k = j - K/2,
// coarse slot jc holds k = jc - Kc/2, so jc = j - (K - Kc)/2; coarse slot 0 is never filled.

// R: coarse[c][jz][jy][jx] = fine[c][jz + o][jy + o][jx + o] (o = (K - Kc)/2), 0 on slot 0
__global__ void k_cube_restrict(const float2* __restrict__ fine, int K, float2* __restrict__ coarse,
                                int Kc, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long kk = (long)Kc * Kc * Kc;
    const long comp = i / kk, r = i - comp * kk;
    const int jx = (int)(r % Kc), jy = (int)((r / Kc) % Kc), jz = (int)(r / ((long)Kc * Kc));
    float2 v = make_float2(0.f, 0.f);
    if (jx >= 1 && jy >= 1 && jz >= 1) {
        const int o = (K - Kc) / 2;
        v = fine[comp * K * K * K + ((long)(jz + o) * K + (jy + o)) * K + (jx + o)];
    }
    coarse[i] = v;
}

// z <- E y on the coarse band, theta z elsewhere (z holds L~^{-1} r on entry)
__global__ void k_cube_two_level(float2* __restrict__ z, int K, const float2* __restrict__ y, int Kc,
                                 float theta, long n) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long kk = (long)K * K * K;
    const long comp = i / kk, r = i - comp * kk;
    const int o = (K - Kc) / 2;
    const int jx = (int)(r % K) - o, jy = (int)((r / K) % K) - o, jz = (int)(r / ((long)K * K)) - o;
    if (jx >= 1 && jy >= 1 && jz >= 1 && jx < Kc && jy < Kc && jz < Kc) {
        z[i] = y[comp * Kc * Kc * Kc + ((long)jz * Kc + jy) * Kc + jx];
    } else {
        const float2 v = z[i];
        z[i] = make_float2(theta * v.x, theta * v.y);
    }
}

int cube_restrict(const float2* fine, int K, float2* coarse, int Kc, int ncomp, cudaStream_t st) {
    if (Kc < 2 || Kc > K || (Kc & 1) || (K & 1)) {
        set_error("cube_restrict: need even 2 <= Kc <= K");
        return LDDMM_EINVAL;
    }
    const long n = (long)ncomp * Kc * Kc * Kc;
    KTRACE("cube_restrict", st, 16.0 * n, 0);
    k_cube_restrict<<<cdiv(n, 256), 256, 0, st>>>(fine, K, coarse, Kc, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int cube_two_level(float2* z, int K, const float2* y, int Kc, float theta, int ncomp, cudaStream_t st) {
    if (Kc < 2 || Kc > K || (Kc & 1) || (K & 1)) {
        set_error("cube_two_level: need even 2 <= Kc <= K");
        return LDDMM_EINVAL;
    }
    const long n = (long)ncomp * K * K * K;
    KTRACE("cube_two_level", st, 16.0 * n, 2.0 * n);
    k_cube_two_level<<<cdiv(n, 256), 256, 0, st>>>(z, K, y, Kc, theta, n);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// ------------------------------------------------------------------- FP64 reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <bool MAX>
__device__ void block_reduce_store(double v, double* out) {
    __shared__ double part[32];
    v = MAX ? warp_max(v) : warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        v = lane < nw ? part[lane] : 0.0;
        v = MAX ? warp_max(v) : warp_sum(v);
        if (lane == 0) *out = v;
    }
}

__global__ void k_dot_f2(const float2* a, const float2* b, long n, double* partials) {
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float2 x = a[i], y = b[i];
        s += (double)x.x * y.x + (double)x.y * y.y;
    }
    block_reduce_store<false>(s, partials + blockIdx.x);
}

// sum over nodes j of w_j <a_j, b_j>, a_j the j-th block of npn elements; w_j the trapezoid
// weights of nodes 0..nodes-1 with step dt (nodes == 1: weight 1)
__global__ void k_dot_f2_nodes(const float2* a, const float2* b, long npn, int nodes, double dt,
                               double* partials) {
    double s = 0.0;
    const long n = npn * nodes;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int j = (int)(i / npn);
        const double w = nodes == 1 ? 1.0 : (j == 0 || j == nodes - 1) ? 0.5 * dt : dt;
        float2 x = a[i], y = b[i];
        s += w * ((double)x.x * y.x + (double)x.y * y.y);
    }
    block_reduce_store<false>(s, partials + blockIdx.x);
}

__global__ void k_maxabs_f2(const float2* a, long n, double* partials) {
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float2 x = a[i];
        s = fmax(s, sqrt((double)x.x * x.x + (double)x.y * x.y));
    }
    block_reduce_store<true>(s, partials + blockIdx.x);
}

__global__ void k_finalize(const double* partials, int n, double* out, int is_max) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        s = is_max ? fmax(s, partials[i]) : s + partials[i];
    if (is_max) block_reduce_store<true>(s, out);
    else block_reduce_store<false>(s, out);
}

int dot_f2(const float2* a, const float2* b, long n, double* partials, double* out,
           cudaStream_t st) {
    {
        KTRACE("dot_f2", st, 16.0 * n, 4.0 * n);
        k_dot_f2<<<kReduceBlocks, 256, 0, st>>>(a, b, n, partials);
    }
    LDDMM_CHECK_LAUNCH();
    KTRACE("finalize", st, 8.0 * kReduceBlocks, kReduceBlocks);
    k_finalize<<<1, 256, 0, st>>>(partials, kReduceBlocks, out, 0);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int dot_f2_nodes(const float2* a, const float2* b, long npn, int nodes, double dt,
                 double* partials, double* out, cudaStream_t st) {
    {
        KTRACE("dot_f2", st, 16.0 * npn * nodes, 5.0 * npn * nodes);
        k_dot_f2_nodes<<<kReduceBlocks, 256, 0, st>>>(a, b, npn, nodes, dt, partials);
    }
    LDDMM_CHECK_LAUNCH();
    KTRACE("finalize", st, 8.0 * kReduceBlocks, kReduceBlocks);
    k_finalize<<<1, 256, 0, st>>>(partials, kReduceBlocks, out, 0);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int max_abs_f2(const float2* a, long n, double* partials, double* out, cudaStream_t st) {
    {
        KTRACE("maxabs_f2", st, 8.0 * n, 3.0 * n);
        k_maxabs_f2<<<kReduceBlocks, 256, 0, st>>>(a, n, partials);
    }
    LDDMM_CHECK_LAUNCH();
    KTRACE("finalize", st, 8.0 * kReduceBlocks, kReduceBlocks);
    k_finalize<<<1, 256, 0, st>>>(partials, kReduceBlocks, out, 1);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// max over voxels of |(s0 u0, s1 u1, s2 u2)| for a 3-plane field u (a displacement in voxels)
__global__ void k_max_norm3(const float* __restrict__ u, long n, float s0, float s1, float s2,
                            double* partials) {
    double m = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double a = (double)u[i] * s0, b = (double)u[n + i] * s1, c = (double)u[2 * n + i] * s2;
        m = fmax(m, sqrt(a * a + b * b + c * c));
    }
    block_reduce_store<true>(m, partials + blockIdx.x);
}

int max_norm3(const float* u, long n, const float s[3], double* partials, double* out, cudaStream_t st) {
    {
        KTRACE("max_norm3", st, 12.0 * n, 8.0 * n);
        k_max_norm3<<<kReduceBlocks, 256, 0, st>>>(u, n, s[0], s[1], s[2], partials);
    }
    LDDMM_CHECK_LAUNCH();
    KTRACE("finalize", st, 8.0 * kReduceBlocks, kReduceBlocks);
    k_finalize<<<1, 256, 0, st>>>(partials, kReduceBlocks, out, 1);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

int finalize_sum(const double* partials, int n, double* out, cudaStream_t st) {
    KTRACE("finalize", st, 8.0 * n, n);
    k_finalize<<<1, 256, 0, st>>>(partials, n, out, 0);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

}  // namespace lddmm
