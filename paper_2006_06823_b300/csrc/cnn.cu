// Learned Gauss-Newton warm start: a 3-D convolutional encoder-decoder that maps the
// (template, reference) pair, band-limited and resampled to D^3 (D = 64), to a velocity on
// the (D/2)^3 grid, whose exact band-limited projection is the solver's initial velocity.
// The paper has no learned component; the Gauss-Newton-Krylov solver always finishes the
// registration and measures the prediction by its own residual.
//
// Layers (base c channels): D^3: conv 2->c, c->c; pool; (D/2)^3: c->2c, 2c->2c; pool;
// (D/4)^3: 2c->4c, 4c->4c; pool; (D/8)^3: 4c->8c, 8c->8c; up; (D/4)^3: [8c up | 4c skip]
// -> 4c, 4c->4c; up; (D/2)^3: [4c up | 2c skip] -> 2c, 2c->2c, 2c->3 (no activation).
// 3x3x3 convolutions with zero padding and ReLU, 2x average pooling, 2x nearest upsampling.
//
// Storage: weights and activations BF16; master weights, gradients and Adam moments FP32;
// every sum accumulates in FP32. A convolution is an implicit GEMM
//   out[co][x] = b[co] + sum_{ci, t} W[co][ci*27 + t] in[ci][x + o(t)],
// tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) for o(t) = (dz, dy, dx) in {-1,0,1}^3. The input
// gradient is the same kernel run on the transposed, tap-flipped weights
// (Wt[ci][co*27 + 26 - t] = W[co][ci*27 + t], since o(26 - t) = -o(t)); the weight gradient
// is a split-K GEMM over voxels with FP32 atomics.
#include "common.cuh"
#include "lddmm.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

namespace lddmm {

static inline int cdiv_i(long a, long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ float ld_f(const float* p) { return *p; }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st_f(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_f(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// value of im2col row k = ci*27 + t at voxel (z, y, x) of a D^3 volume (zero outside)
template <typename TI>
__device__ __forceinline__ float im2col(const TI* __restrict__ in, long nv, int lgD, int k,
                                        int z, int y, int x) {
    const int ci = k / 27, t = k - 27 * ci;
    const int tz = t / 9, r = t - 9 * tz, ty = r / 3, tx = r - 3 * ty;
    const int zz = z + tz - 1, yy = y + ty - 1, xx = x + tx - 1;
    const unsigned D = 1u << lgD;
    if ((unsigned)zz >= D || (unsigned)yy >= D || (unsigned)xx >= D) return 0.f;
    return ld_f(in + (long)ci * nv + ((((long)zz << lgD) + yy) << lgD) + xx);
}

// ------------------------------------------------------------------ implicit-GEMM conv
// CTA tile: 64 output channels x 64 voxels, K chunks of 16; 4 x 4 outputs per thread.
constexpr int CV_M = 64, CV_N = 64, CV_K = 16;

template <typename TI, typename TW, typename TO, bool RELU>
__global__ void __launch_bounds__(256)
k_conv(const TI* __restrict__ in, int cin, int lgD, long in_bstride,
       const TW* __restrict__ W, const float* __restrict__ bias, int cout,
       TO* __restrict__ out, long out_bstride, int out_coff) {
    __shared__ __align__(16) float As[CV_K][CV_M + 4];
    __shared__ __align__(16) float Bs[CV_K][CV_N + 4];
    const int b = blockIdx.z;
    const int co0 = blockIdx.y * CV_M;
    const long nv = 1L << (3 * lgD);
    const long v0 = (long)blockIdx.x * CV_N;
    const int Kdim = cin * 27;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const TI* inb = in + (long)b * in_bstride;
    // this thread's im2col voxel (fixed over the K loop)
    const int nn = tid & 63;
    const long vb = v0 + nn;
    const bool vok = vb < nv;
    const int D = 1 << lgD;
    const int bx = (int)(vb & (D - 1)), by = (int)((vb >> lgD) & (D - 1)), bz = (int)(vb >> (2 * lgD));
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < Kdim; k0 += CV_K) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;  // 0 .. 1023
            {   // A: W[co0 + m][k0 + kk], consecutive threads along k
                const int m = e >> 4, kk = e & 15;
                const int co = co0 + m, k = k0 + kk;
                As[kk][m] = (co < cout && k < Kdim) ? ld_f(W + (long)co * Kdim + k) : 0.f;
            }
            {   // B: im2col rows k0 + (tid >> 6) + 4 r at this thread's voxel
                const int kk = (tid >> 6) + 4 * r;
                const int k = k0 + kk;
                Bs[kk][nn] = (vok && k < Kdim) ? im2col(inb, nv, lgD, k, bz, by, bx) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CV_K; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
            const float4 bb = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
    TO* outb = out + (long)b * out_bstride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + 4 * ty + i;
        if (co >= cout) continue;
        const float bi = bias ? bias[co] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long v = v0 + 4 * tx + j;
            if (v >= nv) continue;
            float r = acc[i][j] + bi;
            if (RELU) r = fmaxf(r, 0.f);
            st_f(outb + (long)(out_coff + co) * nv + v, r);
        }
    }
}

// dW[co][k] += sum over this CTA's voxel slice (all samples) of dout[b][co][v] im2col_k(in)[b][v].
// CTA tile: 64 channels x 64 k, chunks of 16 voxels of the flattened [B][D^3] index;
// gridDim.z slices of the B * D^3 voxels.
template <typename TI>
__global__ void __launch_bounds__(256)
k_conv_wgrad(const float* __restrict__ dout, int cout, long dout_bstride,
             const TI* __restrict__ in, int cin, long in_bstride, int lgD, int B,
             float* __restrict__ dW) {
    __shared__ __align__(16) float As[16][CV_M + 4];
    __shared__ __align__(16) float Bs[16][CV_N + 4];
    const int co0 = blockIdx.y * CV_M, k0 = blockIdx.x * CV_N;
    const long nv = 1L << (3 * lgD);
    const long total = nv * B;
    const long chunk = ((total + gridDim.z - 1) / gridDim.z + 15) & ~15L;
    const long s0 = (long)blockIdx.z * chunk, s1 = min(total, s0 + chunk);
    const int Kdim = cin * 27;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int D = 1 << lgD;
    const int vv = tid & 15;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (long s = s0; s < s1; s += 16) {
        const long sv = s + vv;
        const int b = (int)(sv / nv);
        const long v = sv - (long)b * nv;
        const bool ok = sv < s1;
        const int x = (int)(v & (D - 1)), y = (int)((v >> lgD) & (D - 1)), z = (int)(v >> (2 * lgD));
        const float* db = dout + (long)b * dout_bstride;
        const TI* ib = in + (long)b * in_bstride;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = (tid >> 4) + 16 * r;
            As[vv][m] = (ok && co0 + m < cout) ? db[(long)(co0 + m) * nv + v] : 0.f;
            const int k = k0 + m;
            Bs[vv][m] = (ok && k < Kdim) ? im2col(ib, nv, lgD, k, z, y, x) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(&As[q][4 * ty]);
            const float4 bb = *reinterpret_cast<const float4*>(&Bs[q][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + 4 * ty + i;
        if (co >= cout) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + 4 * tx + j;
            if (k < Kdim) atomicAdd(dW + (long)co * Kdim + k, acc[i][j]);
        }
    }
}

// db[co] += sum over b, v of dout[b][co][v]; grid (cout, slices), one FP32 atomic per CTA
__global__ void __launch_bounds__(256)
k_bias_grad(const float* __restrict__ dout, long nv, int B, long bstride, float* __restrict__ db) {
    const int co = blockIdx.x;
    const long total = nv * B;
    const long chunk = (total + gridDim.y - 1) / gridDim.y;
    const long s0 = (long)blockIdx.y * chunk, s1 = min(total, s0 + chunk);
    float s = 0.f;
    for (long i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const long b = i / nv;
        s += dout[b * bstride + (long)co * nv + (i - b * nv)];
    }
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(db + co, red[0]);
}

// storage copies of a layer's weights: Wb = W, Wt = transposed and tap-flipped W
template <typename TA>
__global__ void k_weights(const float* __restrict__ W, int cout, int cin, TA* __restrict__ Wb,
                          TA* __restrict__ Wt) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)cout * cin * 27) return;
    const int t = (int)(i % 27);
    const long r = i / 27;
    const int ci = (int)(r % cin), co = (int)(r / cin);
    st_f(Wb + i, W[i]);
    st_f(Wt + ((long)ci * cout + co) * 27 + (26 - t), W[i]);
}

// ------------------------------------------------------------------ small layers
// 2x average pool: out[b][c] (d^3) from in[b][in_coff + c] ((2d)^3)
template <typename TA>
__global__ void k_pool2(const TA* __restrict__ in, long in_bstride, int in_coff, int C, int d,
                        TA* __restrict__ out, long out_bstride) {
    const int b = blockIdx.y, D = 2 * d;
    const long n = (long)C * d * d * d;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int X = (int)(i % d), Y = (int)((i / d) % d), Z = (int)((i / ((long)d * d)) % d);
        const int c = (int)(i / ((long)d * d * d));
        const TA* p = in + (long)b * in_bstride + (long)(in_coff + c) * D * D * D;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            s += ld_f(p + ((long)(2 * Z + (q >> 2)) * D + 2 * Y + ((q >> 1) & 1)) * D + 2 * X + (q & 1));
        st_f(out + (long)b * out_bstride + i, 0.125f * s);
    }
}

// pool gradient: dst[b][dst_coff + c][x] += src[b][c][x / 2] / 8   (dst (2d)^3, src d^3)
__global__ void k_pool2_grad(const float* __restrict__ src, long src_bstride, int C, int d,
                             float* __restrict__ dst, long dst_bstride, int dst_coff) {
    const int b = blockIdx.y, D = 2 * d;
    const long n = (long)C * D * D * D;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)((i / ((long)D * D)) % D);
        const int c = (int)(i / ((long)D * D * D));
        const float g = src[(long)b * src_bstride + (((long)c * d + z / 2) * d + y / 2) * d + x / 2];
        dst[(long)b * dst_bstride + (long)dst_coff * D * D * D + i] += 0.125f * g;
    }
}

// 2x nearest upsample: out[b][out_coff + c][x] ((2d)^3) = in[b][c][x / 2] (d^3)
template <typename TA>
__global__ void k_up2(const TA* __restrict__ in, long in_bstride, int C, int d,
                      TA* __restrict__ out, long out_bstride, int out_coff) {
    const int b = blockIdx.y, D = 2 * d;
    const long n = (long)C * D * D * D;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)((i / ((long)D * D)) % D);
        const int c = (int)(i / ((long)D * D * D));
        out[(long)b * out_bstride + (long)out_coff * D * D * D + i] =
            in[(long)b * in_bstride + (((long)c * d + z / 2) * d + y / 2) * d + x / 2];
    }
}

// upsample gradient: dst[b][c][X] (d^3) = sum of the 8 src[b][src_coff + c][2X + q] ((2d)^3)
__global__ void k_up2_grad(const float* __restrict__ src, long src_bstride, int src_coff, int C,
                           int d, float* __restrict__ dst, long dst_bstride) {
    const int b = blockIdx.y, D = 2 * d;
    const long n = (long)C * d * d * d;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int X = (int)(i % d), Y = (int)((i / d) % d), Z = (int)((i / ((long)d * d)) % d);
        const int c = (int)(i / ((long)d * d * d));
        const float* p = src + (long)b * src_bstride + (long)(src_coff + c) * D * D * D;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            s += p[((long)(2 * Z + (q >> 2)) * D + 2 * Y + ((q >> 1) & 1)) * D + 2 * X + (q & 1)];
        dst[(long)b * dst_bstride + i] = s;
    }
}

// ReLU backward in place: g[b][i] = 0 where act[b][i] <= 0 (act is the layer's ReLU output)
template <typename TA>
__global__ void k_relu_mask(float* __restrict__ g, long g_bstride, const TA* __restrict__ act,
                            long a_bstride, long n_per_b) {
    const int b = blockIdx.y;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_per_b; i += (long)gridDim.x * blockDim.x)
        if (!(ld_f(act + (long)b * a_bstride + i) > 0.f)) g[(long)b * g_bstride + i] = 0.f;
}

template <typename TA>
__global__ void k_to_storage(const float* __restrict__ in, TA* __restrict__ out, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        st_f(out + i, in[i]);
}

// MSE: per-block partial sums of (y - t)^2 (FP64) and dy = 2 (y - t) / n
__global__ void __launch_bounds__(256)
k_mse(const float* __restrict__ y, const float* __restrict__ t, long n, float* __restrict__ dy,
      double* __restrict__ partials) {
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)d * d;
        dy[i] = 2.f * d / (float)n;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; c1, c2 = bias corrections 1 - beta^t
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace lddmm

using namespace lddmm;

// ==================================================================== network object
namespace {

struct Layer {
    int cin, cout, D;  // D: spatial size of the layer's input and output
    bool relu;
    long woff, boff;   // offsets of W [cout][cin*27] and b [cout] in the flat parameter vector
};

}  // namespace

struct lddmm_net {
    int D = 64, c = 16, bmax = 1, storage = LDDMM_NET_BF16;
    size_t esz = 2;  // bytes per stored weight / activation
    cudaStream_t st = nullptr;
    std::vector<Layer> L;
    long nparam = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;  // FP32 params, grads, Adam
    void *Wb = nullptr, *Wt = nullptr;                             // stored weights, flipped
    long adam_t = 0;
    // stored activations [bmax][C][d^3]; the skip concatenations cat1 = [up(d2) | e1] and
    // cat2 = [up(e3) | e2] are written in place by their producers
    void *x = nullptr, *a0a = nullptr, *a0b = nullptr, *p0 = nullptr, *a1a = nullptr, *cat1 = nullptr,
         *p1 = nullptr, *a2a = nullptr, *cat2 = nullptr, *p2 = nullptr, *a3a = nullptr, *a3b = nullptr,
         *a4a = nullptr, *a4b = nullptr, *a5a = nullptr, *a5b = nullptr;
    // FP32 output and gradients
    float *y = nullptr, *gA = nullptr, *gB = nullptr, *gC = nullptr, *gcat1 = nullptr,
          *gcat2 = nullptr;
    double* partials = nullptr;
    double* hpart = nullptr;
    // warm-start staging: network input [2][D^3] FP32 and one D^3 coefficient cube
    float *xin = nullptr, *cube = nullptr;
    std::vector<void*> allocs;
};

namespace {

int nalloc(lddmm_net* n, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        *p = nullptr;
        return LDDMM_ENOMEM;
    }
    n->allocs.push_back(*p);
    return LDDMM_OK;
}
template <class T>
int nalloc_t(lddmm_net* n, T** p, size_t count) {
    return nalloc(n, reinterpret_cast<void**>(p), count * sizeof(T));
}

long vol(int D) { return (long)D * D * D; }
int lg2(int D) { return 31 - __builtin_clz((unsigned)D); }

#define NTRY(...)                          \
    do {                                   \
        int rc__ = (__VA_ARGS__);          \
        if (rc__ != LDDMM_OK) return rc__; \
    } while (0)

int elem_grid(long n) { return std::max(1, std::min(cdiv_i(n, 256), 8192)); }

// Typed view of the network's stored tensors (TA = __nv_bfloat16 or float).
template <typename TA>
struct Net {
    lddmm_net* n;
    TA* a(void* p) const { return static_cast<TA*>(p); }
    TA* W(int i) const { return a(n->Wb) + n->L[i].woff; }
    TA* Wt(int i) const { return a(n->Wt) + n->L[i].woff; }
    const float* bias(int i) const { return n->P + n->L[i].boff; }
    float* gw(int i) const { return n->G + n->L[i].woff; }
    float* gb(int i) const { return n->G + n->L[i].boff; }

    // the convolutions run on the tensor cores for BF16 storage (the default) and the FP32
    // tensor-core check form; FP32 storage and LDDMM_NET_BF16_SIMT keep the FP32 SIMT kernels
    bool use_tc() const {
        return n->storage == LDDMM_NET_BF16 || n->storage == LDDMM_NET_FP32_TC;
    }

    template <typename TI, typename TO>
    int conv(const TI* in, int cin, int D, long in_bs, const TA* Wm, const float* b, int cout, TO* out,
             long out_bs, int out_coff, bool relu, int B, const char* name) const {
        dim3 grid(cdiv_i(vol(D), CV_N), cdiv_i(cout, CV_M), B);
        KTRACE(name, n->st,
               (double)B * vol(D) * (cin * sizeof(TI) + cout * sizeof(TO)) + cout * cin * 27.0 * sizeof(TA),
               2.0 * B * vol(D) * cin * 27.0 * cout);
        if (use_tc() && tc_conv_supported(cout, D, false))
            return tc_conv<TI, TA, TO>(in, cin, D, in_bs, Wm, b, cout, out, out_bs, out_coff, relu, B, n->st);
        if (relu)
            k_conv<TI, TA, TO, true><<<grid, 256, 0, n->st>>>(in, cin, lg2(D), in_bs, Wm, b, cout, out, out_bs, out_coff);
        else
            k_conv<TI, TA, TO, false><<<grid, 256, 0, n->st>>>(in, cin, lg2(D), in_bs, Wm, b, cout, out, out_bs, out_coff);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int wgrad(const float* dout, int cout, long dout_bs, const TA* in, int cin, long in_bs, int D,
              int B, float* dW, float* db) const {
        const int Kdim = cin * 27;
        const long total = vol(D) * B;
        const int tiles = cdiv_i(Kdim, CV_N) * cdiv_i(cout, CV_M);
        // about four CTAs per SM in total, each slice at least 256 voxels
        const int splits = (int)std::max(1L, std::min((long)cdiv_i(4 * 148, tiles), total / 256));
        {
            KTRACE("cnn_wgrad", n->st, (double)B * vol(D) * (cin * sizeof(TA) + cout * 4.0) + cout * Kdim * 8.0,
                   2.0 * total * Kdim * cout);
            bool done = false;
            if (use_tc() && tc_conv_supported(cout, D, true)) {
                NTRY(tc_conv_wgrad<TA>(dout, cout, dout_bs, in, cin, in_bs, D, B, dW, n->st));
                done = true;
            }
            if (!done)
                k_conv_wgrad<TA><<<dim3(cdiv_i(Kdim, CV_N), cdiv_i(cout, CV_M), splits), 256, 0, n->st>>>(
                    dout, cout, dout_bs, in, cin, in_bs, lg2(D), B, dW);
        }
        LDDMM_CHECK_LAUNCH();
        {
            KTRACE("cnn_bias_grad", n->st, (double)B * cout * vol(D) * 4.0, (double)B * cout * vol(D));
            const int slices = (int)std::max(1L, std::min((long)cdiv_i(2 * 148, cout), total / 4096));
            k_bias_grad<<<dim3(cout, slices), 256, 0, n->st>>>(dout, vol(D), B, dout_bs, db);
        }
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int relu_mask(float* g, long g_bs, const TA* act, long a_bs, long per_b, int B) const {
        KTRACE("cnn_relu_grad", n->st, (double)B * per_b * (8.0 + sizeof(TA)), 0);
        k_relu_mask<TA><<<dim3(elem_grid(per_b), B), 256, 0, n->st>>>(g, g_bs, act, a_bs, per_b);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int pool(const TA* in, long in_bs, int in_coff, int C, int d, TA* out, long out_bs, int B) const {
        KTRACE("cnn_pool", n->st, (double)B * C * vol(d) * 9.0 * sizeof(TA), 0);
        k_pool2<TA><<<dim3(elem_grid(C * vol(d)), B), 256, 0, n->st>>>(in, in_bs, in_coff, C, d, out, out_bs);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int pool_grad(const float* src, long src_bs, int C, int d, float* dst, long dst_bs, int dst_coff,
                  int B) const {
        KTRACE("cnn_pool_grad", n->st, (double)B * C * vol(d) * 68.0, 0);
        k_pool2_grad<<<dim3(elem_grid(C * vol(2 * d)), B), 256, 0, n->st>>>(src, src_bs, C, d, dst, dst_bs, dst_coff);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int up(const TA* in, long in_bs, int C, int d, TA* out, long out_bs, int out_coff, int B) const {
        KTRACE("cnn_up", n->st, (double)B * C * vol(d) * 9.0 * sizeof(TA), 0);
        k_up2<TA><<<dim3(elem_grid(C * vol(2 * d)), B), 256, 0, n->st>>>(in, in_bs, C, d, out, out_bs, out_coff);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int up_grad(const float* src, long src_bs, int src_coff, int C, int d, float* dst, long dst_bs,
                int B) const {
        KTRACE("cnn_up_grad", n->st, (double)B * C * vol(d) * 36.0, 0);
        k_up2_grad<<<dim3(elem_grid(C * vol(d)), B), 256, 0, n->st>>>(src, src_bs, src_coff, C, d, dst, dst_bs);
        LDDMM_CHECK_LAUNCH();
        return LDDMM_OK;
    }

    int refresh_weights() const {
        for (const Layer& l : n->L) {
            const long cnt = (long)l.cout * l.cin * 27;
            KTRACE("cnn_weights", n->st, cnt * (4.0 + 2 * sizeof(TA)), 0);
            k_weights<TA><<<cdiv_i(cnt, 256), 256, 0, n->st>>>(n->P + l.woff, l.cout, l.cin,
                                                              a(n->Wb) + l.woff, a(n->Wt) + l.woff);
            LDDMM_CHECK_LAUNCH();
        }
        return LDDMM_OK;
    }

    int forward(const float* xin, int B) const;
    int backward(const float* dy, int B) const;
};

// the convolutions in forward order
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, OUT, NL };

// forward pass of B samples xin (FP32 [B][2][D^3]) into n->y ([B][3][(D/2)^3])
template <typename TA>
int Net<TA>::forward(const float* xin, int B) const {
    const int c = n->c, D = n->D, d1 = D / 2, d2 = D / 4, d3 = D / 8;
    const long v0 = vol(D), v1 = vol(d1), v2 = vol(d2), v3 = vol(d3);
    TA *x = a(n->x), *a0a = a(n->a0a), *a0b = a(n->a0b), *p0 = a(n->p0), *a1a = a(n->a1a),
       *cat1 = a(n->cat1), *p1 = a(n->p1), *a2a = a(n->a2a), *cat2 = a(n->cat2), *p2 = a(n->p2),
       *a3a = a(n->a3a), *a3b = a(n->a3b), *a4a = a(n->a4a), *a4b = a(n->a4b), *a5a = a(n->a5a),
       *a5b = a(n->a5b);
    {
        KTRACE("cnn_input", n->st, (double)B * 2 * v0 * (4.0 + sizeof(TA)), 0);
        k_to_storage<TA><<<elem_grid((long)B * 2 * v0), 256, 0, n->st>>>(xin, x, (long)B * 2 * v0);
    }
    LDDMM_CHECK_LAUNCH();
    NTRY(conv(x, 2, D, 2 * v0, W(E0A), bias(E0A), c, a0a, c * v0, 0, true, B, "cnn_conv"));
    NTRY(conv(a0a, c, D, c * v0, W(E0B), bias(E0B), c, a0b, c * v0, 0, true, B, "cnn_conv"));
    NTRY(pool(a0b, c * v0, 0, c, d1, p0, c * v1, B));
    NTRY(conv(p0, c, d1, c * v1, W(E1A), bias(E1A), 2 * c, a1a, 2 * c * v1, 0, true, B, "cnn_conv"));
    NTRY(conv(a1a, 2 * c, d1, 2 * c * v1, W(E1B), bias(E1B), 2 * c, cat1, 6 * c * v1, 4 * c, true, B, "cnn_conv"));
    NTRY(pool(cat1, 6 * c * v1, 4 * c, 2 * c, d2, p1, 2 * c * v2, B));
    NTRY(conv(p1, 2 * c, d2, 2 * c * v2, W(E2A), bias(E2A), 4 * c, a2a, 4 * c * v2, 0, true, B, "cnn_conv"));
    NTRY(conv(a2a, 4 * c, d2, 4 * c * v2, W(E2B), bias(E2B), 4 * c, cat2, 12 * c * v2, 8 * c, true, B, "cnn_conv"));
    NTRY(pool(cat2, 12 * c * v2, 8 * c, 4 * c, d3, p2, 4 * c * v3, B));
    NTRY(conv(p2, 4 * c, d3, 4 * c * v3, W(E3A), bias(E3A), 8 * c, a3a, 8 * c * v3, 0, true, B, "cnn_conv"));
    NTRY(conv(a3a, 8 * c, d3, 8 * c * v3, W(E3B), bias(E3B), 8 * c, a3b, 8 * c * v3, 0, true, B, "cnn_conv"));
    NTRY(up(a3b, 8 * c * v3, 8 * c, d3, cat2, 12 * c * v2, 0, B));
    NTRY(conv(cat2, 12 * c, d2, 12 * c * v2, W(D2A), bias(D2A), 4 * c, a4a, 4 * c * v2, 0, true, B, "cnn_conv"));
    NTRY(conv(a4a, 4 * c, d2, 4 * c * v2, W(D2B), bias(D2B), 4 * c, a4b, 4 * c * v2, 0, true, B, "cnn_conv"));
    NTRY(up(a4b, 4 * c * v2, 4 * c, d2, cat1, 6 * c * v1, 0, B));
    NTRY(conv(cat1, 6 * c, d1, 6 * c * v1, W(D1A), bias(D1A), 2 * c, a5a, 2 * c * v1, 0, true, B, "cnn_conv"));
    NTRY(conv(a5a, 2 * c, d1, 2 * c * v1, W(D1B), bias(D1B), 2 * c, a5b, 2 * c * v1, 0, true, B, "cnn_conv"));
    NTRY(conv(a5b, 2 * c, d1, 2 * c * v1, W(OUT), bias(OUT), 3, n->y, 3 * v1, 0, false, B, "cnn_conv"));
    return LDDMM_OK;
}

// gradients of sum(dy * y) (dy FP32 [B][3][(D/2)^3]) accumulated into n->G; needs the
// activations of the forward pass just run on the same input
template <typename TA>
int Net<TA>::backward(const float* dy, int B) const {
    const int c = n->c, D = n->D, d1 = D / 2, d2 = D / 4, d3 = D / 8;
    const long v0 = vol(D), v1 = vol(d1), v2 = vol(d2), v3 = vol(d3);
    TA *x = a(n->x), *a0a = a(n->a0a), *a0b = a(n->a0b), *p0 = a(n->p0), *a1a = a(n->a1a),
       *cat1 = a(n->cat1), *p1 = a(n->p1), *a2a = a(n->a2a), *cat2 = a(n->cat2), *p2 = a(n->p2),
       *a3a = a(n->a3a), *a3b = a(n->a3b), *a4a = a(n->a4a), *a4b = a(n->a4b), *a5a = a(n->a5a),
       *a5b = a(n->a5b);
    float *gA = n->gA, *gB = n->gB, *gcat1 = n->gcat1, *gcat2 = n->gcat2;
    // out: input a5b
    NTRY(wgrad(dy, 3, 3 * v1, a5b, 2 * c, 2 * c * v1, d1, B, gw(OUT), gb(OUT)));
    NTRY(conv(dy, 3, d1, 3 * v1, Wt(OUT), nullptr, 2 * c, gA, 2 * c * v1, 0, false, B, "cnn_dgrad"));
    // d1b: output a5b, input a5a
    NTRY(relu_mask(gA, 2 * c * v1, a5b, 2 * c * v1, 2 * c * v1, B));
    NTRY(wgrad(gA, 2 * c, 2 * c * v1, a5a, 2 * c, 2 * c * v1, d1, B, gw(D1B), gb(D1B)));
    NTRY(conv(gA, 2 * c, d1, 2 * c * v1, Wt(D1B), nullptr, 2 * c, gB, 2 * c * v1, 0, false, B, "cnn_dgrad"));
    // d1a: output a5a, input cat1 = [up(a4b) | e1]
    NTRY(relu_mask(gB, 2 * c * v1, a5a, 2 * c * v1, 2 * c * v1, B));
    NTRY(wgrad(gB, 2 * c, 2 * c * v1, cat1, 6 * c, 6 * c * v1, d1, B, gw(D1A), gb(D1A)));
    NTRY(conv(gB, 2 * c, d1, 2 * c * v1, Wt(D1A), nullptr, 6 * c, gcat1, 6 * c * v1, 0, false, B, "cnn_dgrad"));
    NTRY(up_grad(gcat1, 6 * c * v1, 0, 4 * c, d2, gA, 4 * c * v2, B));
    // d2b: output a4b, input a4a
    NTRY(relu_mask(gA, 4 * c * v2, a4b, 4 * c * v2, 4 * c * v2, B));
    NTRY(wgrad(gA, 4 * c, 4 * c * v2, a4a, 4 * c, 4 * c * v2, d2, B, gw(D2B), gb(D2B)));
    NTRY(conv(gA, 4 * c, d2, 4 * c * v2, Wt(D2B), nullptr, 4 * c, gB, 4 * c * v2, 0, false, B, "cnn_dgrad"));
    // d2a: output a4a, input cat2 = [up(a3b) | e2]
    NTRY(relu_mask(gB, 4 * c * v2, a4a, 4 * c * v2, 4 * c * v2, B));
    NTRY(wgrad(gB, 4 * c, 4 * c * v2, cat2, 12 * c, 12 * c * v2, d2, B, gw(D2A), gb(D2A)));
    NTRY(conv(gB, 4 * c, d2, 4 * c * v2, Wt(D2A), nullptr, 12 * c, gcat2, 12 * c * v2, 0, false, B, "cnn_dgrad"));
    NTRY(up_grad(gcat2, 12 * c * v2, 0, 8 * c, d3, gA, 8 * c * v3, B));
    // e3b: output a3b, input a3a
    NTRY(relu_mask(gA, 8 * c * v3, a3b, 8 * c * v3, 8 * c * v3, B));
    NTRY(wgrad(gA, 8 * c, 8 * c * v3, a3a, 8 * c, 8 * c * v3, d3, B, gw(E3B), gb(E3B)));
    NTRY(conv(gA, 8 * c, d3, 8 * c * v3, Wt(E3B), nullptr, 8 * c, gB, 8 * c * v3, 0, false, B, "cnn_dgrad"));
    // e3a: output a3a, input p2 = pool(e2)
    NTRY(relu_mask(gB, 8 * c * v3, a3a, 8 * c * v3, 8 * c * v3, B));
    NTRY(wgrad(gB, 8 * c, 8 * c * v3, p2, 4 * c, 4 * c * v3, d3, B, gw(E3A), gb(E3A)));
    NTRY(conv(gB, 8 * c, d3, 8 * c * v3, Wt(E3A), nullptr, 4 * c, gA, 4 * c * v3, 0, false, B, "cnn_dgrad"));
    NTRY(pool_grad(gA, 4 * c * v3, 4 * c, d3, gcat2, 12 * c * v2, 8 * c, B));
    // e2b: output e2 = cat2[8c:12c], input a2a
    {
        float* g2 = gcat2 + 8L * c * v2;
        NTRY(relu_mask(g2, 12 * c * v2, cat2 + 8L * c * v2, 12 * c * v2, 4 * c * v2, B));
        NTRY(wgrad(g2, 4 * c, 12 * c * v2, a2a, 4 * c, 4 * c * v2, d2, B, gw(E2B), gb(E2B)));
        NTRY(conv(g2, 4 * c, d2, 12 * c * v2, Wt(E2B), nullptr, 4 * c, gB, 4 * c * v2, 0, false, B, "cnn_dgrad"));
    }
    // e2a: output a2a, input p1 = pool(e1)
    NTRY(relu_mask(gB, 4 * c * v2, a2a, 4 * c * v2, 4 * c * v2, B));
    NTRY(wgrad(gB, 4 * c, 4 * c * v2, p1, 2 * c, 2 * c * v2, d2, B, gw(E2A), gb(E2A)));
    NTRY(conv(gB, 4 * c, d2, 4 * c * v2, Wt(E2A), nullptr, 2 * c, gA, 2 * c * v2, 0, false, B, "cnn_dgrad"));
    NTRY(pool_grad(gA, 2 * c * v2, 2 * c, d2, gcat1, 6 * c * v1, 4 * c, B));
    // e1b: output e1 = cat1[4c:6c], input a1a
    {
        float* g1 = gcat1 + 4L * c * v1;
        NTRY(relu_mask(g1, 6 * c * v1, cat1 + 4L * c * v1, 6 * c * v1, 2 * c * v1, B));
        NTRY(wgrad(g1, 2 * c, 6 * c * v1, a1a, 2 * c, 2 * c * v1, d1, B, gw(E1B), gb(E1B)));
        NTRY(conv(g1, 2 * c, d1, 6 * c * v1, Wt(E1B), nullptr, 2 * c, gB, 2 * c * v1, 0, false, B, "cnn_dgrad"));
    }
    // e1a: output a1a, input p0 = pool(a0b)
    NTRY(relu_mask(gB, 2 * c * v1, a1a, 2 * c * v1, 2 * c * v1, B));
    NTRY(wgrad(gB, 2 * c, 2 * c * v1, p0, c, c * v1, d1, B, gw(E1A), gb(E1A)));
    NTRY(conv(gB, 2 * c, d1, 2 * c * v1, Wt(E1A), nullptr, c, gA, c * v1, 0, false, B, "cnn_dgrad"));
    LDDMM_CUDA(cudaMemsetAsync(gB, 0, (size_t)B * c * v0 * sizeof(float), n->st));
    NTRY(pool_grad(gA, c * v1, c, d1, gB, c * v0, 0, B));
    // e0b: output a0b, input a0a
    NTRY(relu_mask(gB, c * v0, a0b, c * v0, c * v0, B));
    NTRY(wgrad(gB, c, c * v0, a0a, c, c * v0, D, B, gw(E0B), gb(E0B)));
    NTRY(conv(gB, c, D, c * v0, Wt(E0B), nullptr, c, gA, c * v0, 0, false, B, "cnn_dgrad"));
    // e0a: output a0a, input x
    NTRY(relu_mask(gA, c * v0, a0a, c * v0, c * v0, B));
    NTRY(wgrad(gA, c, c * v0, x, 2, 2 * v0, D, B, gw(E0A), gb(E0A)));
    return LDDMM_OK;
}

bool fp32_storage(const lddmm_net* n) {
    return n->storage == LDDMM_NET_FP32 || n->storage == LDDMM_NET_FP32_TC;
}

int refresh_weights(lddmm_net* n) {
    return fp32_storage(n) ? Net<float>{n}.refresh_weights()
                                        : Net<__nv_bfloat16>{n}.refresh_weights();
}
int forward_impl(lddmm_net* n, const float* xin, int B) {
    return fp32_storage(n) ? Net<float>{n}.forward(xin, B)
                                        : Net<__nv_bfloat16>{n}.forward(xin, B);
}
int backward_impl(lddmm_net* n, const float* dy, int B) {
    return fp32_storage(n) ? Net<float>{n}.backward(dy, B)
                                        : Net<__nv_bfloat16>{n}.backward(dy, B);
}

int net_alloc(lddmm_net* n, unsigned long long seed) {
    const int c = n->c, D = n->D;
    const int d1 = D / 2, d2 = D / 4, d3 = D / 8;
    struct S { int cin, cout, D; bool relu; };
    const S specs[NL] = {{2, c, D, true},          {c, c, D, true},          {c, 2 * c, d1, true},
                         {2 * c, 2 * c, d1, true}, {2 * c, 4 * c, d2, true}, {4 * c, 4 * c, d2, true},
                         {4 * c, 8 * c, d3, true}, {8 * c, 8 * c, d3, true}, {12 * c, 4 * c, d2, true},
                         {4 * c, 4 * c, d2, true}, {6 * c, 2 * c, d1, true}, {2 * c, 2 * c, d1, true},
                         {2 * c, 3, d1, false}};
    long off = 0;
    for (int i = 0; i < NL; ++i) {
        Layer l{specs[i].cin, specs[i].cout, specs[i].D, specs[i].relu, off, 0};
        off += (long)l.cout * l.cin * 27;
        l.boff = off;
        off += l.cout;
        n->L.push_back(l);
    }
    n->nparam = off;
    const size_t e = n->esz;
    NTRY(nalloc_t(n, &n->P, off));
    NTRY(nalloc_t(n, &n->G, off));
    NTRY(nalloc_t(n, &n->M, off));
    NTRY(nalloc_t(n, &n->V, off));
    NTRY(nalloc(n, &n->Wb, off * e));
    NTRY(nalloc(n, &n->Wt, off * e));
    // He initialisation (std sqrt(2 / fan_in)) from a seeded host generator; biases zero
    std::vector<float> h(off, 0.f);
    std::mt19937_64 gen(seed);
    for (const Layer& l : n->L) {
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (l.cin * 27.f)));
        for (long i = 0; i < (long)l.cout * l.cin * 27; ++i) h[l.woff + i] = nd(gen);
    }
    LDDMM_CUDA(cudaMemcpy(n->P, h.data(), off * sizeof(float), cudaMemcpyHostToDevice));
    LDDMM_CUDA(cudaMemset(n->M, 0, off * sizeof(float)));
    LDDMM_CUDA(cudaMemset(n->V, 0, off * sizeof(float)));
    const size_t B = n->bmax;
    NTRY(nalloc(n, &n->x, B * 2 * vol(D) * e));
    NTRY(nalloc(n, &n->a0a, B * c * vol(D) * e));
    NTRY(nalloc(n, &n->a0b, B * c * vol(D) * e));
    NTRY(nalloc(n, &n->p0, B * c * vol(d1) * e));
    NTRY(nalloc(n, &n->a1a, B * 2 * c * vol(d1) * e));
    NTRY(nalloc(n, &n->cat1, B * 6 * c * vol(d1) * e));
    NTRY(nalloc(n, &n->p1, B * 2 * c * vol(d2) * e));
    NTRY(nalloc(n, &n->a2a, B * 4 * c * vol(d2) * e));
    NTRY(nalloc(n, &n->cat2, B * 12 * c * vol(d2) * e));
    NTRY(nalloc(n, &n->p2, B * 4 * c * vol(d3) * e));
    NTRY(nalloc(n, &n->a3a, B * 8 * c * vol(d3) * e));
    NTRY(nalloc(n, &n->a3b, B * 8 * c * vol(d3) * e));
    NTRY(nalloc(n, &n->a4a, B * 4 * c * vol(d2) * e));
    NTRY(nalloc(n, &n->a4b, B * 4 * c * vol(d2) * e));
    NTRY(nalloc(n, &n->a5a, B * 2 * c * vol(d1) * e));
    NTRY(nalloc(n, &n->a5b, B * 2 * c * vol(d1) * e));
    NTRY(nalloc_t(n, &n->y, B * 3 * vol(d1)));
    const size_t gmax = std::max({(long)c * vol(D), 12L * c * vol(d2), 3L * vol(d1)});
    NTRY(nalloc_t(n, &n->gA, B * gmax));
    NTRY(nalloc_t(n, &n->gB, B * gmax));
    NTRY(nalloc_t(n, &n->gC, B * gmax));
    NTRY(nalloc_t(n, &n->gcat1, B * 6 * c * vol(d1)));
    NTRY(nalloc_t(n, &n->gcat2, B * 12 * c * vol(d2)));
    NTRY(nalloc_t(n, &n->partials, 512));
    NTRY(nalloc_t(n, &n->xin, 2 * vol(D)));
    NTRY(nalloc_t(n, &n->cube, 2 * vol(D)));
    LDDMM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&n->hpart), 512 * sizeof(double)));
    return LDDMM_OK;
}

int check_batch(lddmm_net* n, int B, const void* a, const void* b, const void* c, const char* fn) {
    if (!n) {
        set_error(std::string(fn) + ": network is NULL");
        return LDDMM_EINVAL;
    }
    if (B < 1 || B > n->bmax || !a || !b || !c) {
        set_error(std::string(fn) + ": batch must be in 1..batch_max and pointers non-NULL");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

}  // namespace

extern "C" {

int lddmm_net_create(int D, int base_channels, int batch_max, int storage, unsigned long long seed,
                     void* stream, lddmm_net** out) {
    if (!out) {
        set_error("net_create: out is NULL");
        return LDDMM_EINVAL;
    }
    *out = nullptr;
    if (D < 8 || D > 128 || (D & (D - 1)) || base_channels < 1 || base_channels > 64 ||
        batch_max < 1 || batch_max > 64 ||
        storage < LDDMM_NET_BF16 || storage > LDDMM_NET_FP32_TC) {
        set_error("net_create: D must be a power of two in 8..128, base_channels 1..64, batch_max "
                  "1..64, storage LDDMM_NET_BF16, LDDMM_NET_FP32, LDDMM_NET_BF16_SIMT or LDDMM_NET_FP32_TC");
        return LDDMM_EINVAL;
    }
    lddmm_net* n = new lddmm_net();
    n->D = D;
    n->c = base_channels;
    n->bmax = batch_max;
    n->storage = storage;
    n->esz = fp32_storage(n) ? sizeof(float) : sizeof(__nv_bfloat16);
    n->st = static_cast<cudaStream_t>(stream);
    int rc = net_alloc(n, seed);
    if (rc == LDDMM_OK) rc = refresh_weights(n);
    if (rc == LDDMM_OK && cudaStreamSynchronize(n->st) != cudaSuccess) {
        set_error("net_create: initialisation failed");
        rc = LDDMM_ECUDA;
    }
    if (rc != LDDMM_OK) {
        const std::string msg = lddmm_last_error();
        lddmm_net_destroy(n);
        set_error(msg);
        return rc;
    }
    *out = n;
    return LDDMM_OK;
}

int lddmm_net_destroy(lddmm_net* n) {
    if (!n) return LDDMM_OK;
    cudaStreamSynchronize(n->st);
    for (void* p : n->allocs) cudaFree(p);
    if (n->hpart) cudaFreeHost(n->hpart);
    delete n;
    return LDDMM_OK;
}

long lddmm_net_num_params(const lddmm_net* n) { return n ? n->nparam : 0; }

int lddmm_net_get_params(lddmm_net* n, float* dst) {
    if (!n || !dst) {
        set_error("net_get_params: NULL argument");
        return LDDMM_EINVAL;
    }
    LDDMM_CUDA(cudaMemcpyAsync(dst, n->P, n->nparam * sizeof(float), cudaMemcpyDefault, n->st));
    LDDMM_CUDA(cudaStreamSynchronize(n->st));
    return LDDMM_OK;
}

int lddmm_net_set_params(lddmm_net* n, const float* src) {
    if (!n || !src) {
        set_error("net_set_params: NULL argument");
        return LDDMM_EINVAL;
    }
    LDDMM_CUDA(cudaMemcpyAsync(n->P, src, n->nparam * sizeof(float), cudaMemcpyDefault, n->st));
    LDDMM_CUDA(cudaMemsetAsync(n->M, 0, n->nparam * sizeof(float), n->st));
    LDDMM_CUDA(cudaMemsetAsync(n->V, 0, n->nparam * sizeof(float), n->st));
    n->adam_t = 0;
    NTRY(refresh_weights(n));
    LDDMM_CUDA(cudaStreamSynchronize(n->st));
    return LDDMM_OK;
}

int lddmm_net_forward(lddmm_net* n, const float* x, int B, float* y) {
    NTRY(check_batch(n, B, x, y, y, "net_forward"));
    NTRY(forward_impl(n, x, B));
    LDDMM_CUDA(cudaMemcpyAsync(y, n->y, (size_t)B * 3 * vol(n->D / 2) * sizeof(float),
                               cudaMemcpyDeviceToDevice, n->st));
    return LDDMM_OK;
}

int lddmm_net_gradients(lddmm_net* n, const float* x, const float* dy, int B, float* grads) {
    NTRY(check_batch(n, B, x, dy, grads, "net_gradients"));
    NTRY(forward_impl(n, x, B));
    LDDMM_CUDA(cudaMemsetAsync(n->G, 0, n->nparam * sizeof(float), n->st));
    NTRY(backward_impl(n, dy, B));
    LDDMM_CUDA(cudaMemcpyAsync(grads, n->G, n->nparam * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    return LDDMM_OK;
}

int lddmm_net_train_step(lddmm_net* n, const float* x, const float* target, int B, float lr,
                         double* loss) {
    NTRY(check_batch(n, B, x, target, target, "net_train_step"));
    if (!(lr > 0.f) || !std::isfinite(lr)) {
        set_error("net_train_step: lr must be positive");
        return LDDMM_EINVAL;
    }
    NTRY(forward_impl(n, x, B));
    const long ny = (long)B * 3 * vol(n->D / 2);
    const int nb = std::min(512, cdiv_i(ny, 256));
    {
        KTRACE("cnn_loss", n->st, ny * 12.0, ny * 3.0);
        k_mse<<<nb, 256, 0, n->st>>>(n->y, target, ny, n->gC, n->partials);
    }
    LDDMM_CHECK_LAUNCH();
    LDDMM_CUDA(cudaMemsetAsync(n->G, 0, n->nparam * sizeof(float), n->st));
    NTRY(backward_impl(n, n->gC, B));
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    {
        KTRACE("cnn_adam", n->st, n->nparam * 20.0, n->nparam * 10.0);
        k_adam<<<elem_grid(n->nparam), 256, 0, n->st>>>(n->P, n->G, n->M, n->V, n->nparam, lr, b1, b2,
                                                      1e-8f, c1, c2);
    }
    LDDMM_CHECK_LAUNCH();
    NTRY(refresh_weights(n));
    if (loss) {
        LDDMM_CUDA(cudaMemcpyAsync(n->hpart, n->partials, nb * sizeof(double), cudaMemcpyDeviceToHost, n->st));
        LDDMM_CUDA(cudaStreamSynchronize(n->st));
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += n->hpart[i];
        *loss = s / (double)ny;
    }
    return LDDMM_OK;
}

int lddmm_net_input(lddmm_net* n, int nx, int ny, int nz, const float* I0, const float* I1, float* x) {
    if (!n || !I0 || !I1 || !x) {
        set_error("net_input: NULL argument");
        return LDDMM_EINVAL;
    }
    const int D = n->D;
    if (nx < D || ny < D || nz < D) {
        set_error("net_input: every image extent must be at least the network's input size D");
        return LDDMM_EINVAL;
    }
    const float* img[2] = {I0, I1};
    for (int ch = 0; ch < 2; ++ch) {
        NTRY(lddmm_bl_project(nx, ny, nz, D, img[ch], 1, n->cube, LDDMM_PREC_FP32, n->st));
        NTRY(lddmm_bl_include(D, D, D, D, n->cube, 1, x + ch * vol(D), -1, 0, LDDMM_PREC_FP32, n->st));
    }
    return LDDMM_OK;
}

int lddmm_net_warm_start(lddmm_net* n, int nx, int ny, int nz, const float* I0, const float* I1,
                         int K, float* vtilde) {
    if (!n || !vtilde) {
        set_error("net_warm_start: NULL argument");
        return LDDMM_EINVAL;
    }
    if (K > n->D / 2) {
        set_error("net_warm_start: K must not exceed the output grid size D/2");
        return LDDMM_EINVAL;
    }
    NTRY(lddmm_net_input(n, nx, ny, nz, I0, I1, n->xin));
    NTRY(forward_impl(n, n->xin, 1));
    const int d1 = n->D / 2;
    return lddmm_bl_project(d1, d1, d1, K, n->y, 3, vtilde, LDDMM_PREC_FP32, n->st);
}

}  // extern "C"
