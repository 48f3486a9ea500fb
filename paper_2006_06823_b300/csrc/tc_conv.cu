// 3x3x3 convolutions of the warm-start network on the 5th-generation tensor cores (tcgen05),
// for the BF16-storage network: the forward pass, the input gradient and the weight gradient
// are implicit GEMMs whose operands are built in shared memory, multiplied by tcgen05.mma of
// kind::tf32 with FP32 accumulation in tensor memory.
//
//   forward / input gradient:  out[co][v] = sum_k W[co][k] im2col(in)[k][v]
//       M = 128 voxels of one sample, N = cout (rounded up to 16), K = cin * 27;
//   weight gradient:           dW[co][k] += sum_v dout[co][v] im2col(in)[k][v]
//       M = 128 rows k = ci * 27 + t, N = cout (rounded up to 16), K = voxels (a slice of
//       all samples per CTA, partial sums added to dW with FP32 atomics).
// with im2col(in)[ci * 27 + t][v] = in[ci][v + o(t)] (zero outside the D^3 volume), tap
// t = (dz + 1) 9 + (dy + 1) 3 + (dx + 1).
//
// Operands are FP32 words in the 128-byte-swizzled K-major layout (32 per row). BF16 values
// (the stored weights and activations of the BF16 network) are exact in TF32, so they enter
// the MMA unchanged; FP32 operands (the gradients, and every operand of the FP32 tensor-core
// check form) are split hi + lo, hi = x rounded to TF32, lo = (x - hi) rounded to TF32
// (|x - hi - lo| <= 2^-22 |x|), and the products A_hi B_hi + A_lo B_hi + A_hi B_lo are
// accumulated, so every product is the FP32 product up to about 2^-21 relative (the dropped
// A_lo B_lo and the rounding of lo), against 2^-24 for the FP32 SIMT kernels; sums are FP32.
//
// One CTA of 128 threads per output tile: for each 32-wide K chunk all threads build the
// next chunk's operands into the free one of two smem stages while the MMAs of the previous
// chunk run; thread 0 issues the MMAs and commits them to that stage's mbarrier. Every wait is
// bounded by %globaltimer; on expiry the kernel records LDDMM_ETIMEOUT in its device error word
// (read by lddmm_device_error), stops issuing work, waits (bounded) for its own MMAs, frees its
// tensor memory and returns.
#include "common.cuh"
#include "lddmm.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace lddmm {

__device__ int g_conv_error = 0;

namespace {

constexpr int TM = 128;          // MMA M: rows of the output tile
constexpr int KC = 32;           // K per chunk: 32 FP32 words = one 128-byte swizzle row
constexpr int ROWB = 128;        // bytes per operand row
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0; it != 0xFFFFFFFFu; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 255u) == 255u && now_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ uint64_t sw128_desc(unsigned saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// kind::tf32, FP32 accumulate, K-major A and B, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// x rounded to TF32 (nearest, ties away), as an FP32 bit pattern with the low 13 bits zero, so
// that the tensor core's reading of the upper 19 bits is exact
__device__ __forceinline__ float tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ float ldv(const float* p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stv(float* p, float v) { *p = v; }
__device__ __forceinline__ void stv(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// writes the 32 words of one operand row (row r of a 1024-aligned SW128 tile)
__device__ __forceinline__ void put_row(unsigned char* tile, int r, const float (&w)[32]) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4*>(tile + r * ROWB + (((j ^ (r & 7))) << 4)) =
            make_float4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
}

// offset of tap t (0..26) and its validity at (z, y, x): bit t of the returned mask
__device__ __forceinline__ unsigned tap_mask(int z, int y, int x, int D) {
    unsigned m = 0;
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        if ((unsigned)(z + dz) < (unsigned)D && (unsigned)(y + dy) < (unsigned)D &&
            (unsigned)(x + dx) < (unsigned)D)
            m |= 1u << t;
    }
    return m;
}
__device__ __forceinline__ int tap_off(int t, int lgD) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    return (dz << (2 * lgD)) + (dy << lgD) + dx;
}

struct Smem {
    uint64_t bar[2];      // MMA completion per stage
    uint64_t done;        // the last chunk's MMAs
    unsigned tmem;
    int abort;
};

// stage layout (1024-aligned): A hi, A lo (SPLIT_A), B hi, B lo (SPLIT_B); A 16 KB, B NP x 128 B
template <bool SPLIT_A, bool SPLIT_B>
__host__ __device__ constexpr size_t stage_bytes(int NP) {
    return (size_t)(SPLIT_A ? 2 : 1) * TM * ROWB + (size_t)(SPLIT_B ? 2 : 1) * ((NP * ROWB + 1023) & ~1023);
}

// The shared chunk loop: build(q, A_hi, A_lo, B_hi, B_lo) fills chunk q's operands; the MMAs
// accumulate into TMEM columns [0, NP). Returns false on a timed-out wait.
template <bool SPLIT_A, bool SPLIT_B, class Build>
__device__ bool chunk_loop(Smem& sm, unsigned char* base, int NP, int nchunks, Build build) {
    const size_t SB = stage_bytes<SPLIT_A, SPLIT_B>(NP);
    const size_t abytes = (size_t)TM * ROWB, bbytes = (size_t)((NP * ROWB + 1023) & ~1023);
    const uint32_t idesc = idesc_tf32(NP);
    bool ok = true;
    for (int q = 0; q < nchunks; ++q) {
        const int s = q & 1;
        unsigned char* st = base + s * SB;
        unsigned char* ahi = st;
        unsigned char* alo = st + abytes;
        unsigned char* bhi = st + (SPLIT_A ? 2 : 1) * abytes;
        unsigned char* blo = bhi + bbytes;
        // the MMAs that read this stage two chunks ago must be done
        if (q >= 2 && !mbar_wait(&sm.bar[s], (unsigned)(((q >> 1) - 1) & 1))) {
            ok = false;
            sm.abort = 1;
        }
        if (__syncthreads_or(!ok || sm.abort)) return false;
        build(q, ahi, alo, bhi, blo);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < KC / 8; ++kk) {
                const unsigned ko = kk * 32;
                const unsigned acc = (q > 0 || kk > 0) ? 1u : 0u;
                mma_tf32(sm.tmem, sw128_desc(smem_u32(ahi) + ko), sw128_desc(smem_u32(bhi) + ko), idesc, acc);
                if (SPLIT_A)
                    mma_tf32(sm.tmem, sw128_desc(smem_u32(alo) + ko), sw128_desc(smem_u32(bhi) + ko), idesc, 1u);
                if (SPLIT_B)
                    mma_tf32(sm.tmem, sw128_desc(smem_u32(ahi) + ko), sw128_desc(smem_u32(blo) + ko), idesc, 1u);
            }
            mma_commit(&sm.bar[s]);
            if (q == nchunks - 1) mma_commit(&sm.done);
        }
    }
    return true;
}

// common prologue: barriers, TMEM allocation (warp 0)
__device__ __forceinline__ void prologue(Smem& sm, unsigned cols) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.bar[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        sm.abort = 0;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// waits for the last MMAs (bounded), then frees the tensor memory
__device__ __forceinline__ bool finish_mma(Smem& sm, int nchunks, bool ok) {
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        bool d = nchunks > 0 ? mbar_wait(&sm.done, 0) : true;
        if (!ok || !d) {
            atomicExch(&g_conv_error, LDDMM_ETIMEOUT);
            // drain: every committed stage must complete before the memory is freed
            for (int s = 0; s < 2; ++s) mbar_wait(&sm.bar[s], 0), mbar_wait(&sm.bar[s], 1);
        }
        ok_sh = ok && d;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return ok_sh != 0;
}
__device__ __forceinline__ void epilogue_free(Smem& sm, unsigned cols) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(sm.tmem), "r"(cols));
}

// ---------------------------------------------------------------- forward / input gradient
// out[b][out_coff + co][v] = relu?(bias[co] + sum_k W[co][k] im2col(in[b])[k][v])
template <typename TI, typename TW, typename TO, bool RELU>
__global__ void __launch_bounds__(128)
k_conv_tc(const TI* __restrict__ in, int cin, int lgD, long in_bstride,
          const TW* __restrict__ W, const float* __restrict__ bias, int cout, int NP,
          TO* __restrict__ out, long out_bstride, int out_coff, unsigned cols) {
    constexpr bool SPLIT_A = sizeof(TI) == 4;   // FP32 operands: hi + lo
    constexpr bool SPLIT_B = sizeof(TW) == 4;
    extern __shared__ unsigned char dyn[];
    __shared__ Smem sm;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    prologue(sm, cols);
    const int b = blockIdx.y;
    const int D = 1 << lgD;
    const long nv = 1L << (3 * lgD);
    const long v = (long)blockIdx.x * TM + threadIdx.x;      // this thread's voxel (A row)
    const bool vok = v < nv;
    const int x = (int)(v & (D - 1)), y = (int)((v >> lgD) & (D - 1)), z = (int)(v >> (2 * lgD));
    const unsigned mask = vok ? tap_mask(z, y, x, D) : 0u;
    const TI* inb = in + (long)b * in_bstride;
    const int Kdim = cin * 27;
    const int nchunks = (Kdim + KC - 1) / KC;
    auto build = [&](int q, unsigned char* ahi, unsigned char* alo, unsigned char* bhi, unsigned char* blo) {
        const int k0 = q * KC;
        // A row: im2col values of this voxel for k0 .. k0 + 31
        {
            float hi[32], lo[32];
            int ci = k0 / 27, t = k0 - 27 * ci;
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                float val = 0.f;
                if (k0 + kk < Kdim && ((mask >> t) & 1u))
                    val = ldv(inb + (long)ci * nv + v + tap_off(t, lgD));
                if (SPLIT_A) {
                    hi[kk] = tf32_rna(val);
                    lo[kk] = tf32_rna(val - hi[kk]);
                } else {
                    hi[kk] = val;
                }
                if (++t == 27) {
                    t = 0;
                    ++ci;
                }
            }
            put_row(ahi, threadIdx.x, hi);
            if (SPLIT_A) put_row(alo, threadIdx.x, lo);
        }
        // B rows: W[co][k0 .. k0 + 31] (BF16: exact in TF32; FP32: hi + lo), zero past cout
        // and Kdim
        for (int co = threadIdx.x; co < NP; co += TM) {
            float w[32], wl[32];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                const float val = (co < cout && k0 + kk < Kdim) ? ldv(W + (long)co * Kdim + k0 + kk) : 0.f;
                if (SPLIT_B) {
                    w[kk] = tf32_rna(val);
                    wl[kk] = tf32_rna(val - w[kk]);
                } else {
                    w[kk] = val;
                }
            }
            put_row(bhi, co, w);
            if (SPLIT_B) put_row(blo, co, wl);
        }
    };
    bool ok = chunk_loop<SPLIT_A, SPLIT_B>(sm, base, NP, nchunks, build);
    ok = finish_mma(sm, nchunks, ok);
    if (ok) {
        // TMEM lane = tile row = voxel; warp w reads lanes 32 w .. 32 w + 31
        const int warp = threadIdx.x >> 5;
        TO* outb = out + (long)b * out_bstride;
        for (int c0 = 0; c0 < NP; c0 += 32) {
            float acc[32];
            tmem_ld32(sm.tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, acc);
            if (vok) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int co = c0 + i;
                    if (co < cout) {
                        float r = acc[i] + (bias ? bias[co] : 0.f);
                        if (RELU) r = fmaxf(r, 0.f);
                        stv(outb + (long)(out_coff + co) * nv + v, r);
                    }
                }
            }
        }
    }
    epilogue_free(sm, cols);
}

// ---------------------------------------------------------------- weight gradient
// dW[co][k] += sum over this CTA's voxel slice of dout[b][co][v] im2col(in[b])[k][v]; rows of
// the tile are k = blockIdx.x * 128 + r, K chunks are 32 consecutive voxels of the flattened
// [B][D^3] index (D >= 32, so a chunk is one x-row segment of one sample).
template <typename TA>
__global__ void __launch_bounds__(128)
k_conv_wgrad_tc(const float* __restrict__ dout, int cout, long dout_bstride,
                const TA* __restrict__ in, int cin, long in_bstride, int lgD, int B,
                int NP, float* __restrict__ dW, unsigned cols) {
    constexpr bool SPLIT_A = sizeof(TA) == 4;
    extern __shared__ unsigned char dyn[];
    __shared__ Smem sm;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    prologue(sm, cols);
    const int D = 1 << lgD;
    const long nv = 1L << (3 * lgD);
    const int Kdim = cin * 27;
    const int k = blockIdx.x * TM + threadIdx.x;       // this thread's A row
    const bool kok = k < Kdim;
    const int ci = kok ? k / 27 : 0, t = kok ? k - 27 * (k / 27) : 13;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const long total_chunks = (long)B * nv / KC;
    const long per = (total_chunks + gridDim.y - 1) / gridDim.y;
    const long c_begin = blockIdx.y * per;
    const long c_end = c_begin + per < total_chunks ? c_begin + per : total_chunks;
    const int nchunks = c_end > c_begin ? (int)(c_end - c_begin) : 0;
    auto build = [&](int q, unsigned char* ahi, unsigned char* alo, unsigned char* bhi, unsigned char* blo) {
        const long g0 = (c_begin + q) * KC;                 // first flattened voxel of the chunk
        const int b = (int)(g0 >> (3 * lgD));
        const long v0 = g0 - ((long)b << (3 * lgD));
        const int x0 = (int)(v0 & (D - 1)), y = (int)((v0 >> lgD) & (D - 1)), z = (int)(v0 >> (2 * lgD));
        // A row k: in[b][ci][v + o(t)] for the chunk's 32 voxels (x0 .. x0 + 31 of row (z, y))
        {
            float a[32], al[32];
            const bool rowok = kok && (unsigned)(z + dz) < (unsigned)D && (unsigned)(y + dy) < (unsigned)D;
            const TA* src = in + (long)b * in_bstride + (long)ci * nv +
                            (((long)(z + dz) << (2 * lgD)) + ((long)(y + dy) << lgD));
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                const int xx = x0 + i + dx;
                const float val = (rowok && (unsigned)xx < (unsigned)D) ? ldv(src + xx) : 0.f;
                if (SPLIT_A) {
                    a[i] = tf32_rna(val);
                    al[i] = tf32_rna(val - a[i]);
                } else {
                    a[i] = val;
                }
            }
            put_row(ahi, threadIdx.x, a);
            if (SPLIT_A) put_row(alo, threadIdx.x, al);
        }
        // B rows co: dout[b][co][v0 .. v0 + 31], split hi + lo
        for (int co = threadIdx.x; co < NP; co += TM) {
            float hi[32], lo[32];
            const float* src = dout + (long)b * dout_bstride + (long)co * nv + v0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float4 f4 = co < cout ? *reinterpret_cast<const float4*>(src + 4 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float f[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    hi[4 * j + e] = tf32_rna(f[e]);
                    lo[4 * j + e] = tf32_rna(f[e] - hi[4 * j + e]);
                }
            }
            put_row(bhi, co, hi);
            put_row(blo, co, lo);
        }
    };
    bool ok = chunk_loop<SPLIT_A, true>(sm, base, NP, nchunks, build);
    ok = finish_mma(sm, nchunks, ok);
    if (ok && nchunks > 0) {   // CTA-uniform: every lane takes part in the collective loads
        const int warp = threadIdx.x >> 5;
        for (int c0 = 0; c0 < NP; c0 += 32) {
            float acc[32];
            tmem_ld32(sm.tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, acc);
            if (kok) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (c0 + i < cout) atomicAdd(dW + (long)(c0 + i) * Kdim + k, acc[i]);
            }
        }
    }
    epilogue_free(sm, cols);
}

unsigned tmem_cols_for(int NP) {
    unsigned c = 32;
    while ((int)c < NP) c <<= 1;
    return c;
}

}  // namespace

bool tc_conv_supported(int cout, int D, bool wgrad) {
    const int NP = (cout + 15) & ~15;
    return NP >= 16 && NP <= 256 && D >= 2 && (D & (D - 1)) == 0 && (!wgrad || D >= KC);
}

template <typename TI, typename TW, typename TO>
int tc_conv(const TI* in, int cin, int D, long in_bstride, const TW* W, const float* bias,
            int cout, TO* out, long out_bstride, int out_coff, bool relu, int B, cudaStream_t st) {
    const int NP = (cout + 15) & ~15;
    constexpr bool SPLIT_A = sizeof(TI) == 4, SPLIT_B = sizeof(TW) == 4;
    const int smem = (int)(2 * stage_bytes<SPLIT_A, SPLIT_B>(NP) + 1024);
    const unsigned cols = tmem_cols_for(NP);
    int lgD = 0;
    while ((1 << lgD) < D) ++lgD;
    const long nv = 1L << (3 * lgD);
    dim3 grid((unsigned)((nv + TM - 1) / TM), (unsigned)B);
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaError_t e;
    if (relu) {
        e = cudaFuncSetAttribute(k_conv_tc<TI, TW, TO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            k_conv_tc<TI, TW, TO, true><<<grid, TM, smem, st>>>(in, cin, lgD, in_bstride, W, bias, cout, NP,
                                                                out, out_bstride, out_coff, cols);
    } else {
        e = cudaFuncSetAttribute(k_conv_tc<TI, TW, TO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            k_conv_tc<TI, TW, TO, false><<<grid, TM, smem, st>>>(in, cin, lgD, in_bstride, W, bias, cout, NP,
                                                                 out, out_bstride, out_coff, cols);
    }
    LDDMM_CUDA(e);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

using bf16 = __nv_bfloat16;
template int tc_conv<bf16, bf16, bf16>(const bf16*, int, int, long, const bf16*, const float*, int,
                                       bf16*, long, int, bool, int, cudaStream_t);
template int tc_conv<bf16, bf16, float>(const bf16*, int, int, long, const bf16*, const float*, int,
                                        float*, long, int, bool, int, cudaStream_t);
template int tc_conv<float, bf16, float>(const float*, int, int, long, const bf16*, const float*, int,
                                         float*, long, int, bool, int, cudaStream_t);
template int tc_conv<float, float, float>(const float*, int, int, long, const float*, const float*, int,
                                          float*, long, int, bool, int, cudaStream_t);

template <typename TA>
int tc_conv_wgrad(const float* dout, int cout, long dout_bstride, const TA* in, int cin,
                  long in_bstride, int D, int B, float* dW, cudaStream_t st) {
    const int NP = (cout + 15) & ~15;
    constexpr bool SPLIT_A = sizeof(TA) == 4;
    const int smem = (int)(2 * stage_bytes<SPLIT_A, true>(NP) + 1024);
    const unsigned cols = tmem_cols_for(NP);
    int lgD = 0;
    while ((1 << lgD) < D) ++lgD;
    const long nv = 1L << (3 * lgD);
    const int Kdim = cin * 27;
    const int ktiles = (Kdim + TM - 1) / TM;
    const long chunks = (long)B * nv / KC;
    // about four CTAs per SM over the k tiles and voxel slices, each slice >= 8 chunks
    const int slices = (int)std::max(1L, std::min<long>((4L * 148 + ktiles - 1) / ktiles, chunks / 8));
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    LDDMM_CUDA(cudaFuncSetAttribute(k_conv_wgrad_tc<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_conv_wgrad_tc<TA><<<dim3((unsigned)ktiles, (unsigned)slices), TM, smem, st>>>(
        dout, cout, dout_bstride, in, cin, in_bstride, lgD, B, NP, dW, cols);
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

template int tc_conv_wgrad<bf16>(const float*, int, long, const bf16*, int, long, int, int, float*,
                                 cudaStream_t);
template int tc_conv_wgrad<float>(const float*, int, long, const float*, int, long, int, int, float*,
                                  cudaStream_t);

int tc_conv_take_error(int* code) {
    int zero = 0;
    LDDMM_CUDA(cudaMemcpyFromSymbol(code, g_conv_error, sizeof(int)));
    LDDMM_CUDA(cudaMemcpyToSymbol(g_conv_error, &zero, sizeof(int)));
    return LDDMM_OK;
}

}  // namespace lddmm
