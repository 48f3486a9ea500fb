// Tensor-core (tcgen05) row GEMM for the x stages of pi and iota (Sec. 2.2):
//
//     OUT[row][n] = sum_k IN[row][k] * W[n][k],   rows = ncomp * nz * ny
//
// pi stage X:   IN = field rows (k = jx < nx),     W[2kx + {0,1}][jx] = {cos, -sin}(kx jx 2pi/nx)
// iota stage X: IN = (Re, Im) coefficient rows,    W[x][2kx + {0,1}] = w_kx {cos, -sin}(kx x 2pi/nx)
//
// Both are dense contractions with a small fixed W, so they run on the 5th-generation tensor
// cores: a persistent CTA per SM keeps W (split into hi + lo operands) resident in shared
// memory, TMA streams 128-row x 32-column FP32 tiles of IN into a 4-stage ring (128-byte swizzle, the K-major layout the MMA reads), four warps split each
// tile into hi and lo parts, one thread issues tcgen05.mma into a double-buffered TMEM
// accumulator, and four further warps read the accumulator back with tcgen05.ld and store it
// through TMA while the next tile is being split.
//
// Precision: FP32 inputs are represented as hi + lo with hi = x rounded to TF32 (low 13
// mantissa bits cleared) and lo = x - hi (exact in FP32); A*B ~ Ah*Bh + Ah*Bl + Al*Bh, FP32
// accumulation. The dropped Al*Bl term and the TF32 rounding of lo are ~2^-21 relative, so
// the result matches FP32 arithmetic to within its rounding. (BF16 hi + lo with kind::f16
// is the lower-precision variant of the same scheme.)
//
// Epilogue forms (EPI): 0 stores OUT row-major through TMA; 1 stores it transposed per slab of
// `rps` rows (OUT[slab][n][row in slab], so that the next stage reads it K-major: the x stage
// of pi feeding the Y stage); 2 and 3 finish a complex contraction written as a real GEMM
// over (Re, Im) input rows: rows come in (Re, Im) pairs of one complex line (adjacent lanes),
// the W rows in (cos, sin) pairs of one output position p, and each lane combines its own
// cos-sum with its partner's sin-sum (exchanged by a warp shuffle):
//   2 (pi, e^{-i theta}):  Re = C_re + S_im,  Im = C_im - S_re
//   3 (iota, e^{+i theta}): Re = C_re - S_im,  Im = C_im + S_re
// and stores OUT[slab][p0 + p][line].{re, im} (interleaved complex, line = kx fastest).
//
// Every mbarrier wait is bounded; on timeout the kernel records an error code in a device
// word (read by lddmm_device_error), stops issuing work, waits (bounded) for its own copies
// and MMAs, frees its TMEM and returns.
#include "common.cuh"
#include "lddmm.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace lddmm {

__device__ int g_tc_error = 0;

namespace {

constexpr int TM = 128;            // rows per tile (MMA M)
constexpr int CHUNK = 32;          // FP32 columns per TMA box = 128 bytes = one swizzle row
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
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

// Parity wait bounded by wall-clock time (and, as a backstop, by an iteration count);
// returns false on timeout. The clock is read only once the phase has been found incomplete
// (a %globaltimer read is slow next to a completed try_wait).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    const unsigned a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0; it != 0xFFFFFFFFu; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 255u) == 255u && now_ns() - t0 > limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// K-major operand, 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(unsigned saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version for sm_100 family
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

// W images with 2N <= 256 keep each chunk's hi rows and lo rows adjacent ([hi N rows | lo N
// rows]), so that A_hi * [B_hi | B_lo] is one MMA of width 2N and only A_lo * B_hi needs a
// second (2 instead of 3 MMAs per k-step; the epilogue adds the two column halves).
__host__ __device__ constexpr bool wcat(int N) { return 2 * N <= 256; }

// kind::tf32, FP32 accumulate, both operands K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// kind::f16 with BF16 A and B, FP32 accumulate, K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// BF16 split: hi = RN(x), lo = RN(x - hi); returns the packed bits of four elements
__device__ __forceinline__ void bf16_split4(float4 v, uint2& hi, uint2& lo) {
    __nv_bfloat16 h[4], l[4];
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = __float2bfloat16_rn(x[i]);
        l[i] = __float2bfloat16_rn(x[i] - __bfloat162float(h[i]));
    }
    hi.x = (unsigned)__bfloat16_as_ushort(h[0]) | ((unsigned)__bfloat16_as_ushort(h[1]) << 16);
    hi.y = (unsigned)__bfloat16_as_ushort(h[2]) | ((unsigned)__bfloat16_as_ushort(h[3]) << 16);
    lo.x = (unsigned)__bfloat16_as_ushort(l[0]) | ((unsigned)__bfloat16_as_ushort(l[1]) << 16);
    lo.y = (unsigned)__bfloat16_as_ushort(l[2]) | ((unsigned)__bfloat16_as_ushort(l[3]) << 16);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 32 consecutive TMEM columns of this warp's 32 lanes.
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

__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// byte offset of (row r, byte b in the 128-byte row) in a 1024-aligned SW128 tile
__device__ __forceinline__ unsigned sw128_off(int r, int b) {
    return (unsigned)(r * 128 + ((((b >> 4) ^ (r & 7))) << 4) + (b & 15));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];\n" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// named barrier of the four epilogue warps
__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, 128;\n" ::: "memory");
}

constexpr int NWORK = 8;                 // split warps 0..7
constexpr int NEPI = 4;                  // epilogue warps 8..11 (TMEM lane quarters 0..3)
constexpr int WARP_TMA = NWORK + NEPI;   // TMA producer warp
constexpr int WARP_MMA = WARP_TMA + 1;   // MMA issuer (and TMEM owner)
constexpr int NTHREADS_WS = 32 * (NWORK + NEPI + 2);
constexpr int NRAW_MAX = 6;
constexpr int NOP_MAX = 4;               // split-operand ring (released by MMA completion)
constexpr int TILE_B = TM * 128;         // 16 KB
// Ring depths. TF32: the landed FP32 tile is itself the hi operand (the tensor core reads
// only the upper 19 bits of a TF32 operand, i.e. the truncation hi = x with its low 13
// mantissa bits cleared), so only lo = x - hi is materialised (4 raw + 4 lo tiles) and a
// raw slot is released by MMA completion. BF16: hi and lo are both materialised (4 raw + 2 x
// 2 operand tiles) and the raw slot is released after the split.
// DEPTH 4, or 3 when the stage's W (hi + lo) is too large for the deeper rings (nx = 256).
__host__ __device__ constexpr int nraw(int prec, int depth) { return depth; }
__host__ __device__ constexpr int nop(int prec, int depth) { return prec == 0 ? depth : 2; }
static_assert(nraw(0, 4) == nop(0, 4) && nraw(0, 3) == nop(0, 3), "TF32 rings share release barriers");
__host__ __device__ constexpr int nop_planes(int prec) { return prec == 0 ? 1 : 2; }

}  // namespace

// Warp-specialised pipeline. Chunk q: tile t = q / nchunk, column block c = q % nchunk.
//   producer : wait raw_empty[q%NRAW], TMA 128 x 32 tile -> raw[q%NRAW]
//   split    : (warps 0-3) wait raw_full, wait op_empty[q%NOP]; split raw -> op (TF32: lo
//              only; BF16: hi and lo, then arrive raw_empty); arrive op_full
//   MMA warp : wait op_full (and, for c == 0, accempty of TMEM buffer t&1); 3 x k-step MMAs
//              (TF32: A hi read straight from raw); commit -> op_empty (TF32: which also frees
//              raw slot q%NRAW, the two rings having equal depth);
//              last chunk of the tile: commit -> accfull[t&1]
//   epilogue : (warps 4-7, concurrent with the split of the next tile) wait accfull[t&1];
//              TMEM 32-column blocks -> swizzled staging (2 buffers) -> TMA store; arrive
//              accempty[t&1]
// OUT is the 3-D tensor [ncomp][rpc][n_out] behind tmap_out (rows r = comp * rpc + local).
// PREC 0: TF32 hi + lo (4 k-steps of 8 per 32-column chunk). PREC 1: BF16 hi + lo, the 32
// elements of a chunk in the first 64 bytes of each 128-byte operand row (2 k-steps of 16).
template <int PREC, int DEPTH, int EPI>
__global__ void __launch_bounds__(NTHREADS_WS, 1)
k_tc_rowgemm(const __grid_constant__ CUtensorMap tmap_in, const __grid_constant__ CUtensorMap tmap_out,
             const unsigned char* __restrict__ w_image, int N, int kdim, long rows,
             float* __restrict__ out, long rpc, long comp_stride, int n_out, unsigned tmem_cols,
             int ptot, int p0, int lines, int nblk) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int NRAW = nraw(PREC, DEPTH);
    constexpr int NOP = nop(PREC, DEPTH);
    __shared__ uint64_t raw_full[NRAW_MAX], raw_empty[NRAW_MAX], op_full[NOP_MAX], op_empty[NOP_MAX], w_bar;
    __shared__ uint64_t accfull_bar[2], accempty_bar[2];
    __shared__ unsigned tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ long consumed_sh, issued_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // W: nblk column blocks of N rows, each an image of hi and lo parts (2 wbytes)
    const size_t wbytes = (size_t)nchunk * N * 128;
    unsigned char* w_hi = base;
    unsigned char* w_lo = base + wbytes;
    unsigned char* raw = base + 2 * wbytes * nblk;   // NRAW x 16 KB
    unsigned char* op_lo = raw + NRAW * TILE_B;      // NOP x 16 KB
    unsigned char* op_hi = op_lo + NOP * TILE_B;     // NOP x 16 KB (BF16 only)
    unsigned char* stg = op_lo + nop_planes(PREC) * NOP * TILE_B;  // 2 x 16 KB epilogue staging

    if (tid == 0) {
        mbar_init(&w_bar, 1);
        for (int i = 0; i < NRAW; ++i) {
            mbar_init(&raw_full[i], 1);
            mbar_init(&raw_empty[i], PREC == 0 ? 1 : NWORK);
        }
        for (int i = 0; i < NOP; ++i) {
            mbar_init(&op_full[i], NWORK);
            mbar_init(&op_empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull_bar[b], 1);
            mbar_init(&accempty_bar[b], NEPI);
        }
        abort_flag = 0;
        consumed_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        // W (hi | lo, already in the swizzled operand layout) arrives by bulk copies; only
        // the MMA warp waits for it
        const unsigned wtot = (unsigned)(2 * wbytes * nblk);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&w_bar)),
                     "r"(wtot)
                     : "memory");
        for (unsigned o = 0; o < wtot; o += 16384) {
            const unsigned len = min(16384u, wtot - o);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(w_hi + o)),
                "l"(w_image + o), "r"(len), "r"(smem_u32(&w_bar))
                : "memory");
        }
    }
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_holder;

    // work items: (row tile, column block) pairs, item = tile * nblk + block
    const long ntiles = (rows + TM - 1) / TM * nblk;
    const long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long total = my_tiles * nchunk;
    const uint32_t idesc = PREC == 0 ? idesc_tf32(N) : idesc_bf16(N);
    const bool cat = wcat(N);
    const int accw = cat ? 2 * N : N;    // accumulator columns per TMEM buffer
    const uint32_t idesc_cat = PREC == 0 ? idesc_tf32(accw) : idesc_bf16(accw);

    if (warp == WARP_TMA) {
        if (lane == 0) {
            // ring slot s, its use count u, column block c and global tile t advance
            // incrementally (no divisions in the issue loop)
            int s = 0, c = 0;
            unsigned u = 0;
            long t = blockIdx.x;
            for (long q = 0; q < total; ++q) {
                // TF32: raw slot s is operand slot s (equal ring depths), released by the same
                // MMA commit as the lo tile
                uint64_t* freed = PREC == 0 ? &op_empty[s] : &raw_empty[s];
                if (u > 0 && !mbar_wait(freed, (u - 1) & 1)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                tma_load_2d(raw + (size_t)s * TILE_B, &tmap_in, c * CHUNK, (int)(t / nblk * TM),
                            &raw_full[s], TILE_B);
                issued_sh = q + 1;
                if (++s == NRAW) {
                    s = 0;
                    ++u;
                }
                if (++c == nchunk) {
                    c = 0;
                    t += gridDim.x;
                }
            }
        }
    } else if (warp == WARP_MMA) {
        if (lane == 0) {
            if (total > 0 && !mbar_wait(&w_bar, 0)) abort_flag = 1;
            int o = 0, c = 0, s = 0;
            unsigned uo = 0;   // use count of operand slot o
            long t = 0;        // local tile index
            for (long q = 0; q < total && !abort_flag; ++q) {
                const int b = (int)(t & 1);
                if (c == 0 && t >= 2 && !mbar_wait(&accempty_bar[b], (unsigned)(((t >> 1) - 1) & 1))) {
                    abort_flag = 1;
                    break;
                }
                if (!mbar_wait(&op_full[o], uo & 1)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                fence_after();
                const unsigned d = tmem + (unsigned)(b * accw);
                const unsigned ah = PREC == 0 ? smem_u32(raw + (size_t)s * TILE_B)
                                              : smem_u32(op_hi + (size_t)o * TILE_B);
                const unsigned al = smem_u32(op_lo + (size_t)o * TILE_B);
                const size_t wblk = 2 * wbytes * (size_t)((blockIdx.x + t * gridDim.x) % nblk);
                const unsigned wh = smem_u32(w_hi + wblk + (size_t)c * (cat ? 2 * N : N) * 128);
                const unsigned wl = cat ? wh + (unsigned)(N * 128)
                                        : smem_u32(w_lo + wblk + (size_t)c * N * 128);
                if (PREC == 0) {
#pragma unroll
                    for (int kk = 0; kk < CHUNK / 8; ++kk) {
                        const unsigned ko = kk * 32;
                        const unsigned acc = (c > 0 || kk > 0) ? 1u : 0u;
                        if (cat) {
                            mma_tf32(d, sw128_desc(ah + ko), sw128_desc(wh + ko), idesc_cat, acc);
                        } else {
                            mma_tf32(d, sw128_desc(ah + ko), sw128_desc(wh + ko), idesc, acc);
                            mma_tf32(d, sw128_desc(ah + ko), sw128_desc(wl + ko), idesc, 1u);
                        }
                        mma_tf32(d, sw128_desc(al + ko), sw128_desc(wh + ko), idesc, 1u);
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < CHUNK / 16; ++kk) {
                        const unsigned ko = kk * 32;
                        const unsigned acc = (c > 0 || kk > 0) ? 1u : 0u;
                        if (cat) {
                            mma_bf16(d, sw128_desc(ah + ko), sw128_desc(wh + ko), idesc_cat, acc);
                        } else {
                            mma_bf16(d, sw128_desc(ah + ko), sw128_desc(wh + ko), idesc, acc);
                            mma_bf16(d, sw128_desc(ah + ko), sw128_desc(wl + ko), idesc, 1u);
                        }
                        mma_bf16(d, sw128_desc(al + ko), sw128_desc(wh + ko), idesc, 1u);
                    }
                }
                mma_commit(&op_empty[o]);
                if (c == nchunk - 1) mma_commit(&accfull_bar[b]);
                if (++o == NOP) {
                    o = 0;
                    ++uo;
                }
                if (++s == NRAW) s = 0;
                if (++c == nchunk) {
                    c = 0;
                    ++t;
                }
            }
        }
    } else if (warp >= NWORK && EPI != 0) {
        // ------------------------------------------- epilogue warps, direct-store forms
        const int et = tid - 32 * NWORK;
        const int quarter = (warp - NWORK) & 3;
        for (long t = 0; t < my_tiles; ++t) {
            // warp-uniform decisions: the completion step below exchanges values between lanes
            if (__any_sync(0xffffffffu, abort_flag != 0)) break;
            const int b = (int)(t & 1);
            const bool ok = mbar_wait(&accfull_bar[b], (unsigned)((t >> 1) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                abort_flag = 1;
                break;
            }
            fence_after();
            const long item = blockIdx.x + t * gridDim.x;
            const long row = item / nblk * TM + et;
            const int pblk = p0 + (int)(item % nblk) * (N >> 1);   // first position of the block
            const bool live = row < rows;
            const long slab = row / rpc;
            const long r = row - slab * rpc;        // row within its slab
            for (int c0 = 0; c0 < N; c0 += 32) {
                float v[32];
                const unsigned trow = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * accw + c0);
                tmem_ld32(trow, v);
                if (cat) {
                    float v2[32];
                    tmem_ld32(trow + (unsigned)N, v2);
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] += v2[i];
                }
                if (EPI == 1) {
                    // OUT[slab][n][r]: for each n the warp's 32 rows are 32 consecutive floats
                    if (live) {
                        float* dst = out + (slab * N + c0) * rpc + r;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i < n_out) dst[(long)i * rpc] = v[i];
                    }
                } else {
                    // rows r = 2 line + c (c = 0: Re, 1: Im); columns 2 p + {0: cos, 1: sin}
                    const int c = (int)(r & 1);
                    const long line = r >> 1;
                    const float sg = ((EPI == 2) == (c == 0)) ? 1.f : -1.f;
                    float* dst = out + ((slab * ptot + pblk + (c0 >> 1)) * lines + line) * 2 + c;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float sp = __shfl_xor_sync(0xffffffffu, v[2 * i + 1], 1);
                        if (live && (c0 >> 1) + i < (n_out >> 1))
                            dst[(long)i * lines * 2] = v[2 * i] + sg * sp;
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty_bar[b]);
        }
    } else if (warp >= NWORK) {
        // ---------------------------------------------------------------- epilogue warps
        const int et = tid - 32 * NWORK;   // 0 .. 127: the tile row this thread stores
        const int quarter = (warp - NWORK) & 3;  // TMEM lanes 32 quarter .. 32 quarter + 31
        long sblock = 0;                   // staging blocks used so far (buffer = sblock & 1)
        for (long t = 0; t < my_tiles && !abort_flag; ++t) {
            const int b = (int)(t & 1);
            if (!mbar_wait(&accfull_bar[b], (unsigned)((t >> 1) & 1))) {
                abort_flag = 1;
                break;
            }
            fence_after();
            const long tg = blockIdx.x + t * gridDim.x;
            const long row0 = tg * TM;
            const long comp0 = row0 / rpc;
            const long local0 = row0 - comp0 * rpc;
            const long split = rpc - local0;  // tile rows at or past `split` belong to comp0 + 1
            const long row = row0 + et;
            for (int c0 = 0; c0 < N; c0 += 32) {
                float v[32];
                const unsigned trow = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * accw + c0);
                tmem_ld32(trow, v);
                if (cat) {   // + the A_hi * B_lo half
                    float v2[32];
                    tmem_ld32(trow + (unsigned)N, v2);
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] += v2[i];
                }
                unsigned char* sb = stg + (size_t)(sblock & 1) * TILE_B;
                // the store issued two blocks ago from this buffer must have read it
                if (et == 0) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
                epi_sync();
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4*>(sb + sw128_off(et, j * 16)) =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                epi_sync();
                if (et == 0)
                    tma_store_3d(&tmap_out, sb, c0, (int)local0, (int)comp0);
                // rows of a second component (only when a tile straddles a component boundary)
                if (et >= split && row < rows) {
                    float* dst = out + (comp0 + 1) * comp_stride + (et - split) * n_out + c0;
                    const int nv = min(32, n_out - c0);
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < nv) dst[i] = v[i];
                }
                ++sblock;
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty_bar[b]);
        }
        if (et == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    } else {
        // ---------------------------------------------------------------- split warps
        const int wt = tid;  // 0 .. 32 NWORK - 1
        int s = 0, o = 0;
        unsigned us = 0, uo = 0;   // use counts of raw slot s and operand slot o
        for (long q = 0; q < total; ++q) {
            if (!mbar_wait(&raw_full[s], us & 1) || (uo > 0 && !mbar_wait(&op_empty[o], (uo - 1) & 1)) ||
                abort_flag) {
                abort_flag = 1;
                break;
            }
            const float4* src = reinterpret_cast<const float4*>(raw + (size_t)s * TILE_B);
            float4* hi = reinterpret_cast<float4*>(op_hi + (size_t)o * TILE_B);
            float4* lo = reinterpret_cast<float4*>(op_lo + (size_t)o * TILE_B);
#pragma unroll
            for (int i = 0; i < TILE_B / 16 / (32 * NWORK); ++i) {
                const int e = wt + i * 32 * NWORK;
                const float4 v = src[e];
                if (PREC == 0) {
                    const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                    lo[e] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                } else {
                    // raw 16-byte chunk e = (row r, physical chunk p) holds logical chunk
                    // j = p ^ (r & 7), i.e. elements 4j..4j+3 -> bf16 bytes 8j..8j+7
                    const int r = e >> 3, pch = e & 7, j = pch ^ (r & 7);
                    const unsigned off = sw128_off(r, 8 * j);
                    uint2 h2, l2;
                    bf16_split4(v, h2, l2);
                    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(hi) + off) = h2;
                    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(lo) + off) = l2;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                if (PREC != 0) mbar_arrive(&raw_empty[s]);
                mbar_arrive(&op_full[o]);
            }
            if (wt == 0) consumed_sh = q + 1;
            if (++s == NRAW) {
                s = 0;
                ++us;
            }
            if (++o == NOP) {
                o = 0;
                ++uo;
            }
        }
    }

    __syncthreads();
    if (abort_flag && tid == 0) {
        atomicExch(&g_tc_error, LDDMM_ETIMEOUT);
        for (long qq = consumed_sh; qq < issued_sh; ++qq)
            mbar_wait(&raw_full[qq % NRAW], (unsigned)((qq / NRAW) & 1));
    }
    if (abort_flag && warp == WARP_MMA && lane == 0) {
        mma_commit(&accfull_bar[0]);
        mbar_wait(&accfull_bar[0], 0);
        mbar_wait(&accfull_bar[0], 1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == WARP_MMA)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(tmem_cols));
}

template <int PREC>
__device__ __forceinline__ void mma_kind(unsigned tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
    if (PREC == 0) mma_tf32(tmem_d, a, b, idesc, accumulate);
    else mma_bf16(tmem_d, a, b, idesc, accumulate);
}

// Transposed form for narrow outputs (16 <= N <= 64: the x stage of pi), OUT^T = W IN^T.
// One tcgen05.mma instruction takes about the same time for every N up to 256 at M = 128, so
// the row GEMM above (input rows as A, N = 2 N_out and N_out per k-step) leaves most of each
// instruction's array idle when N is small. Here W is the A operand and the input rows are B,
// and one instruction per k-step covers 128 input rows and all four split products:
//   A (MA rows)  = W rows interleaved: row 2n + h = W_h[n] (h = 0 hi, 1 lo; n < N), zero rows
//                  from 2N on; MA = 64 for N <= 32, else 128
//   B (256 rows) = [IN_hi (128 rows); IN_lo (128 rows)] of one 32-column chunk
//   D[2n + h][j]: j < 128 the input row j times W_h, j >= 128 the lo part of row j - 128
//   OUT[row j][n] = D[2n][j] + D[2n][128 + j] + D[2n + 1][j] + D[2n + 1][128 + j]
//                 = (W_hi + W_lo)(IN_hi + IN_lo) (all four products)
// The epilogue adds the two column halves in each lane and the lane pair (2n, 2n + 1) by a
// shuffle, and stores OUT transposed per slab of rpc rows, OUT[slab][n][row in slab] (the form
// the Y stage reads). D row r of an M = 128 MMA is TMEM lane r; of an M = 64 MMA, lane
// 32 (r / 16) + r % 16 (the first 16 lanes of each quarter). Warp roles as in k_tc_rowgemm:
// 0-7 split the landed tile into hi and lo (both materialised, so the raw slot is released
// right after the split), 8-11 epilogue (the lane quarters holding rows < 2N), 12 TMA
// producer, 13 MMA issuer. The smaller A image of MA = 64 leaves room for a deeper raw ring.
// W's operand image is
// rebuilt in shared memory from the row GEMM's image (per chunk [hi N rows | lo N rows],
// 128-byte swizzle) by warps 0-11 while the first tiles load.
constexpr int TR_OP_B = 2 * TILE_B;   // one B operand: hi and lo tiles, 32 KB
constexpr int TR_NOP = 2;             // B operand ring

template <int PREC, int NRAW>
__global__ void __launch_bounds__(NTHREADS_WS, 1)
k_tc_rowgemm_t(const __grid_constant__ CUtensorMap tmap_in, const unsigned char* __restrict__ w_image,
               int N, int kdim, long rows, float* __restrict__ out, long rpc, int n_out, int ma) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t raw_full[NRAW], raw_empty[NRAW], op_full[TR_NOP], op_empty[TR_NOP], w_bar;
    __shared__ uint64_t accfull_bar[2], accempty_bar[2];
    __shared__ unsigned tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ long consumed_sh, issued_sh;
    constexpr unsigned TMEM_COLS = 2 * 2 * TM;   // two accumulators of 256 columns

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int abytes = ma * 128;                             // one chunk of the A image
    unsigned char* wT = base;                                // nchunk x abytes
    unsigned char* raw = wT + (size_t)nchunk * abytes;       // NRAW x 16 KB
    unsigned char* ops = raw + (size_t)NRAW * TILE_B;        // TR_NOP x 32 KB

    if (tid == 0) {
        mbar_init(&w_bar, 1);
        for (int i = 0; i < NRAW; ++i) {
            mbar_init(&raw_full[i], 1);
            mbar_init(&raw_empty[i], NWORK);
        }
        for (int i = 0; i < TR_NOP; ++i) {
            mbar_init(&op_full[i], NWORK);
            mbar_init(&op_empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull_bar[b], 1);
            mbar_init(&accempty_bar[b], NEPI);
        }
        abort_flag = 0;
        consumed_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_holder;

    const long ntiles = (rows + TM - 1) / TM;
    const long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long total = my_tiles * nchunk;

    if (warp < WARP_TMA) {
        // A image: row r = 2n + h of chunk c from source row c 2N + h N + n; each 16-byte piece
        // j moves from its source position j ^ (n & 7) to j ^ (r & 7) (rows of 128 bytes,
        // 8-row swizzle groups; 2N is a multiple of 32, so chunk bases keep phase 0)
        // (eight loads in flight per thread before their stores)
        constexpr int TPB = 32 * WARP_TMA, BATCH = 8;
        const int cshift = ma == 64 ? 9 : 10;                // log2(ma * 8 pieces)
        const int npieces = nchunk * ma * 8;
        for (int b0 = 0; b0 < npieces; b0 += BATCH * TPB) {
            uint4 v[BATCH];
            int dst[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                const int idx = b0 + u * TPB + tid;
                const int c = idx >> cshift, rem = idx & ((1 << cshift) - 1), r = rem >> 3, j = rem & 7;
                const int n = r >> 1, h = r & 1;
                v[u] = make_uint4(0u, 0u, 0u, 0u);
                dst[u] = idx < npieces ? (c * ma + r) * 128 + ((j ^ (r & 7)) << 4) : -1;
                if (idx < npieces && n < N) {
                    const int sr = c * 2 * N + h * N + n;
                    v[u] = __ldg(reinterpret_cast<const uint4*>(w_image + (size_t)sr * 128 + ((j ^ (sr & 7)) << 4)));
                }
            }
#pragma unroll
            for (int u = 0; u < BATCH; ++u)
                if (dst[u] >= 0) *reinterpret_cast<uint4*>(wT + dst[u]) = v[u];
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("bar.sync 2, %0;\n" ::"r"(32 * WARP_TMA) : "memory");
        if (tid == 0) mbar_arrive(&w_bar);
    }

    if (warp == WARP_TMA) {
        if (lane == 0) {
            int s = 0, c = 0;
            unsigned u = 0;
            long t = blockIdx.x;
            for (long q = 0; q < total; ++q) {
                if (u > 0 && !mbar_wait(&raw_empty[s], (u - 1) & 1)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                tma_load_2d(raw + (size_t)s * TILE_B, &tmap_in, c * CHUNK, (int)(t * TM), &raw_full[s], TILE_B);
                issued_sh = q + 1;
                if (++s == NRAW) {
                    s = 0;
                    ++u;
                }
                if (++c == nchunk) {
                    c = 0;
                    t += gridDim.x;
                }
            }
        }
    } else if (warp == WARP_MMA) {
        if (lane == 0) {
            if (total > 0 && !mbar_wait(&w_bar, 0)) abort_flag = 1;
            const uint32_t idesc = (PREC == 0 ? idesc_tf32(2 * TM) : idesc_bf16(2 * TM)) & ~(31u << 24) |
                                   ((uint32_t)(ma >> 4) << 24);   // M = ma
            constexpr int KSTEP = PREC == 0 ? 8 : 16;   // elements per MMA k-step
            int o = 0, c = 0;
            unsigned uo = 0;
            long t = 0;
            for (long q = 0; q < total && !abort_flag; ++q) {
                const int b = (int)(t & 1);
                if (c == 0 && t >= 2 && !mbar_wait(&accempty_bar[b], (unsigned)(((t >> 1) - 1) & 1))) {
                    abort_flag = 1;
                    break;
                }
                if (!mbar_wait(&op_full[o], uo & 1)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                fence_after();
                const unsigned d = tmem + (unsigned)(b * 2 * TM);
                const unsigned a = smem_u32(wT + (size_t)c * abytes);
                const unsigned bo = smem_u32(ops + (size_t)o * TR_OP_B);
#pragma unroll
                for (int kk = 0; kk < CHUNK / KSTEP; ++kk) {
                    const unsigned ko = kk * 32;
                    mma_kind<PREC>(d, sw128_desc(a + ko), sw128_desc(bo + ko), idesc,
                                   (c > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&op_empty[o]);
                if (c == nchunk - 1) mma_commit(&accfull_bar[b]);
                if (++o == TR_NOP) {
                    o = 0;
                    ++uo;
                }
                if (++c == nchunk) {
                    c = 0;
                    ++t;
                }
            }
        }
    } else if (warp >= NWORK) {
        // ---------------------------------------------------------------- epilogue warps
        const int quarter = (warp - NWORK) & 3;        // TMEM lanes 32 quarter .. + 31
        const int qrows = ma / 4;                      // D rows per lane quarter (lanes 0 .. qrows-1)
        const bool active = quarter * (qrows / 2) < N; // lane l holds row 2n + h, n = quarter qrows / 2 + l / 2
        const int n = quarter * (qrows / 2) + (lane >> 1), h = lane & 1;
        const bool lane_ok = lane < qrows;
        const bool vec = (rpc % 16) == 0;              // 16-row groups never straddle a slab
        for (long t = 0; t < my_tiles; ++t) {
            if (__any_sync(0xffffffffu, abort_flag != 0)) break;
            const int b = (int)(t & 1);
            const bool ok = mbar_wait(&accfull_bar[b], (unsigned)((t >> 1) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                abort_flag = 1;
                break;
            }
            fence_after();
            const long row0 = (blockIdx.x + t * gridDim.x) * TM;
            if (active) {
                for (int cb = 0; cb < TM / 32; ++cb) {
                    float v[32], w[32];
                    const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * 2 * TM + cb * 32);
                    tmem_ld32(ta, v);
                    tmem_ld32(ta + TM, w);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float sum = v[i] + w[i];
                        v[i] = sum + __shfl_xor_sync(0xffffffffu, sum, 1);
                    }
                    // the lane pair both hold rows cb 32 .. cb 32 + 31 of output n: lane h
                    // stores the 16 rows from 16 h
                    float o16[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) o16[i] = h ? v[16 + i] : v[i];
                    const long r0 = row0 + cb * 32 + 16 * h;
                    if (lane_ok && n < n_out) {
                        if (vec) {
                            if (r0 < rows) {
                                const long slab = r0 / rpc, rr = r0 - slab * rpc;
                                float4* dst = reinterpret_cast<float4*>(out + (slab * N + n) * rpc + rr);
#pragma unroll
                                for (int k = 0; k < 4; ++k)
                                    dst[k] = make_float4(o16[4 * k], o16[4 * k + 1], o16[4 * k + 2], o16[4 * k + 3]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const long r = r0 + i;
                                if (r < rows) {
                                    const long slab = r / rpc;
                                    out[(slab * N + n) * rpc + (r - slab * rpc)] = o16[i];
                                }
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty_bar[b]);
        }
    } else {
        // ---------------------------------------------------------------- split warps
        int s = 0, o = 0;
        unsigned us = 0, uo = 0;
        for (long q = 0; q < total; ++q) {
            if (!mbar_wait(&raw_full[s], us & 1) || (uo > 0 && !mbar_wait(&op_empty[o], (uo - 1) & 1)) ||
                abort_flag) {
                abort_flag = 1;
                break;
            }
            const float4* src = reinterpret_cast<const float4*>(raw + (size_t)s * TILE_B);
            unsigned char* hi = ops + (size_t)o * TR_OP_B;
            unsigned char* lo = hi + TILE_B;
            if (PREC == 0) {
#pragma unroll
                for (int i = 0; i < TILE_B / 16 / (32 * NWORK); ++i) {
                    const int e = tid + i * 32 * NWORK;
                    const float4 v = src[e];
                    const float4 hv = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                    reinterpret_cast<float4*>(hi)[e] = hv;
                    reinterpret_cast<float4*>(lo)[e] = make_float4(v.x - hv.x, v.y - hv.y, v.z - hv.z, v.w - hv.w);
                }
            } else {
                // raw 16-byte chunk e = (row r, physical chunk p) holds logical chunk
                // j = p ^ (r & 7), elements 4j .. 4j + 3 -> BF16 bytes 8j .. 8j + 7. The
                // physical pair (2m', 2m' + 1) holds the logical pair (2m, 2m + 1),
                // m = (2m' ^ (r & 7)) / 2, i.e. one 16-byte BF16 piece of hi and of lo
#pragma unroll
                for (int i = 0; i < TILE_B / 32 / (32 * NWORK); ++i) {
                    const int e0 = 2 * (tid + i * 32 * NWORK);
                    const int r = e0 >> 3, j0 = (e0 & 7) ^ (r & 7);
                    const float4 va = src[e0], vb = src[e0 + 1];
                    const bool swap = (j0 & 1) != 0;        // e0 holds the odd logical chunk
                    uint2 ha, la, hb, lb;
                    bf16_split4(swap ? vb : va, ha, la);
                    bf16_split4(swap ? va : vb, hb, lb);
                    const unsigned off = sw128_off(r, 16 * (j0 >> 1));
                    *reinterpret_cast<uint4*>(hi + off) = make_uint4(ha.x, ha.y, hb.x, hb.y);
                    *reinterpret_cast<uint4*>(lo + off) = make_uint4(la.x, la.y, lb.x, lb.y);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&raw_empty[s]);
                mbar_arrive(&op_full[o]);
            }
            if (tid == 0) consumed_sh = q + 1;
            if (++s == NRAW) {
                s = 0;
                ++us;
            }
            if (++o == TR_NOP) {
                o = 0;
                ++uo;
            }
        }
    }

    __syncthreads();
    if (abort_flag && tid == 0) {
        atomicExch(&g_tc_error, LDDMM_ETIMEOUT);
        for (long qq = consumed_sh; qq < issued_sh; ++qq)
            mbar_wait(&raw_full[qq % NRAW], (unsigned)((qq / NRAW) & 1));
    }
    if (abort_flag && warp == WARP_MMA && lane == 0) {
        mma_commit(&accfull_bar[0]);
        mbar_wait(&accfull_bar[0], 0);
        mbar_wait(&accfull_bar[0], 1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == WARP_MMA)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

// W (N x kdim FP32) -> its shared-memory operand image: hi and lo parts, each nchunk x N rows
// of 128 bytes in the 128-byte-swizzled K-major layout (zero past kdim); per chunk [hi | lo]
// when wcat(N), else all hi chunks then all lo chunks.
template <int PREC>
__global__ void k_build_wimage(const float* __restrict__ W, int N, int kdim,
                               unsigned char* __restrict__ img) {
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nchunk * N * CHUNK) return;
    const int c = e / (N * CHUNK);
    const int rem = e - c * N * CHUNK;
    const int n = rem / CHUNK, k = rem - n * CHUNK;
    const int kk = c * CHUNK + k;
    const float w = kk < kdim ? W[(long)n * kdim + kk] : 0.f;
    const size_t wbytes = (size_t)nchunk * N * 128;
    // hi and lo blocks: adjacent per chunk (wcat) or two separate halves of the image
    const size_t hbase = wcat(N) ? (size_t)c * 2 * N * 128 : (size_t)c * N * 128;
    const size_t lbase = wcat(N) ? hbase + (size_t)N * 128 : wbytes + hbase;
    if (PREC == 0) {
        const float h = tf32_hi(w);
        const unsigned off = sw128_off(n, k * 4);
        *reinterpret_cast<float*>(img + hbase + off) = h;
        *reinterpret_cast<float*>(img + lbase + off) = w - h;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        const __nv_bfloat16 l = __float2bfloat16_rn(w - __bfloat162float(h));
        const unsigned off = sw128_off(n, k * 2);
        *reinterpret_cast<__nv_bfloat16*>(img + hbase + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(img + lbase + off) = l;
    }
}

long tc_wimage_bytes(int N, int kdim) {
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    return 2L * nchunk * N * 128;
}

int tc_build_wimage(const float* W, int N, int kdim, int prec, unsigned char* img,
                    cudaStream_t st) {
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    const int total = nchunk * N * CHUNK;
    // BF16 images leave the upper 64 bytes of each operand row unused: clear them
    LDDMM_CUDA(cudaMemsetAsync(img, 0, tc_wimage_bytes(N, kdim), st));
    {
        KTRACE("twiddle", st, 12.0 * total, 0);
        if (prec == 0)
            k_build_wimage<0><<<(total + 255) / 256, 256, 0, st>>>(W, N, kdim, img);
        else
            k_build_wimage<1><<<(total + 255) / 256, 256, 0, st>>>(W, N, kdim, img);
    }
    LDDMM_CHECK_LAUNCH();
    return LDDMM_OK;
}

// --------------------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// W hi + lo, the raw ring, the split operands and (TMA-store epilogue only) two staging
// tiles, + alignment slack
int tc_smem_bytes(int N, int kdim, int prec, int depth, int epi, int nblk = 1) {
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    return 2 * nchunk * N * 128 * nblk +
           (nraw(prec, depth) + nop_planes(prec) * nop(prec, depth) + (epi == 0 ? 2 : 0)) * TILE_B + 1024;
}

constexpr int kTcSmemLimit = 220 * 1024;

// the deepest ring that fits (4, else 3, else 2 for the direct-store epilogues); 0 if none
int tc_depth(int N, int kdim, int prec, int epi, int nblk = 1) {
    if (tc_smem_bytes(N, kdim, prec, 4, epi, nblk) <= kTcSmemLimit) return 4;
    if (tc_smem_bytes(N, kdim, prec, 3, epi, nblk) <= kTcSmemLimit) return 3;
    if (epi != 0 && tc_smem_bytes(N, kdim, prec, 2, epi, nblk) <= kTcSmemLimit) return 2;
    return 0;
}

template <int PREC, int DEPTH, int EPI>
cudaError_t tc_launch(int grid, int smem, cudaStream_t st, const CUtensorMap& map, const CUtensorMap& omap,
                      const unsigned char* W, int N, int kdim, long rows, float* out, long rpc,
                      long comp_stride, int n_out, unsigned cols, int ptot, int p0, int lines,
                      int nblk) {
    static int attr = 0;   // largest dynamic size requested so far (under the caller's lock)
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_rowgemm<PREC, DEPTH, EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    k_tc_rowgemm<PREC, DEPTH, EPI><<<grid, NTHREADS_WS, smem, st>>>(
        map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk);
    return cudaGetLastError();
}

template <int PREC, int EPI>
cudaError_t tc_launch_depth(int depth, int grid, int smem, cudaStream_t st, const CUtensorMap& map,
                            const CUtensorMap& omap, const unsigned char* W, int N, int kdim,
                            long rows, float* out, long rpc, long comp_stride, int n_out,
                            unsigned cols, int ptot, int p0, int lines, int nblk) {
    if (depth == 4)
        return tc_launch<PREC, 4, EPI>(grid, smem, st, map, omap, W, N, kdim, rows, out, rpc,
                                       comp_stride, n_out, cols, ptot, p0, lines, nblk);
    if (depth == 3)
        return tc_launch<PREC, 3, EPI>(grid, smem, st, map, omap, W, N, kdim, rows, out, rpc,
                                       comp_stride, n_out, cols, ptot, p0, lines, nblk);
    if constexpr (EPI != 0) {
        if (depth == 2)
            return tc_launch<PREC, 2, EPI>(grid, smem, st, map, omap, W, N, kdim, rows, out, rpc,
                                           comp_stride, n_out, cols, ptot, p0, lines, nblk);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool tc_rowgemm_supported(int N, int kdim, long rows, const void* in, long in_row_floats,
                          int epi, int prec, int nblk) {
    if (N < 16 || N > 256 || (N % 16) != 0) return false;
    if (kdim < 1 || (in_row_floats % 4) != 0) return false;
    if ((reinterpret_cast<uintptr_t>(in) & 15) != 0) return false;
    if (rows < 1 || rows > 0x7fffffffL) return false;
    if (epi < 0 || epi > 3 || (epi >= 2 && (rows & 1))) return false;
    if (nblk < 1 || (nblk > 1 && epi < 2)) return false;
    if (prec < 0) {
        if (tc_depth(N, kdim, 0, epi, nblk) == 0 || tc_depth(N, kdim, 1, epi, nblk) == 0) return false;
    } else if (tc_depth(N, kdim, prec, epi, nblk) == 0) {
        return false;
    }
    return encode_fn() != nullptr;
}

int tc_rowgemm(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
               int N, int prec, float* out, long rpc, long comp_stride, int n_out,
               const char* trace_name, double trace_bytes, cudaStream_t st) {
    return tc_rowgemm_ex(in, rows, kdim, in_row_floats, W, N, prec, 0, out, rpc, comp_stride,
                         n_out, 0, 0, 0, 1, trace_name, trace_bytes, st);
}

// in: rows x in_row_floats FP32 (the first kdim columns are used), W: nblk blocks of N x kdim
// FP32 as consecutive operand images (tc_wimage_bytes(N, kdim) each).
int tc_rowgemm_ex(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
                  int N, int prec, int epi, float* out, long rpc, long comp_stride, int n_out,
                  int ptot, int p0, int lines, int nblk, const char* trace_name,
                  double trace_bytes, cudaStream_t st) {
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)in_row_floats, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)in_row_floats * 4};
    cuuint32_t box[2] = {CHUNK, TM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(in), dims,
                             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tc_rowgemm: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return LDDMM_ECUDA;
    }
    if (epi < 0 || epi > 3 || rpc < 1 || (epi >= 2 && (rows & 1)) || nblk < 1 ||
        (nblk > 1 && epi < 2)) {
        set_error("tc_rowgemm: bad epilogue arguments");
        return LDDMM_EINVAL;
    }
    // output of the TMA-store epilogue: [ncomp][rpc][n_out] with component stride comp_stride
    // floats (the direct-store epilogues address OUT themselves; the map is then unused)
    CUtensorMap omap = map;
    if (epi == 0) {
        const long ncomp_out = (rows + rpc - 1) / rpc;
        cuuint64_t odims[3] = {(cuuint64_t)n_out, (cuuint64_t)rpc, (cuuint64_t)ncomp_out};
        cuuint64_t ostr[2] = {(cuuint64_t)n_out * 4, (cuuint64_t)(ncomp_out > 1 ? comp_stride : rpc * n_out) * 4};
        cuuint32_t obox[3] = {32, TM, 1};
        cuuint32_t oestr[3] = {1, 1, 1};
        r = encode_fn()(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out, odims, ostr, obox, oestr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("tc_rowgemm: cuTensorMapEncodeTiled (output) failed (" + std::to_string((int)r) + ")");
            return LDDMM_ECUDA;
        }
    }
    const int depth = tc_depth(N, kdim, prec, epi, nblk);
    if (depth == 0) {
        set_error("tc_rowgemm: W too large for shared memory");
        return LDDMM_EINVAL;
    }
    const int smem = tc_smem_bytes(N, kdim, prec, depth, epi, nblk);
    // two accumulators at columns 0 and N; the epilogue reads 32-column blocks, so the
    // second buffer's last block ends at N + roundup(N, 32)
    const int accw = wcat(N) ? 2 * N : N;
    const int need_cols = accw + (wcat(N) ? N : 0) + ((N + 31) / 32) * 32;
    unsigned cols = 32;
    while ((int)cols < need_cols) cols <<= 1;
    if (cols > 512) {
        set_error("tc_rowgemm: N too large for tensor memory");
        return LDDMM_EINVAL;
    }
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, v = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        nsm = v;
    }
    const long ntiles = (rows + TM - 1) / TM * nblk;
    const int grid = (int)std::min<long>(ntiles, nsm);
    {
        KTRACE(trace_name, st, trace_bytes, 2.0 * rows * (double)N * kdim);
        static std::mutex mu;   // serialises the per-instantiation shared-memory attribute
        std::lock_guard<std::mutex> lock(mu);
        cudaError_t e = cudaErrorInvalidValue;
        switch (prec * 4 + epi) {
            case 0: e = tc_launch_depth<0, 0>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 1: e = tc_launch_depth<0, 1>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 2: e = tc_launch_depth<0, 2>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 3: e = tc_launch_depth<0, 3>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 4: e = tc_launch_depth<1, 0>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 5: e = tc_launch_depth<1, 1>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 6: e = tc_launch_depth<1, 2>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            case 7: e = tc_launch_depth<1, 3>(depth, grid, smem, st, map, omap, W, N, kdim, rows, out, rpc, comp_stride, n_out, cols, ptot, p0, lines, nblk); break;
            default: break;
        }
        LDDMM_CUDA(e);
    }
    return LDDMM_OK;
}

// ------------------------------------------------- transposed form (narrow outputs)
namespace {

// rows of the A image: 64 (the M = 64 MMA) when the 2N interleaved W rows fit, else 128
int tc_t_ma(int N) { return 2 * N <= 64 ? 64 : 128; }

int tc_t_smem_bytes(int kdim, int nraw, int ma) {
    const int nchunk = (kdim + CHUNK - 1) / CHUNK;
    return nchunk * ma * 128 + nraw * TILE_B + TR_NOP * TR_OP_B + 1024;
}

// the deepest raw ring (6, 4, 3 or 2 slots) that fits with W's image; 0 if none
int tc_t_depth(int kdim, int ma) {
    for (int d : {6, 4, 3, 2})
        if (tc_t_smem_bytes(kdim, d, ma) <= kTcSmemLimit) return d;
    return 0;
}

template <int PREC, int NRAW>
cudaError_t tc_t_launch(int grid, int smem, cudaStream_t st, const CUtensorMap& map,
                        const unsigned char* W, int N, int kdim, long rows, float* out, long rpc,
                        int n_out, int ma) {
    static int attr = 0;   // largest dynamic size requested so far (under the caller's lock)
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_rowgemm_t<PREC, NRAW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    k_tc_rowgemm_t<PREC, NRAW><<<grid, NTHREADS_WS, smem, st>>>(map, W, N, kdim, rows, out, rpc, n_out, ma);
    return cudaGetLastError();
}

}  // namespace

bool tc_rowgemm_t_supported(int N, int kdim, long rows, const void* in, long in_row_floats) {
    if (N < 16 || N > 64 || (N % 16) != 0) return false;
    if (kdim < 1 || kdim > in_row_floats || (in_row_floats % 4) != 0) return false;
    if ((reinterpret_cast<uintptr_t>(in) & 15) != 0) return false;
    if (rows < 1 || rows > 0x7fffffffL) return false;
    if (tc_t_depth(kdim, tc_t_ma(N)) == 0) return false;
    return encode_fn() != nullptr;
}

int tc_rowgemm_t(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
                 int N, int prec, float* out, long rpc, int n_out, const char* trace_name,
                 double trace_bytes, cudaStream_t st) {
    if (!tc_rowgemm_t_supported(N, kdim, rows, in, in_row_floats) || rpc < 1 || n_out < 1 ||
        n_out > N || (prec != 0 && prec != 1) || (reinterpret_cast<uintptr_t>(out) & 15) != 0) {
        set_error("tc_rowgemm_t: unsupported arguments");
        return LDDMM_EINVAL;
    }
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)in_row_floats, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)in_row_floats * 4};
    cuuint32_t box[2] = {CHUNK, TM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(in), dims,
                             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tc_rowgemm_t: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return LDDMM_ECUDA;
    }
    const int ma = tc_t_ma(N);
    const int depth = tc_t_depth(kdim, ma);
    const int smem = tc_t_smem_bytes(kdim, depth, ma);
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, v = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        nsm = v;
    }
    const long ntiles = (rows + TM - 1) / TM;
    const int grid = (int)std::min<long>(ntiles, nsm);
    {
        KTRACE(trace_name, st, trace_bytes, 2.0 * rows * (double)N * kdim);
        static std::mutex mu;   // serialises the per-instantiation shared-memory attribute
        std::lock_guard<std::mutex> lock(mu);
        cudaError_t e = cudaErrorInvalidValue;
        switch (prec * 8 + depth) {
            case 2: e = tc_t_launch<0, 2>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 3: e = tc_t_launch<0, 3>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 4: e = tc_t_launch<0, 4>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 6: e = tc_t_launch<0, 6>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 10: e = tc_t_launch<1, 2>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 11: e = tc_t_launch<1, 3>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 12: e = tc_t_launch<1, 4>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            case 14: e = tc_t_launch<1, 6>(grid, smem, st, map, W, N, kdim, rows, out, rpc, n_out, ma); break;
            default: break;
        }
        LDDMM_CUDA(e);
    }
    return LDDMM_OK;
}

// Self-test of the bounded waits: one thread waits, through the same routine as the
// tensor-core kernel, on an mbarrier phase that nothing completes; when the bound runs out it
// records LDDMM_ETIMEOUT in the device error word as a production kernel would, and returns.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool done = mbar_wait(&bar, 0, limit_ns);
    if (!done) atomicExch(&g_tc_error, LDDMM_ETIMEOUT);
    *status = done ? LDDMM_OK : LDDMM_ETIMEOUT;
}

int wait_selftest(double seconds, int* status) {
    if (!status || !(seconds > 0.0) || seconds > 1.0) {
        set_error("selftest_wait: need status != NULL and 0 < seconds <= 1");
        return LDDMM_EINVAL;
    }
    int* d = nullptr;
    LDDMM_CUDA(cudaMalloc(&d, sizeof(int)));
    k_wait_selftest<<<1, 32>>>((unsigned long long)(seconds * 1e9), d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(status, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_error(std::string("selftest_wait: ") + cudaGetErrorString(e));
        return LDDMM_ECUDA;
    }
    return LDDMM_OK;
}

// Reads and clears the device error word of the tensor-core kernels.
int tc_take_error(int* code) {
    int zero = 0;
    LDDMM_CUDA(cudaMemcpyFromSymbol(code, g_tc_error, sizeof(int)));
    LDDMM_CUDA(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int)));
    return LDDMM_OK;
}

}  // namespace lddmm
