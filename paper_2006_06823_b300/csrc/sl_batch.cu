// Persistent batched SL transport: the state sweep D_t m = 0 (Table 1 row 1; Sec. 3.1,
// Eqs. 40-43) of many independent image pairs of different grid sizes in ONE cooperative
// launch. Every block takes tiles (32 x 8 voxels in x, y, four consecutive z planes per thread)
// from one work list that spans all active pairs; the characteristics (trilinear, RK2) are
// computed for every pair first, then
// the nt gather steps follow, separated by a grid-wide barrier (step j + 1 reads what step j
// wrote, anywhere in the same pair's grid).
//
// The barrier is a counter + generation word in device memory. Its wait is bounded by
// %globaltimer: a block that does not see the generation advance within the bound records
// LDDMM_ETIMEOUT in the status word and leaves the kernel, as every other block then does at
// the same barrier, so a missing block can stall the launch for the bound at most. A
// cooperative launch guarantees that all blocks are resident, so in normal operation the
// barrier always completes; the self-test form asks for one arrival more than the grid has,
// which nothing supplies.
//
// The arithmetic per voxel is that of the single-pair kernels (k_sl_char / k_sl_gather with
// trilinear interpolation), so each pair's result equals lddmm_sl_transport's bit for bit.
#include "common.cuh"
#include "lddmm.h"

#include <algorithm>
#include <string>
#include <vector>

namespace lddmm {
namespace {

constexpr int kBatchMaxPairs = 256;
constexpr int kTile = 256;   // threads per block: 32 x 8 (x, y), each over kZt consecutive z planes
constexpr int kTx = 32, kTy = 8, kZt = 4;

struct BatchPair {
    int nx, ny, nz;
    int active;
    int tx, txy;             // tiles along x, and per z block (tx * ty)
    long tile0;              // first tile of this pair in the work list
    const float* vel;        // 3 planes, voxels per unit time
    const float* field;
    float* out;
    float* tmp;              // ping-pong partner of out
    float* D;                // departure offsets, 3 planes
};

struct BatchTable {
    BatchPair p[kBatchMaxPairs];
};

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ float clampD(float d) { return fminf(fmaxf(d, -1048576.f), 1048576.f); }

__device__ __forceinline__ int wrapi(int i, int n) {
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
}

template <bool RO>
__device__ __forceinline__ float tap(const float* p) {
    // RO: data no block writes during the launch (read-only path); else a coherent load, since
    // the field was written by other blocks before the last barrier
    return RO ? __ldg(p) : __ldca(p);
}

// trilinear interpolation of f at (x, y, z) + (dx, dy, dz), periodic (the single-pair
// kernels' cell and weights)
template <bool RO>
__device__ __forceinline__ float lin_at(const float* f, int nx, int ny, int nz, int x,
                                        int y, int z, float dx, float dy, float dz) {
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
    const float v000 = tap<RO>(f + z0 + y0 + x0), v001 = tap<RO>(f + z0 + y0 + x1);
    const float v010 = tap<RO>(f + z0 + y1 + x0), v011 = tap<RO>(f + z0 + y1 + x1);
    const float v100 = tap<RO>(f + z1 + y0 + x0), v101 = tap<RO>(f + z1 + y0 + x1);
    const float v110 = tap<RO>(f + z1 + y1 + x0), v111 = tap<RO>(f + z1 + y1 + x1);
    const float a00 = fmaf(tx, v001 - v000, v000), a01 = fmaf(tx, v011 - v010, v010);
    const float a10 = fmaf(tx, v101 - v100, v100), a11 = fmaf(tx, v111 - v110, v110);
    const float b0 = fmaf(ty, a01 - a00, a00), b1 = fmaf(ty, a11 - a10, a10);
    return fmaf(tz, b1 - b0, b0);
}

// Grid-wide barrier with a bounded wait. bar[0] counts arrivals, bar[1] is the generation.
// Returns false (and records ETIMEOUT) if the generation does not advance within limit_ns.
__device__ bool grid_barrier(unsigned* bar, unsigned expected, unsigned long long limit_ns,
                             int* status) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = now_ns();
            for (unsigned it = 0;; ++it) {
                if (*gen != g0) break;
                if ((it & 63u) == 63u && now_ns() - t0 > limit_ns) {
                    ok = 0;
                    atomicExch(status, LDDMM_ETIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// pair of work-list tile t (binary search over the pairs' first tiles)
__device__ __forceinline__ int pair_of(const BatchTable& tb, int npairs, long t) {
    int lo = 0, hi = npairs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb.p[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// tile t of pair P: this thread's (x, y) and first z plane; false if outside the grid
__device__ __forceinline__ bool tile_voxel(const BatchPair& P, long t, int& x, int& y, int& z, int& zend) {
    const int tl = (int)(t - P.tile0);
    const int bz = tl / P.txy, r = tl - bz * P.txy;
    const int by = r / P.tx, bx = r - by * P.tx;
    x = bx * kTx + (int)(threadIdx.x & (kTx - 1));
    y = by * kTy + (int)(threadIdx.x / kTx);
    z = bz * kZt;
    zend = min(z + kZt, P.nz);
    return x < P.nx && y < P.ny && z < zend;
}

__global__ void __launch_bounds__(kTile, 5)
k_sl_transport_batch(const __grid_constant__ BatchTable tb, int npairs, long ntiles, int nt,
                     float dts, unsigned* bar, unsigned extra_arrivals,
                     unsigned long long limit_ns, int* status) {
    const unsigned expected = gridDim.x + extra_arrivals;
    const float h = 0.5f * dts;
    // ---- characteristics: D = dt/2 (v(X*) + v(x)), X* = x + dts v(x)  (dts = -dt forward)
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchPair& P = tb.p[pair_of(tb, npairs, t)];
        int x, y, z, zend;
        if (!P.active || !tile_voxel(P, t, x, y, z, zend)) continue;
        const int n = P.nx * P.ny * P.nz, plane = P.nx * P.ny;
        for (int i = (z * P.ny + y) * P.nx + x; z < zend; ++z, i += plane) {
            const float V0 = __ldcs(P.vel + i), V1 = __ldcs(P.vel + n + i), V2 = __ldcs(P.vel + 2 * n + i);
            const float W0 = lin_at<true>(P.vel, P.nx, P.ny, P.nz, x, y, z, dts * V0, dts * V1, dts * V2);
            const float W1 = lin_at<true>(P.vel + n, P.nx, P.ny, P.nz, x, y, z, dts * V0, dts * V1, dts * V2);
            const float W2 = lin_at<true>(P.vel + 2 * n, P.nx, P.ny, P.nz, x, y, z, dts * V0, dts * V1, dts * V2);
            P.D[i] = h * (W0 + V0);
            P.D[n + i] = h * (W1 + V1);
            P.D[2 * n + i] = h * (W2 + V2);
        }
    }
    // ---- nt steps m^{j+1} = m^j o X, ping-pong so that the last one lands in out; the offsets
    // of plane z + 1 are loaded while the taps of plane z are in flight
    for (int j = 0; j < nt; ++j) {
        if (!grid_barrier(bar, expected, limit_ns, status)) return;
        const bool to_out = ((nt - 1 - j) % 2) == 0;
        for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const BatchPair& P = tb.p[pair_of(tb, npairs, t)];
            int x, y, z, zend;
            if (!P.active || !tile_voxel(P, t, x, y, z, zend)) continue;
            const int n = P.nx * P.ny * P.nz, plane = P.nx * P.ny;
            const float* src = j == 0 ? P.field : (to_out ? P.tmp : P.out);
            float* dst = to_out ? P.out : P.tmp;
            int i = (z * P.ny + y) * P.nx + x;
            float d0 = __ldcs(P.D + i), d1 = __ldcs(P.D + n + i), d2 = __ldcs(P.D + 2 * n + i);
            for (;;) {
                const bool more = z + 1 < zend;
                const int ip = more ? i + plane : i;
                const float e0 = __ldcs(P.D + ip), e1 = __ldcs(P.D + n + ip), e2 = __ldcs(P.D + 2 * n + ip);
                const float v = j == 0 ? lin_at<true>(src, P.nx, P.ny, P.nz, x, y, z, d0, d1, d2)
                                       : lin_at<false>(src, P.nx, P.ny, P.nz, x, y, z, d0, d1, d2);
                __stcs(dst + i, v);
                if (!more) break;
                ++z;
                i = ip;
                d0 = e0; d1 = e1; d2 = e2;
            }
        }
    }
}

}  // namespace
}  // namespace lddmm

using namespace lddmm;

extern "C" int lddmm_sl_transport_batch(int n, const int* dims, int nt, int direction,
                                        const float* const* vel, const float* const* field,
                                        float* const* out, const int* active,
                                        double wait_seconds, void* stream) {
    if (n < 0 || n > kBatchMaxPairs) {
        set_error("sl_transport_batch: need 0 <= n <= " + std::to_string(kBatchMaxPairs));
        return LDDMM_EINVAL;
    }
    if (n == 0) return LDDMM_OK;
    if (!dims || !vel || !field || !out) {
        set_error("sl_transport_batch: NULL array");
        return LDDMM_EINVAL;
    }
    if (nt < 1) { set_error("sl_transport_batch: nt must be >= 1"); return LDDMM_EINVAL; }
    if (direction != 1 && direction != -1) {
        set_error("sl_transport_batch: direction must be +1 or -1");
        return LDDMM_EINVAL;
    }
    if (wait_seconds > 10.0) {
        set_error("sl_transport_batch: wait bound above 10 s");
        return LDDMM_EINVAL;
    }
    BatchTable tb{};
    long ntiles = 0, scratch = 0;
    for (int p = 0; p < n; ++p) {
        const int nx = dims[3 * p], ny = dims[3 * p + 1], nz = dims[3 * p + 2];
        int rc = check_grid(nx, ny, nz);
        if (rc) return rc;
        if (!vel[p] || !field[p] || !out[p]) {
            set_error("sl_transport_batch: NULL pointer of pair " + std::to_string(p));
            return LDDMM_EINVAL;
        }
        if (field[p] == out[p]) {
            set_error("sl_transport_batch: field and out of pair " + std::to_string(p) +
                      " must not be the same buffer");
            return LDDMM_EINVAL;
        }
        const long nv = (long)nx * ny * nz;
        BatchPair& P = tb.p[p];
        P.nx = nx;
        P.ny = ny;
        P.nz = nz;
        P.active = 1;
        P.tx = (nx + kTx - 1) / kTx;
        P.txy = P.tx * ((ny + kTy - 1) / kTy);
        P.tile0 = ntiles;
        P.vel = vel[p];
        P.field = field[p];
        P.out = out[p];
        ntiles += (long)P.txy * ((nz + kZt - 1) / kZt);
        scratch += 4 * nv;   // D (3 planes) + the ping-pong field
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // scratch: D and tmp per pair, and the barrier and status words, from the stream-ordered pool
    float* buf = nullptr;
    unsigned* bar = nullptr;
    LDDMM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), scratch * sizeof(float) + 256, st));
    struct Free {
        void* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } guard{buf, st};
    bar = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(buf) + scratch * sizeof(float));
    int* status = reinterpret_cast<int*>(bar + 2);
    LDDMM_CUDA(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
    {
        float* q = buf;
        for (int p = 0; p < n; ++p) {
            const long nv = (long)tb.p[p].nx * tb.p[p].ny * tb.p[p].nz;
            tb.p[p].D = q;
            tb.p[p].tmp = q + 3 * nv;
            q += 4 * nv;
        }
    }
    if (active) {
        // the caller's device mask, read once here (it selects the work list on the host side)
        std::vector<int> a(n);
        LDDMM_CUDA(cudaMemcpyAsync(a.data(), active, n * sizeof(int), cudaMemcpyDeviceToHost, st));
        LDDMM_CUDA(cudaStreamSynchronize(st));
        for (int p = 0; p < n; ++p) tb.p[p].active = a[p] != 0;
    }
    long active_voxels = 0;
    for (int p = 0; p < n; ++p)
        if (tb.p[p].active) active_voxels += (long)tb.p[p].nx * tb.p[p].ny * tb.p[p].nz;
    // self-test form: a negative bound asks for one arrival more than the grid supplies
    const unsigned extra = wait_seconds < 0 ? 1u : 0u;
    const double secs = wait_seconds < 0 ? -wait_seconds : (wait_seconds > 0 ? wait_seconds : 1.0);
    const unsigned long long limit_ns = (unsigned long long)(secs * 1e9);
    int dev = 0, nsm = 0, per_sm = 0;
    LDDMM_CUDA(cudaGetDevice(&dev));
    LDDMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    LDDMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sl_transport_batch, kTile, 0));
    const long grid = std::max(1L, std::min<long>(ntiles, (long)std::max(per_sm, 1) * nsm));
    const double dt = 1.0 / nt;
    float dts = (float)(direction > 0 ? -dt : dt);
    int npairs = n;
    int nt_ = nt;
    void* args[] = {&tb, &npairs, &ntiles, &nt_, &dts, &bar, const_cast<unsigned*>(&extra),
                    const_cast<unsigned long long*>(&limit_ns), &status};
    {
        // algorithmic bytes: characteristics 36 B and each step 20 B per voxel of the active
        // pairs (the single-pair kernels' counts)
        KTRACE("sl_transport_batch", st, (36.0 + 20.0 * nt) * (double)active_voxels, 0);
        LDDMM_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_sl_transport_batch),
                                               dim3((unsigned)grid), dim3(kTile), args, 0, st));
    }
    int hstatus = 0;
    LDDMM_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LDDMM_CUDA(cudaStreamSynchronize(st));
    if (hstatus != 0) {
        set_error("sl_transport_batch: grid barrier wait ran out (" + std::to_string(secs) + " s)");
        return hstatus;
    }
    return LDDMM_OK;
}
