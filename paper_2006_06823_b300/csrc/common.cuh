// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "lddmm.h"

namespace lddmm {

// Records `msg` as the calling thread's last error (read through lddmm_last_error()).
void set_error(const std::string& msg);

#define LDDMM_CUDA(expr)                                                              \
    do {                                                                              \
        cudaError_t e__ = (expr);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            ::lddmm::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__)); \
            return LDDMM_ECUDA;                                                       \
        }                                                                             \
    } while (0)

#define LDDMM_CHECK_LAUNCH() LDDMM_CUDA(cudaGetLastError())

// Scope around one kernel launch: counts it and, when tracing is on, brackets it with CUDA
// events on `st`, recording the launch's algorithmic bytes and flops.
class KTrace {
  public:
    KTrace(const char* name, cudaStream_t st, double bytes, double flops = 0.0);
    ~KTrace();
    KTrace(const KTrace&) = delete;
    KTrace& operator=(const KTrace&) = delete;

  private:
    const char* name_;
    cudaStream_t st_;
    double bytes_, flops_;
    void* a_;
};
// Graph capture bookkeeping: launches made while capturing are counted into the graph and
// added to the process count each time the graph is launched.
void capture_begin();
long capture_end();
void count_launches(long n);
bool tracing();

#define KTRACE(name, st, bytes, flops) ::lddmm::KTrace ktrace__(name, st, (double)(bytes), (double)(flops))

struct Grid {
    int nx, ny, nz;
    __host__ __device__ long ntot() const { return (long)nx * ny * nz; }
};

constexpr int kMaxIotaYBlocks = 8;   // 2 ny / 256 rounded up, ny <= 1024

// Twiddle tables [K][n] per axis: cos/sin(2 pi k j / n) for k = slot - K/2, FP64-evaluated,
// stored FP32. All six tables sit in one allocation of table_floats(grid, K) floats.
struct Twiddles {
    int K;
    const float *cx, *sx, *cy, *sy, *cz, *sz;
    // x-stage matrices for the tensor-core path: W_pi[n][jx] (n = 2kx + re/im, K x nx) and
    // W_io[x][j] (nx x K, weights 1 for kx = 0 and 2 otherwise)
    const float *wpi, *wio;
    // the same two matrices as tensor-core operand images (hi | lo, swizzled), 16-B aligned:
    // [0] TF32 split, [1] BF16 split
    const unsigned char *wpi_img[2], *wio_img[2];
    // Y/Z-stage contraction matrices, complex [q][p] (p fastest): mpy[y][jy] = e^{-i ky y},
    // miy[jy][y] = e^{+i ky y} (0 for jy = 0), mpz[z][jz] = e^{-i kz z}
    const float2 *mpy, *miy, *mpz;
    // Y stages on the tensor cores (tc_y): real W matrices with (cos, sin) row pairs as operand
    // images per precision form: pi, W[2 jy + {0, 1}][y] = {cos, sin}(ky y 2pi/ny) (N = 2K,
    // kdim = ny); iota in iy_blocks blocks of iy_nyb positions, W[2 y + {0, 1}][jy] = the same
    // (0 for jy = 0; N = 2 iy_nyb, kdim = K)
    bool tc_y;
    int iy_blocks, iy_nyb;
    const unsigned char *wpy_img[2], *wiy_img[2][kMaxIotaYBlocks];
};
long twiddle_floats(const Grid& g, int K);
// Fills `mem` (twiddle_floats floats, device) and points `tw` into it.
int twiddle_init(const Grid& g, int K, float* mem, Twiddles& tw, cudaStream_t st);

// Argument checks of the stand-alone spectral operators (capi.cu), shared by every entry
// point that runs bl_project / bl_include so that all accept the same grids, bands and
// precision forms. Each returns LDDMM_OK or LDDMM_EINVAL with the message set.
int check_grid(int nx, int ny, int nz);
int check_band(int nx, int ny, int nz, int K);
int check_spectral_precision(int precision);

// float2 elements of each of the two scratch buffers that bl_project / bl_include need
// for `ncomp` components.
long spectral_scratch_elems(const Grid& g, int K, int ncomp);

// Tensor-core row GEMM OUT[row][n] = sum_k IN[row][k] W[n][k] (tc_rowgemm.cu). epi selects
// the store: 0 row-major OUT[comp][row in comp][n] (rpc rows per component, component stride
// comp_stride); 1 transposed per slab of rpc rows, OUT[slab][n][row in slab]; 2 / 3 complex
// completion of a real-GEMM complex contraction (rows: (Re, Im) pairs of `lines` complex lines
// per slab of rpc = 2 lines rows; W rows: (cos, sin) pairs), writing interleaved complex
// OUT[slab][p0 + p][line] (ptot positions per slab) with e^{-i} (2) or e^{+i} (3) phases.
// prec < 0 in the support test asks for both precision forms.
bool tc_rowgemm_supported(int N, int kdim, long rows, const void* in, long in_row_floats,
                          int epi = 0, int prec = -1, int nblk = 1);
int tc_rowgemm(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
               int N, int prec, float* out, long rpc, long comp_stride, int n_out,
               const char* trace_name, double trace_bytes, cudaStream_t st);
// nblk > 1 (complex completion forms only): W holds nblk consecutive operand images of N
// rows each, block b covering positions p0 + b N / 2 ...; the work items are (row tile, block)
// pairs in one launch.
int tc_rowgemm_ex(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
                  int N, int prec, int epi, float* out, long rpc, long comp_stride, int n_out,
                  int ptot, int p0, int lines, int nblk, const char* trace_name,
                  double trace_bytes, cudaStream_t st);
// Transposed tensor-core form for narrow outputs (16 <= N <= 64, N % 16 == 0; the x stage of
// pi): the same OUT as tc_rowgemm_ex with epi = 1 (OUT[slab][n][row in slab], slabs of rpc
// rows), from the same W operand image, with W as the MMA's A operand and 128 input rows per
// instruction (tc_rowgemm.cu).
bool tc_rowgemm_t_supported(int N, int kdim, long rows, const void* in, long in_row_floats);
int tc_rowgemm_t(const float* in, long rows, int kdim, long in_row_floats, const unsigned char* W,
                 int N, int prec, float* out, long rpc, int n_out, const char* trace_name,
                 double trace_bytes, cudaStream_t st);
long tc_wimage_bytes(int N, int kdim);
int tc_build_wimage(const float* W, int N, int kdim, int prec, unsigned char* img,
                    cudaStream_t st);
int tc_take_error(int* code);
// Bounded-wait self-test (a wait nothing completes, limited to `seconds`): *status =
// LDDMM_ETIMEOUT, and the device error word records it. Synchronous.
int wait_selftest(double seconds, int* status);

// pi: ncomp fields (component stride fstride floats) -> ncomp cubes (stride K^3 float2).
int bl_project(const Grid& g, const Twiddles& tw, const float* f, long fstride, int ncomp,
               float2* c, float2* s1, float2* s2, int precision, cudaStream_t st);

// iota: ncomp cubes -> ncomp fields (component stride fstride). deriv_axis -1 none,
// 0..2 spectral derivative, 3 divergence of a 3-component cube (writes one field).
int bl_include(const Grid& g, const Twiddles& tw, const float2* c, int ncomp, float* f,
               long fstride, int deriv_axis, int bspline, float2* s1, float2* s2,
               int precision, cudaStream_t st);

// ---------------------------------------------------------------- K^3 cube kernels
// out = a*x + b*y over n complex values (x or y may be null => treated as zero).
int cube_axpby(float2* out, float a, const float2* x, float b, const float2* y, long n,
               cudaStream_t st);
// out = wL * L~ x + a * y  (y may be null); mode 1: L~, mode -1: L~^{-1} (y ignored).
int cube_apply_L(float2* out, const float2* x, float wL, float a, const float2* y, int K,
                 int ncomp, double alpha, int s, int mode, cudaStream_t st);
// Hermitian symmetrisation of ncomp cubes in place: c <- (c + conj c_{-k}) / 2, slot-0
// planes zeroed.
int cube_hermitian(float2* c, int K, int ncomp, cudaStream_t st);
// Two-level preconditioner on band-limited cubes: R (the coarse band S_c of edge Kc, slot 0
// zero) and z <- E y on S_c, theta z on the other modes.
int cube_restrict(const float2* fine, int K, float2* coarse, int Kc, int ncomp, cudaStream_t st);
int cube_two_level(float2* z, int K, const float2* y, int Kc, float theta, int ncomp, cudaStream_t st);

// FP64 reductions into device doubles (deterministic two-pass).
int dot_f2(const float2* a, const float2* b, long n, double* partials, double* out,
           cudaStream_t st);
int max_abs_f2(const float2* a, long n, double* partials, double* out, cudaStream_t st);
// max over voxels of the length of the 3-plane field u scaled per component by s (FP64)
int max_norm3(const float* u, long n, const float s[3], double* partials, double* out, cudaStream_t st);
// sum_j w_j <a_j, b_j> over `nodes` blocks of npn elements, w_j trapezoid weights of step dt
// (nodes == 1: plain dot)
int dot_f2_nodes(const float2* a, const float2* b, long npn, int nodes, double dt,
                 double* partials, double* out, cudaStream_t st);
constexpr int kReduceBlocks = 296;  // 2 x 148 SMs

// ---------------------------------------------------------------- tensor-core convolutions
// 3x3x3 convolutions of the warm-start network on tcgen05 (tc_conv.cu). W: stored weights
// [cout][cin * 27] (the forward weights, or the transposed tap-flipped ones for the input
// gradient), BF16 or FP32; TI / TO: the stored activation type or FP32 (gradients, output).
bool tc_conv_supported(int cout, int D, bool wgrad);
template <typename TI, typename TW, typename TO>
int tc_conv(const TI* in, int cin, int D, long in_bstride, const TW* W, const float* bias,
            int cout, TO* out, long out_bstride, int out_coff, bool relu, int B, cudaStream_t st);
// dW[co][ci * 27 + t] += sum over the B samples of dout[b][co][v] in[b][ci][v + o(t)]
template <typename TA>
int tc_conv_wgrad(const float* dout, int cout, long dout_bstride, const TA* in, int cin,
                  long in_bstride, int D, int B, float* dW, cudaStream_t st);
int tc_conv_take_error(int* code);

// ---------------------------------------------------------------- spatial form (spatial.cu)
// Full-grid FFT plans and buffers of one context (cuFFT R2C / C2R on its stream).
struct SpatialFFT;
int spatial_fft_create(const Grid& g, cudaStream_t st, SpatialFFT** out);
void spatial_fft_destroy(SpatialFFT* f);
// out_c = wL L x_c + a y_c (mode 1; y may be null) or L^{-1} x_c (mode -1), ncomp fields of
// ntot floats; L = (Id - alpha Laplacian)^s on [0, 2 pi)^3. out may alias x.
int spatial_apply_L(SpatialFFT* f, float* out, const float* x, float wL, float a, const float* y,
                    int ncomp, double alpha, int s, int mode, cudaStream_t st);
// spectral d/dx_axis of ncomp fields (component c to out + c fstride), axis 0..2; axis 3:
// divergence of three fields into one. The Nyquist wavenumber of a derivative axis is zero.
int spatial_deriv(SpatialFFT* f, const float* in, int ncomp, int axis, float* out, long fstride,
                  cudaStream_t st);
// max |a_i| over n floats
int max_abs_f32(const float* a, long n, double* partials, double* out, cudaStream_t st);
// Spectral restriction of nimg periodic images from grid gf to the half grid gc (gc = gf / 2 per
// axis): Fourier modes with 2|k_a| < gc_a kept, synthesised on gc (full-grid cuFFT plans made
// and released inside the call; synchronises the stream).
int spectral_restrict_half(const Grid& gf, const float* const* in, const Grid& gc, float* const* out,
                           int nimg, cudaStream_t st);

// ---------------------------------------------------------------- SL kernels (sl.cu)
struct SLArgs {
    Grid g;
    int interp;      // 1 or 3
    int bx = 32;     // block shape of the one-voxel-per-thread kernels (bx * by = 256)
    int by = 8;
    int zt = 0;      // z planes per thread of the pipelined trilinear kernels (0: by grid size)
};
// D = offsets of departure points; vsrc = samples (linear) or spline coefficients (cubic)
// of the velocity, vval its samples; scale[a] converts component a to voxels.
int sl_characteristics(const SLArgs& a, const float* vsrc, const float* vval,
                       const float scale[3], double dt_signed, float* D, cudaStream_t st);
// out[c] = src[c] o (x + D), ncomp components of stride g.ntot().
int sl_gather(const SLArgs& a, const float* src, const float* D, int ncomp, float* out,
              cudaStream_t st);
// out[c] = src[c] o (x + D) * gam(x)
int sl_gather_scale(const SLArgs& a, const float* src, const float* D, const float* gam,
                    int ncomp, float* out, cudaStream_t st);
// out[c] = src[c] o (x + D) + add[c](x)
int sl_gather_add(const SLArgs& a, const float* src, const float* D, const float* add,
                  int ncomp, float* out, cudaStream_t st);
// gam = 1 + dt/2 (d(X+) + (1 + dt d(X+)) d(x)),  W = dt/2 (v(X) + v(x))
int sl_prep_adjoint(const SLArgs& a, const float* dsrc, const float* dval, const float* Dp,
                    double dt, float* gam, cudaStream_t st);
int sl_prep_source(const SLArgs& a, const float* vsrc, const float* vval, const float* D,
                   double dt, float* W, cudaStream_t st);
// m1 = I0 o (x - u1*to_vox), G = grad(I0 interpolant) there (physical units),
// rho = -(2/sigma2) (m1 - I1) G, partial sums of (m1 - I1)^2 (kReduceBlocks doubles).
int sl_warp_image(const SLArgs& a, const float* I0src, const float* u1, const float to_vox[3],
                  const float* I1, double sigma2, float* m1, float* G, float* rho,
                  double* partials, cudaStream_t st);
// incremental deformation state step: Fnew_a = dv_a - sum_b Du[a*3+b] dv_b;
// out = U o X + dt/2 (Fold o X + Fnew)
// Du: the 9 Jacobian planes of one node, FP32 or (du_bf16) BF16
int sl_inc_defstate(const SLArgs& a, const float* U, const float* D, const float* Fold,
                    const void* Du, bool du_bf16, const float* dv, double dt, float* out,
                    float* Fnew, cudaStream_t st);
// Fnew_a = dv_a - sum_b Du[a*3+b] dv_b (the first node)
int defstate_rhs(const Grid& g, const void* Du, bool du_bf16, const float* dv, float* F,
                 cudaStream_t st);
// out = mul * src o (x - U to_vox) (mul may be null; U: 3 physical planes)
int sl_compose(const SLArgs& a, const float* src, const float* U, const float to_vox[3],
               const float* mul, float* out, cudaStream_t st);
// dlambda(1) = -(2/sigma2) dm1 with dm1 = -G . du1
int state_dlam1(const Grid& g, const float* G, const float* du1, double sigma2, float* out,
                cudaStream_t st);
// drho = -(2/sigma2) dm1 G with dm1 = -G . du1
int defstate_drho1(const Grid& g, const float* G, const float* du1, double sigma2, float* drho,
                   cudaStream_t st);
// acc_b (+)= w sum_a Du[a*3+b] R_a   (init != 0 overwrites)
int accum_JT(const Grid& g, const void* Du, bool du_bf16, const float* R, float w, float* acc,
             int init, cudaStream_t st);
// acc_b = sum_{j=nt..0} w_j sum_a Du_j[a*3+b] R_j[a] in one pass over nt + 1 nodes (R_j at
// R + 3 n j; Du_j at node stride 9 n floats or jac_bf16_stride(n) BF16 elements; w_j = w_end
// at j = 0 and nt, w_mid between): the same bits as accum_JT node by node from j = nt down
int accum_JT_nodes(const Grid& g, const void* Du, bool du_bf16, const float* R, int nt,
                   float w_end, float w_mid, float* acc, cudaStream_t st);
// J = det(I - Du) per voxel (J may be NULL) and kReduceBlocks per-block minima / maxima
int jacobian_det(const Grid& g, const float* Du, float* J, double* pmin, double* pmax, cudaStream_t st);
// Jacobian planes in the packed BF16 form the Hessian kernels read: per node, the 8 entries
// Du[0..7] of each voxel as one 16-byte word ([n] words), then the plane of Du[8]; node stride
// jac_bf16_stride(n) BF16 elements (16-byte aligned); round to nearest even
long jac_bf16_stride(long n);
int pack_jac_bf16(const float* in, void* out, long n, int nodes, cudaStream_t st);
// out[i] = v, i < n
int fill_field(float* out, float v, long n, cudaStream_t st);
// x_out = a * x (n floats)
int scale_field(float* out, const float* in, float a, long n, cudaStream_t st);
// partial sums over (a - b)^2 into kReduceBlocks doubles, then final into out
int sum_sq_diff(const float* a, const float* b, long n, double* partials, double* out,
                cudaStream_t st);
int finalize_sum(const double* partials, int n, double* out, cudaStream_t st);
// periodic cubic B-spline coefficients of ncomp fields (out may alias in)
int bspline_prefilter(const Grid& g, const float* in, int ncomp, float* out, cudaStream_t st);
// image variant: incremental state step, its first right-hand side, accumulation, lambda(1)
int sl_inc_image(const SLArgs& a, const float* U, const float* D, const float* Fold,
                 const float* Gm, const float* dv, double dt, float* out, float* Fnew,
                 cudaStream_t st);
int image_rhs(const Grid& g, const float* Gm, const float* dv, float* F, cudaStream_t st);
int accum_sv(const Grid& g, const float* s, const float* Gm, float w, float* acc, int init,
             cudaStream_t st);
// acc_b = sum_{j=nt..0} w_j s_j Gm_{j,b} in one pass over nt + 1 nodes (s_j at S + n j, Gm_j at
// Gm + 3 n j; w_j = w_end at j = 0 and nt, w_mid between): the same bits as accum_sv node by
// node from j = nt down
int accum_sv_nodes(const Grid& g, const float* S, const float* Gm, int nt, float w_end, float w_mid,
                   float* acc, cudaStream_t st);
int scaled_diff(const Grid& g, const float* a, const float* b, float coef, float* out,
                cudaStream_t st);

}  // namespace lddmm
