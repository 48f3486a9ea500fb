// C ABI of the library: contexts, the Gauss-Newton-Krylov driver and the stand-alone
// operators. The driver follows Sec. 2.2 (Eqs. 13-14): v~ <- v~ + eps dv~, dv~ from PCG on
// H dv~ = -g~ with preconditioner L~^{-1}; the gradient and Hessian-vector products of the
// image-transport variant (Sec. 2.3.1) and the deformation-state variant (Sec. 2.3.3) are
// assembled from the SL-RK sweeps of Table 1.
//
// Readings fixed here (the cited stopping rules are not written out in the paper):
// PCG from zero with forcing eta = min(0.5, sqrt(||g||/||g_ref||)); Armijo backtracking
// from eps = 1 (halving, at most 10 times, constant 1e-4); stop on ||g||/||g_ref|| <= gtol
// with g_ref the gradient at v~ = 0; time integrals by the trapezoid rule on the nt + 1
// nodes. FP64 holds every inner product, energy, comparison and the stopping test.
#include "common.cuh"
#include "lddmm.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace lddmm {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace lddmm

using namespace lddmm;

#define TRY(expr)                      \
    do {                               \
        int rc__ = (expr);             \
        if (rc__ != LDDMM_OK) return rc__; \
    } while (0)

struct lddmm_ctx {
    lddmm_params p;
    Grid g;
    long n = 0;       // voxels
    long kc = 0;      // K^3
    int K = 0;
    cudaStream_t st = nullptr;
    double dt = 0;
    float to_vox[3];
    int sticky = LDDMM_OK;
    std::vector<void*> allocs;
    Twiddles tw;
    SLArgs sl;

    // images
    float *I0 = nullptr, *I1 = nullptr, *I0c = nullptr;
    // velocity fields of the current v~: one node (stationary) or nt + 1 nodes (v, vc: 3
    // planes each, d, dc: 1), and one step (stationary) or nt steps of offsets Df, Db,
    // source W (3 planes each) and adjoint factor gam (1)
    float *v = nullptr, *vc = nullptr, *d = nullptr, *dc = nullptr;
    float *Df = nullptr, *Db = nullptr, *gam = nullptr, *W = nullptr;
    // trajectories
    float2* ut = nullptr;   // DEFSTATE, STATE: u~_j, (nt+1) x 3 x K^3
    float* Du = nullptr;    // DEFSTATE, STATE: (nt+1) x 9 planes
    void* Du16 = nullptr;   // the same, LDDMM_PREC_BF16X3_JBF16: BF16 copy read by the Hessian
    float* ms = nullptr;    // IMAGE: m_j, (nt+1) planes
    float* Gm = nullptr;    // IMAGE, STATE: iota(grad~ pi(m_j)), (nt+1) x 3 planes
    float* Wb = nullptr;    // STATE: source of the nu~ step, -dt/2 (v(X+) + v(x)), 3 planes per step
    float* PJ = nullptr;    // STATE: per node iota(nu~_j) (3 planes, physical) and J_j (1 plane)
    float* Rn = nullptr;    // DEFSTATE, stationary: per node iota(rho~_j) of the adjoint sweep, 3 planes
    float* Sn = nullptr;    // IMAGE, STATE, stationary: per node the projected adjoint scalar, 1 plane
    // spatial form: full-grid FFT plans (the "cubes" of this context are fields on the grid)
    SpatialFFT* fft = nullptr;
    float *G = nullptr, *m1 = nullptr;
    // work fields
    float *fa = nullptr, *fb = nullptr, *fc = nullptr, *fd = nullptr, *acc = nullptr,
          *dvsp = nullptr;
    // spectral scratch
    float2 *s1 = nullptr, *s2 = nullptr;
    // cube vectors (3 x K^3 each, x (nt + 1) nodes in a non-stationary context)
    enum { C_V, C_VT, C_G, C_R, C_Z, C_P, C_HP, C_X, C_T0, C_T1, C_T2, C_CUR, C_DV, C_RP, C_NUM };
    float2* cv[C_NUM];
    // reductions
    double* partials = nullptr;
    double* dsc = nullptr;     // device scalars
    double* hsc = nullptr;     // pinned host mirror
    // cache
    bool vel_valid = false;    // velocity fields + state of cv[C_CUR]
    bool traj_valid = false;   // + Jacobians / grad m~ for the Hessian
    bool warp_valid = false;   // DEFSTATE, STATE: m1 and G of the current state
    int solves = 0;
    // CUDA graph of the PCG Hessian-vector product (cv[C_P] -> cv[C_HP])
    bool use_graphs = false;
    bool graph_failed = false;
    int hv_eager_runs = 0;
    cudaGraphExec_t hv_exec = nullptr;
    long hv_graph_launches = 0;
    // two-level preconditioner: the half-grid context of the coarse level (owned) and the cap
    // on its PCG iterations per application (0: the spectral preconditioner L~^{-1} alone)
    lddmm_ctx* coarse = nullptr;
    int tl_inner = 0;
    bool have_images = false;
    // device bytes of the context's own allocations (checked against the workspace limit)
    long long ws_bytes = 0;
    // convergence history of the last registration: per Gauss-Newton iterate {seconds since
    // the call began, ||g||_2 / ||g_ref||_2, E, PCG iterations so far, solves so far}
    std::vector<std::array<double, 5>> hist;
};

// Process-wide cap on the device bytes one context may allocate (0: none).
static std::atomic<long long> g_ws_limit{0};

static int fail(lddmm_ctx* c, int rc) {
    if (c && c->sticky == LDDMM_OK) c->sticky = rc;
    return rc;
}

static int dalloc(lddmm_ctx* c, void** p, size_t bytes) {
    const long long lim = g_ws_limit.load();
    if (lim > 0 && c->ws_bytes + (long long)bytes > lim) {
        set_error("workspace limit: the context needs more than the " + std::to_string(lim) +
                  " bytes allowed (lddmm_set_workspace_limit)");
        *p = nullptr;
        return LDDMM_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        *p = nullptr;
        return LDDMM_ENOMEM;
    }
    c->allocs.push_back(*p);
    c->ws_bytes += (long long)bytes;
    return LDDMM_OK;
}
template <class T>
static int dalloc_t(lddmm_ctx* c, T** p, size_t count) {
    return dalloc(c, reinterpret_cast<void**>(p), count * sizeof(T));
}

static int validate(const lddmm_params* p) {
    if (!p) { set_error("params is NULL"); return LDDMM_EINVAL; }
    if (p->nx < 4 || p->ny < 4 || p->nz < 4 || p->nx > 1024 || p->ny > 1024 || p->nz > 4096) {
        set_error("grid must be 4..1024 (x, y) and 4..4096 (z) voxels per axis");
        return LDDMM_EINVAL;
    }
    if ((long)p->nx * p->ny * p->nz > 0x7fffffffL / 3) {
        set_error("grid too large: nx*ny*nz must stay below 2^31/3 voxels");
        return LDDMM_EINVAL;
    }
    if (p->spatial != 0 && p->spatial != 1) {
        set_error("spatial must be 0 or 1");
        return LDDMM_EINVAL;
    }
    if (p->spatial && (p->nx & 1)) {
        set_error("the spatial form needs an even nx");
        return LDDMM_EINVAL;
    }
    if (!p->spatial &&
        (p->K < 4 || (p->K & 1) || p->K > 64 || p->K > p->nx || p->K > p->ny || p->K > p->nz)) {
        set_error("band K must be even, 4 <= K <= min(64, nx, ny, nz)");
        return LDDMM_EINVAL;
    }
    if (p->nt < 1 || p->nt > 1000) { set_error("nt must be 1..1000"); return LDDMM_EINVAL; }
    if (p->variant != LDDMM_V_IMAGE && p->variant != LDDMM_V_STATE &&
        p->variant != LDDMM_V_DEFSTATE) {
        set_error("variant must be LDDMM_V_IMAGE, LDDMM_V_STATE or LDDMM_V_DEFSTATE");
        return LDDMM_EINVAL;
    }
    if (p->nonstationary != 0 && p->nonstationary != 1) {
        set_error("nonstationary must be 0 or 1");
        return LDDMM_EINVAL;
    }

    if (p->interp != LDDMM_INTERP_LINEAR && p->interp != LDDMM_INTERP_CUBIC) {
        set_error("interp must be LDDMM_INTERP_LINEAR or LDDMM_INTERP_CUBIC");
        return LDDMM_EINVAL;
    }
    if (!(p->sigma2 > 0) || !(p->alpha >= 0) || p->s < 0 || p->s > 8) {
        set_error("need sigma2 > 0, alpha >= 0, 0 <= s <= 8");
        return LDDMM_EINVAL;
    }
    if (p->max_gn < 0 || p->max_pcg < 1 || !(p->gtol >= 0)) {
        set_error("need max_gn >= 0, max_pcg >= 1, gtol >= 0");
        return LDDMM_EINVAL;
    }
    if (p->precision != LDDMM_PREC_FP32 && p->precision != LDDMM_PREC_BF16X3 &&
        p->precision != LDDMM_PREC_FP32_SIMT && p->precision != LDDMM_PREC_BF16X3_JBF16) {
        set_error("precision must be LDDMM_PREC_FP32, LDDMM_PREC_BF16X3, LDDMM_PREC_FP32_SIMT or "
                  "LDDMM_PREC_BF16X3_JBF16");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

// ------------------------------------------------------------------ small helpers
// precision of the spectral stages (the JBF16 form uses the BF16 split there)
static int spec_prec(const lddmm_ctx* c) {
    return c->p.precision == LDDMM_PREC_BF16X3_JBF16 ? LDDMM_PREC_BF16X3 : c->p.precision;
}
static bool jac_bf16(const lddmm_ctx* c) { return c->p.precision == LDDMM_PREC_BF16X3_JBF16; }
// Spatial form (Sec. 2.1 with SL in Omega): velocity-shaped vectors are fields on the grid,
// pi and iota are the identity, derivatives and L go through full-grid FFTs.
static bool spatial(const lddmm_ctx* c) { return c->p.spatial != 0; }
// factor of the device dot products: l2 over cube coefficients (band-limited) or the voxel
// mean (spatial)
static double dscale(const lddmm_ctx* c) { return spatial(c) ? 1.0 / (double)c->n : 1.0; }

static int project(lddmm_ctx* c, const float* f, int ncomp, float2* out) {
    if (spatial(c)) {
        if (reinterpret_cast<const void*>(f) != out)
            LDDMM_CUDA(cudaMemcpyAsync(out, f, (size_t)ncomp * c->n * sizeof(float),
                                       cudaMemcpyDeviceToDevice, c->st));
        return LDDMM_OK;
    }
    return bl_project(c->g, c->tw, f, c->n, ncomp, out, c->s1, c->s2, spec_prec(c), c->st);
}
static int include(lddmm_ctx* c, const float2* cube, int ncomp, float* f, long fstride,
                   int deriv, int bspline) {
    if (spatial(c)) {
        const float* src = reinterpret_cast<const float*>(cube);
        const long n = c->n;
        if (deriv < 0 && bspline) {
            if (fstride != n) { set_error("internal: strided spline coefficients"); return LDDMM_EINVAL; }
            return bspline_prefilter(c->g, src, ncomp, f, c->st);
        }
        if (deriv < 0) {
            for (int k = 0; k < ncomp; ++k)
                if (src + k * n != f + k * fstride)
                    LDDMM_CUDA(cudaMemcpyAsync(f + k * fstride, src + k * n, n * sizeof(float),
                                               cudaMemcpyDeviceToDevice, c->st));
            return LDDMM_OK;
        }
        if (deriv == 3) {
            TRY(spatial_deriv(c->fft, src, 3, 3, f, fstride, c->st));
            return bspline ? bspline_prefilter(c->g, f, 1, f, c->st) : LDDMM_OK;
        }
        if (bspline) { set_error("internal: spline coefficients of a derivative"); return LDDMM_EINVAL; }
        return spatial_deriv(c->fft, src, ncomp, deriv, f, fstride, c->st);
    }
    return bl_include(c->g, c->tw, cube, ncomp, f, fstride, deriv, bspline, c->s1, c->s2,
                      spec_prec(c), c->st);
}
// out = wL L~ x + a y (mode 1) or L~^{-1} x (mode -1) over ncube cubes (fields when spatial)
static int op_L(lddmm_ctx* c, float2* out, const float2* x, float wL, float a, const float2* y,
                int ncube, int mode) {
    if (spatial(c))
        return spatial_apply_L(c->fft, reinterpret_cast<float*>(out), reinterpret_cast<const float*>(x),
                               wL, a, reinterpret_cast<const float*>(y), ncube, c->p.alpha, c->p.s, mode,
                               c->st);
    return cube_apply_L(out, x, wL, a, y, c->K, ncube, c->p.alpha, c->p.s, mode, c->st);
}
// max |.| of a velocity-shaped vector of nf2 float2 (complex modulus per coefficient; per value
// when spatial)
static int max_abs(lddmm_ctx* c, const float2* v, long nf2, double* out) {
    if (spatial(c))
        return max_abs_f32(reinterpret_cast<const float*>(v), 2 * nf2, c->partials, out, c->st);
    return max_abs_f2(v, nf2, c->partials, out, c->st);
}

// the Jacobian planes of node j, as the Hessian (hess) or the gradient reads them
static const void* jac(const lddmm_ctx* c, int j, bool hess) {
    if (hess && jac_bf16(c)) return static_cast<const uint16_t*>(c->Du16) + (long)j * jac_bf16_stride(c->n);
    return c->Du + (long)j * 9 * c->n;
}
static bool cubic(const lddmm_ctx* c) { return c->p.interp == LDDMM_INTERP_CUBIC; }
// the forward state is the displacement u~ (phi = id - iota(u~)): DEFSTATE and STATE
static bool has_u(const lddmm_ctx* c) { return c->p.variant != LDDMM_V_IMAGE; }
static bool state_eq(const lddmm_ctx* c) { return c->p.variant == LDDMM_V_STATE; }

// Non-stationary form: nt + 1 velocity nodes and nt distinct steps; the stationary form has
// one node and one step that serve every time.
static bool ns(const lddmm_ctx* c) { return c->p.nonstationary != 0; }
static int nodes(const lddmm_ctx* c) { return ns(c) ? c->p.nt + 1 : 1; }
static long nvec(const lddmm_ctx* c) { return (long)nodes(c) * 3 * c->kc; }   // float2 per velocity
static long node_off(const lddmm_ctx* c, int j, long planes) { return ns(c) ? (long)j * planes * c->n : 0; }
static float* vnode(lddmm_ctx* c, int j) { return c->v + node_off(c, j, 3); }
static float* vcnode(lddmm_ctx* c, int j) { return c->vc + node_off(c, j, 3); }
static float* dnode(lddmm_ctx* c, int j) { return c->d + node_off(c, j, 1); }
static float* dcnode(lddmm_ctx* c, int j) { return c->dc + node_off(c, j, 1); }
static float* Dfstep(lddmm_ctx* c, int j) { return c->Df + node_off(c, j, 3); }
static float* Dbstep(lddmm_ctx* c, int j) { return c->Db + node_off(c, j, 3); }
static float* Wstep(lddmm_ctx* c, int j) { return c->W + node_off(c, j, 3); }
static float* Wbstep(lddmm_ctx* c, int j) { return c->Wb + node_off(c, j, 3); }
static float* gamstep(lddmm_ctx* c, int j) { return c->gam + node_off(c, j, 1); }
// cube j of a velocity-shaped vector (node j; the one cube when stationary)
static const float2* vcube(const lddmm_ctx* c, const float2* vt, int j) {
    return vt + (ns(c) ? (long)j * 3 * c->kc : 0);
}
static float2* vcube(const lddmm_ctx* c, float2* vt, int j) {
    return vt + (ns(c) ? (long)j * 3 * c->kc : 0);
}

// Reads `count` device doubles from c->dsc into c->hsc (synchronises the stream).
static int read_scalars(lddmm_ctx* c, int count) {
    LDDMM_CUDA(cudaMemcpyAsync(c->hsc, c->dsc, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    LDDMM_CUDA(cudaStreamSynchronize(c->st));
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(c->hsc[i])) {
            set_error("non-finite value in an energy or inner product");
            return LDDMM_ENONFINITE;
        }
    return LDDMM_OK;
}

static double trap_w(const lddmm_ctx* c, int j) {
    return (j == 0 || j == c->p.nt) ? 0.5 * c->dt : c->dt;
}

// ------------------------------------------------------------------ velocity (Sec. 3.2)
// v = iota(v~), d = iota(div~ v~), departure offsets forward / backward (Eqs. 40-42, 46),
// the adjoint factor gam and the deformation-state source W.
static int prepare_velocity(lddmm_ctx* c, const float2* vt) {
    const long n = c->n;
    for (int j = 0; j < nodes(c); ++j) {
        const float2* vj = vcube(c, vt, j);
        TRY(include(c, vj, 3, vnode(c, j), n, -1, 0));
        TRY(include(c, vj, 3, dnode(c, j), n, 3, 0));
        if (cubic(c)) {
            TRY(include(c, vj, 3, vcnode(c, j), n, -1, 1));
            TRY(include(c, vj, 3, dcnode(c, j), n, 3, 1));
        }
    }
    // step j runs from node a = j to node b = j + 1 (stationary: both node 0)
    const int steps = ns(c) ? c->p.nt : 1;
    for (int j = 0; j < steps; ++j) {
        const int a = j, b = ns(c) ? j + 1 : j;
        const float* vsrc_a = cubic(c) ? vcnode(c, a) : vnode(c, a);   // interpolated fields
        const float* vsrc_b = cubic(c) ? vcnode(c, b) : vnode(c, b);
        const float* dsrc_b = cubic(c) ? dcnode(c, b) : dnode(c, b);
        // state: X* = x - dt v_b(x), X = x - dt/2 (v_b(x) + v_a(X*))
        TRY(sl_characteristics(c->sl, vsrc_a, vnode(c, b), c->to_vox, -c->dt, Dfstep(c, j), c->st));
        // adjoint: X+* = x + dt v_a(x), X+ = x + dt/2 (v_a(x) + v_b(X+*))
        TRY(sl_characteristics(c->sl, vsrc_b, vnode(c, a), c->to_vox, +c->dt, Dbstep(c, j), c->st));
        // gamma = 1 + dt/2 (d_b(X+) + (1 + dt d_b(X+)) d_a(x))
        TRY(sl_prep_adjoint(c->sl, dsrc_b, dnode(c, a), Dbstep(c, j), c->dt, gamstep(c, j), c->st));
        // W = dt/2 (v_a(X) + v_b(x))
        if (has_u(c))
            TRY(sl_prep_source(c->sl, vsrc_a, vnode(c, b), Dfstep(c, j), c->dt, Wstep(c, j), c->st));
        // STATE: Wb = -dt/2 (v_b(X+) + v_a(x)), the source of the nu~ step
        if (state_eq(c))
            TRY(sl_prep_source(c->sl, vsrc_b, vnode(c, a), Dbstep(c, j), -c->dt, Wbstep(c, j), c->st));
    }
    return LDDMM_OK;
}

// ------------------------------------------------------------------ state equations
// DEFSTATE: D~_t u~ = v~ (Eq. 34): u~_{j+1} = pi(iota(u~_j) o X + W), u~_0 = 0.
static int state_defstate(lddmm_ctx* c) {
    const long kc3 = 3 * c->kc;
    LDDMM_CUDA(cudaMemsetAsync(c->ut, 0, kc3 * sizeof(float2), c->st));
    for (int j = 0; j < c->p.nt; ++j) {
        // iota(u~_0) = 0 (and so are its B-spline coefficients): cleared, not synthesised
        if (j == 0) LDDMM_CUDA(cudaMemsetAsync(c->fa, 0, 3 * c->n * sizeof(float), c->st));
        else TRY(include(c, c->ut + j * kc3, 3, c->fa, c->n, -1, cubic(c)));
        TRY(sl_gather_add(c->sl, c->fa, Dfstep(c, j), Wstep(c, j), 3, c->fb, c->st));
        TRY(project(c, c->fb, 3, c->ut + (j + 1) * kc3));
    }
    c->solves++;
    return LDDMM_OK;
}

// IMAGE: D_t m = 0 (Eq. 17): m_{j+1} = m_j o X, m_0 = I0 (spatial).
static int state_image(lddmm_ctx* c) {
    const long n = c->n;
    LDDMM_CUDA(cudaMemcpyAsync(c->ms, c->I0, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    for (int j = 0; j < c->p.nt; ++j) {
        const float* src = c->ms + j * n;
        if (cubic(c)) {
            TRY(bspline_prefilter(c->g, src, 1, c->fa, c->st));
            src = c->fa;
        }
        TRY(sl_gather(c->sl, src, Dfstep(c, j), 1, c->ms + (j + 1) * n, c->st));
    }
    c->solves++;
    return LDDMM_OK;
}

// E_data = (1/sigma2) mean (m1 - I1)^2 into dsc[0]; DEFSTATE and STATE also form m1, G and
// (optionally) rho(1) = -(2/sigma2) r G into `rho`.
static int data_term(lddmm_ctx* c, float* rho) {
    const long n = c->n;
    if (has_u(c)) {
        TRY(include(c, c->ut + (long)c->p.nt * 3 * c->kc, 3, c->fa, n, -1, 0));
        const float* I0src = cubic(c) ? c->I0c : c->I0;
        TRY(sl_warp_image(c->sl, I0src, c->fa, c->to_vox, c->I1, c->p.sigma2, c->m1, c->G, rho,
                          c->partials, c->st));
        TRY(finalize_sum(c->partials, kReduceBlocks, c->dsc, c->st));
        c->warp_valid = true;
    } else {
        TRY(sum_sq_diff(c->ms + (long)c->p.nt * n, c->I1, n, c->partials, c->dsc, c->st));
    }
    return LDDMM_OK;
}

// E_reg = 1/2 <L~ v~, v~> into dsc[1] (non-stationary: sum_j w_j <L~ v~_j, v~_j>)
static int reg_term(lddmm_ctx* c, const float2* vt) {
    float2* t = c->cv[lddmm_ctx::C_T0];
    TRY(op_L(c, t, vt, 1.f, 0.f, nullptr, 3 * nodes(c), 1));
    TRY(dot_f2_nodes(t, vt, 3 * c->kc, nodes(c), c->dt, c->partials, c->dsc + 1, c->st));
    return LDDMM_OK;
}

// Makes the velocity fields and the state of vt current (copied into cv[C_CUR]).
static int ensure_state(lddmm_ctx* c, const float2* vt, bool known_same) {
    if (known_same && c->vel_valid) return LDDMM_OK;
    float2* cur = c->cv[lddmm_ctx::C_CUR];
    if (vt != cur)
        LDDMM_CUDA(cudaMemcpyAsync(cur, vt, nvec(c) * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
    c->vel_valid = false;
    c->traj_valid = false;
    c->warp_valid = false;
    TRY(prepare_velocity(c, cur));
    if (has_u(c)) TRY(state_defstate(c));
    else TRY(state_image(c));
    c->vel_valid = true;
    return LDDMM_OK;
}

// STATE (Sec. 2.3.2): iota(grad~ pi(m_j)) of m_j = I0 o phi_j, phi_j = id - iota(u~_j), and the
// backward maps of every node: nu~ from -D~_t nu~ = -v~, nu~(1) = 0, stored as iota(nu~_j), and
// J_j = 1 - iota(U~_j) from -D~_t U~ = -div~ v~ + U~ * div~ v~, U~(1) = 0. J~ = pi(1) - U~ obeys
// -D~_t J~ = J~ * div~ v~, the adjoint step of Table 1 row 2 (the same SL-Heun arithmetic), so
// J~ is what is stepped; iota(J~_j) = 1 - iota(U~_j).
static int state_traj(lddmm_ctx* c) {
    const long n = c->n, kc3 = 3 * c->kc;
    const int nt = c->p.nt;
    float2* mt = c->cv[lddmm_ctx::C_T1];
    const float* I0src = cubic(c) ? c->I0c : c->I0;
    for (int j = 0; j <= nt; ++j) {
        TRY(include(c, c->ut + (long)j * kc3, 3, c->fa, n, -1, 0));
        TRY(sl_compose(c->sl, I0src, c->fa, c->to_vox, nullptr, c->fb, c->st));
        TRY(project(c, c->fb, 1, mt));
        for (int b = 0; b < 3; ++b)
            TRY(include(c, mt, 1, c->Gm + (long)j * 3 * n + b * n, n, b, 0));
    }
    float2* nut = c->cv[lddmm_ctx::C_T1];   // nu~_j
    float2* Jt = c->cv[lddmm_ctx::C_T2];    // J~_j (first K^3)
    float* pj = c->PJ + (long)nt * 4 * n;
    LDDMM_CUDA(cudaMemsetAsync(pj, 0, 3 * n * sizeof(float), c->st));
    TRY(fill_field(pj + 3 * n, 1.f, n, c->st));
    LDDMM_CUDA(cudaMemsetAsync(nut, 0, kc3 * sizeof(float2), c->st));
    TRY(project(c, pj + 3 * n, 1, Jt));
    for (int j = nt - 1; j >= 0; --j) {
        const float* src_nu = pj;          // iota(nu~_{j+1}), iota(J~_{j+1})
        const float* src_J = pj + 3 * n;
        if (cubic(c)) {
            TRY(include(c, nut, 3, c->fa, n, -1, 1));
            TRY(include(c, Jt, 1, c->fd, n, -1, 1));
            src_nu = c->fa;
            src_J = c->fd;
        }
        TRY(sl_gather_add(c->sl, src_nu, Dbstep(c, j), Wbstep(c, j), 3, c->fb, c->st));
        TRY(sl_gather_scale(c->sl, src_J, Dbstep(c, j), gamstep(c, j), 1, c->fc, c->st));
        TRY(project(c, c->fb, 3, nut));
        TRY(project(c, c->fc, 1, Jt));
        pj = c->PJ + (long)j * 4 * n;
        TRY(include(c, nut, 3, pj, n, -1, 0));
        TRY(include(c, Jt, 1, pj + 3 * n, n, -1, 0));
    }
    c->solves++;
    return LDDMM_OK;
}

// Spatial derivatives of the stored trajectory needed by gradient and Hessian.
static int ensure_traj(lddmm_ctx* c) {
    if (c->traj_valid) return LDDMM_OK;
    const long n = c->n;
    if (has_u(c)) {
        // the Jacobian of u~_0 = 0 vanishes
        LDDMM_CUDA(cudaMemsetAsync(c->Du, 0, 9 * n * sizeof(float), c->st));
        for (int j = 1; j <= c->p.nt; ++j)
            for (int b = 0; b < 3; ++b)
                TRY(include(c, c->ut + (long)j * 3 * c->kc, 3, c->Du + (long)j * 9 * n + b * n,
                            3 * n, b, 0));
        if (jac_bf16(c)) TRY(pack_jac_bf16(c->Du, c->Du16, n, c->p.nt + 1, c->st));
        if (state_eq(c)) TRY(state_traj(c));
    } else {
        float2* mt = c->cv[lddmm_ctx::C_T1];
        for (int j = 0; j <= c->p.nt; ++j) {
            TRY(project(c, c->ms + (long)j * n, 1, mt));
            for (int b = 0; b < 3; ++b)
                TRY(include(c, mt, 1, c->Gm + (long)j * 3 * n + b * n, n, b, 0));
        }
    }
    c->traj_valid = true;
    return LDDMM_OK;
}

// ------------------------------------------------------------------ adjoint sweeps
// DEFSTATE (Eqs. 35, 37; Table 1 rows 4, 8), backward from rho(1) given spatially in `rho1`:
// out = wL L~ base + sum_j w_j (rho~_j - pi((D iota u~_j)^T iota(rho~_j))). The sweep keeps
// iota(rho~_j) of every node (Rn) and the trapezoid sum of (D iota u~_j)^T iota(rho~_j) runs
// in one pass over all nodes at the end, which writes the accumulator once.
static int adjoint_defstate(lddmm_ctx* c, const float* rho1, const float2* base, float2* out,
                            bool hess) {
    const long n = c->n, kc3 = 3 * c->kc;
    const int nt = c->p.nt;
    float2* rt = c->cv[lddmm_ctx::C_T1];     // rho~_j
    float2* rsum = c->cv[lddmm_ctx::C_T2];   // sum_j w_j rho~_j
    auto rnode = [&](int j) { return c->Rn + (long)j * 3 * n; };
    TRY(project(c, rho1, 3, rt));
    TRY(cube_axpby(rsum, (float)trap_w(c, nt), rt, 0.f, nullptr, kc3, c->st));
    TRY(include(c, rt, 3, rnode(nt), n, -1, 0));  // iota(rho~_nt) values
    for (int j = nt - 1; j >= 0; --j) {
        const float* src = rnode(j + 1);
        if (cubic(c)) {
            TRY(include(c, rt, 3, c->fa, n, -1, 1));
            src = c->fa;
        }
        TRY(sl_gather_scale(c->sl, src, c->Db, c->gam, 3, c->fd, c->st));
        TRY(project(c, c->fd, 3, rt));
        TRY(cube_axpby(rsum, 1.f, rsum, (float)trap_w(c, j), rt, kc3, c->st));
        TRY(include(c, rt, 3, rnode(j), n, -1, 0));
    }
    TRY(accum_JT_nodes(c->g, jac(c, 0, hess), jac_bf16(c) && hess, c->Rn, nt, (float)trap_w(c, 0),
                       (float)c->dt, c->acc, c->st));
    c->solves++;
    float2* pacc = c->cv[lddmm_ctx::C_T0];
    TRY(project(c, c->acc, 3, pacc));
    TRY(cube_axpby(rsum, 1.f, rsum, -1.f, pacc, kc3, c->st));
    TRY(op_L(c, out, base, 1.f, 1.f, rsum, 3, 1));
    return LDDMM_OK;
}

// Non-stationary DEFSTATE adjoint, backward from rho(1): at every node j
// out_j = L~ base_j + rho~_j - pi((D iota u~_j)^T iota(rho~_j)) (the integrand of Eqs. 32-33
// at t_j), step j along X+_j with the factor gamma_j of nodes j and j + 1.
static int adjoint_defstate_ns(lddmm_ctx* c, const float* rho1, const float2* base, float2* out,
                               bool hess) {
    const long n = c->n, kc3 = 3 * c->kc;
    const int nt = c->p.nt;
    float2* rt = c->cv[lddmm_ctx::C_T1];     // rho~_j
    float2* pj = c->cv[lddmm_ctx::C_T0];     // node j's assembled data term
    TRY(project(c, rho1, 3, rt));
    for (int j = nt; j >= 0; --j) {
        if (j < nt) {
            const float* src = c->fc;        // iota(rho~_{j+1})
            if (cubic(c)) {
                TRY(include(c, rt, 3, c->fa, n, -1, 1));
                src = c->fa;
            }
            TRY(sl_gather_scale(c->sl, src, Dbstep(c, j), gamstep(c, j), 3, c->fd, c->st));
            TRY(project(c, c->fd, 3, rt));
        }
        TRY(include(c, rt, 3, c->fc, n, -1, 0));
        TRY(accum_JT(c->g, jac(c, j, hess), jac_bf16(c) && hess, c->fc, 1.f, c->acc, 1, c->st));
        TRY(project(c, c->acc, 3, pj));
        TRY(cube_axpby(pj, 1.f, rt, -1.f, pj, kc3, c->st));
        TRY(op_L(c, vcube(c, out, j), vcube(c, base, j), 1.f, 1.f, pj, 3, 1));
    }
    c->solves++;
    return LDDMM_OK;
}

// Image-type assembly (IMAGE and STATE, Eqs. 15-16): node j contributes pi(s_j Gm_j), s_j the
// values of a projected scalar, which the sweeps write to image_vals(c, j). Stationary: the
// sweep keeps s_j of every node, and at the end one pass over all nodes forms
// acc = sum_j w_j s_j Gm_j, then out = L~ base + pi(acc). Non-stationary: out_j = L~ base_j +
// pi(s_j Gm_j) at every node.
static float* image_vals(lddmm_ctx* c, int j) { return ns(c) ? c->fc : c->Sn + (long)j * c->n; }
static int image_term(lddmm_ctx* c, int j, const float* vals, const float2* base, float2* out) {
    if (!ns(c)) return LDDMM_OK;
    const float* gm = c->Gm + (long)j * 3 * c->n;
    TRY(accum_sv(c->g, vals, gm, 1.f, c->acc, 1, c->st));
    float2* pacc = c->cv[lddmm_ctx::C_T0];
    TRY(project(c, c->acc, 3, pacc));
    return op_L(c, vcube(c, out, j), vcube(c, base, j), 1.f, 1.f, pacc, 3, 1);
}
static int image_finish(lddmm_ctx* c, const float2* base, float2* out) {
    if (ns(c)) return LDDMM_OK;
    TRY(accum_sv_nodes(c->g, c->Sn, c->Gm, c->p.nt, (float)trap_w(c, 0), (float)c->dt, c->acc, c->st));
    float2* pacc = c->cv[lddmm_ctx::C_T0];
    TRY(project(c, c->acc, 3, pacc));
    return op_L(c, out, base, 1.f, 1.f, pacc, 3, 1);
}

// STATE, gradient and Hessian (Eqs. 15-16 with lambda(t) = J(t) lambda(1) o psi(t)):
// out = L~ base + sum_j w_j pi(iota(pi(f_j)) Gm_j), f_j = J_j f1 o psi_j, with f1 = lambda(1) for the
// gradient and dlambda(1) for the Gauss-Newton Hessian. No recurrence: every node reads f1.
static int pullback_assemble(lddmm_ctx* c, const float* f1, const float2* base, float2* out) {
    const long n = c->n;
    const int nt = c->p.nt;
    const float* src = f1;
    if (cubic(c)) {
        TRY(bspline_prefilter(c->g, f1, 1, c->fa, c->st));
        src = c->fa;
    }
    float2* lt = c->cv[lddmm_ctx::C_T1];
    for (int j = nt; j >= 0; --j) {
        const float* pj = c->PJ + (long)j * 4 * n;
        TRY(sl_compose(c->sl, src, pj, c->to_vox, pj + 3 * n, c->fd, c->st));
        TRY(project(c, c->fd, 1, lt));
        TRY(include(c, lt, 1, image_vals(c, j), n, -1, 0));
        TRY(image_term(c, j, image_vals(c, j), base, out));
    }
    c->solves++;
    return image_finish(c, base, out);
}

// IMAGE, gradient (Eqs. 15, 18; Table 1 row 2): spatial adjoint lambda from
// lambda(1) = -(2/sigma2)(m1 - I1); g = L~ v~ + sum_j w_j pi(iota(pi(lambda_j)) Gm_j).
static int gradient_image_adjoint(lddmm_ctx* c, const float2* vt, float2* g) {
    const long n = c->n;
    const int nt = c->p.nt;
    float2* lt = c->cv[lddmm_ctx::C_T1];
    TRY(scaled_diff(c->g, c->ms + (long)nt * n, c->I1, (float)(-2.0 / c->p.sigma2), c->fb, c->st));
    for (int j = nt; j >= 0; --j) {
        // fb holds lambda_j (spatial)
        TRY(project(c, c->fb, 1, lt));
        TRY(include(c, lt, 1, image_vals(c, j), n, -1, 0));
        TRY(image_term(c, j, image_vals(c, j), vt, g));
        if (j > 0) {
            const float* src = c->fb;
            if (cubic(c)) {
                TRY(bspline_prefilter(c->g, c->fb, 1, c->fa, c->st));
                src = c->fa;
            }
            // step j - 1 runs between nodes j - 1 and j
            TRY(sl_gather_scale(c->sl, src, Dbstep(c, j - 1), gamstep(c, j - 1), 1, c->fd, c->st));
            std::swap(c->fb, c->fd);
        }
    }
    c->solves++;
    return image_finish(c, vt, g);
}

// ------------------------------------------------------------------ objective / gradient
static int objective_impl(lddmm_ctx* c, const float2* vt, bool known_same, double* E, double* Er,
                          double* Ed) {
    TRY(ensure_state(c, vt, known_same));
    TRY(data_term(c, nullptr));
    TRY(reg_term(c, vt));
    TRY(read_scalars(c, 2));
    double ed = c->hsc[0] / (double)c->n / c->p.sigma2, er = 0.5 * c->hsc[1] * dscale(c);
    if (E) *E = er + ed;
    if (Er) *Er = er;
    if (Ed) *Ed = ed;
    return LDDMM_OK;
}

static int gradient_impl(lddmm_ctx* c, const float2* vt, bool known_same, float2* g, double* E,
                         double* Er, double* Ed) {
    TRY(ensure_state(c, vt, known_same));
    TRY(ensure_traj(c));
    float2* cur = c->cv[lddmm_ctx::C_CUR];
    if (state_eq(c)) {
        TRY(data_term(c, nullptr));
        TRY(scaled_diff(c->g, c->m1, c->I1, (float)(-2.0 / c->p.sigma2), c->fb, c->st));
        TRY(pullback_assemble(c, c->fb, cur, g));
    } else if (c->p.variant == LDDMM_V_DEFSTATE) {
        TRY(data_term(c, c->fb));
        if (ns(c)) TRY(adjoint_defstate_ns(c, c->fb, cur, g, false));
        else TRY(adjoint_defstate(c, c->fb, cur, g, false));
    } else {
        TRY(data_term(c, nullptr));
        TRY(gradient_image_adjoint(c, cur, g));
    }
    TRY(reg_term(c, cur));
    TRY(read_scalars(c, 2));
    double ed = c->hsc[0] / (double)c->n / c->p.sigma2, er = 0.5 * c->hsc[1] * dscale(c);
    if (E) *E = er + ed;
    if (Er) *Er = er;
    if (Ed) *Ed = ed;
    return LDDMM_OK;
}

// Gauss-Newton H dv~ at the current velocity (state and trajectory must be current).
static int hessian_impl(lddmm_ctx* c, const float2* dvt, float2* out) {
    TRY(ensure_traj(c));
    if (has_u(c) && !c->warp_valid) TRY(data_term(c, nullptr));
    const long n = c->n, kc3 = 3 * c->kc;
    const int nt = c->p.nt;
    TRY(include(c, dvt, 3, c->dvsp, n, -1, 0));
    if (has_u(c)) {
        // incremental state D~_t du~ = dv~ - D~u~ * dv~ (Eq. 36; Table 1 row 7)
        float2* dut = c->cv[lddmm_ctx::C_T1];
        float* Fold = c->fa;
        float* Fnew = c->fd;
        TRY(defstate_rhs(c->g, jac(c, 0, true), jac_bf16(c), c->dvsp, Fold, c->st));
        LDDMM_CUDA(cudaMemsetAsync(dut, 0, kc3 * sizeof(float2), c->st));
        for (int j = 0; j < nt; ++j) {
            // du~_0 = 0: its values (or B-spline coefficients) are cleared, not synthesised
            if (j == 0) LDDMM_CUDA(cudaMemsetAsync(c->fb, 0, 3 * n * sizeof(float), c->st));
            else TRY(include(c, dut, 3, c->fb, n, -1, cubic(c)));
            const float* Fsrc = Fold;
            if (cubic(c)) {
                TRY(bspline_prefilter(c->g, Fold, 3, c->acc, c->st));
                Fsrc = c->acc;
            }
            // non-stationary: the right-hand side at node j + 1 uses dv~_{j+1}
            if (ns(c)) TRY(include(c, vcube(c, dvt, j + 1), 3, c->dvsp, n, -1, 0));
            TRY(sl_inc_defstate(c->sl, c->fb, Dfstep(c, j), Fsrc, jac(c, j + 1, true), jac_bf16(c),
                                c->dvsp, c->dt, c->fc, Fnew, c->st));
            TRY(project(c, c->fc, 3, dut));
            std::swap(Fold, Fnew);
        }
        c->solves++;
        TRY(include(c, dut, 3, c->fa, n, -1, 0));
        if (state_eq(c)) {
            // Gauss-Newton: dlambda(t) = J(t) dlambda(1) o psi(t), dlambda(1) = -(2/sigma2) dm1,
            // dm1 = -G . iota(du~(1))
            TRY(state_dlam1(c->g, c->G, c->fa, c->p.sigma2, c->fb, c->st));
            return pullback_assemble(c, c->fb, dvt, out);
        }
        // drho(1) = pi(-(2/sigma2) dm1 G), dm1 = -G . iota(du~(1))
        TRY(defstate_drho1(c->g, c->G, c->fa, c->p.sigma2, c->fb, c->st));
        if (ns(c)) return adjoint_defstate_ns(c, c->fb, dvt, out, true);
        return adjoint_defstate(c, c->fb, dvt, out, true);
    }
    // IMAGE: incremental state D~_t dm~ = -grad~ m~ * dv~ (Eq. 19; Table 1 row 5)
    float2* dmt = c->cv[lddmm_ctx::C_T1];
    float* Fold = c->fa;
    float* Fnew = c->fd;
    TRY(image_rhs(c->g, c->Gm, c->dvsp, Fold, c->st));
    LDDMM_CUDA(cudaMemsetAsync(dmt, 0, c->kc * sizeof(float2), c->st));
    for (int j = 0; j < nt; ++j) {
        // dm~_0 = 0: cleared, not synthesised
        if (j == 0) LDDMM_CUDA(cudaMemsetAsync(c->fb, 0, n * sizeof(float), c->st));
        else TRY(include(c, dmt, 1, c->fb, n, -1, cubic(c)));
        const float* Fsrc = Fold;
        if (cubic(c)) {
            TRY(bspline_prefilter(c->g, Fold, 1, c->acc, c->st));
            Fsrc = c->acc;
        }
        // non-stationary: the right-hand side at node j + 1 uses dv~_{j+1}
        if (ns(c)) TRY(include(c, vcube(c, dvt, j + 1), 3, c->dvsp, n, -1, 0));
        TRY(sl_inc_image(c->sl, c->fb, Dfstep(c, j), Fsrc, c->Gm + (long)(j + 1) * 3 * n, c->dvsp,
                         c->dt, c->fc, Fnew, c->st));
        TRY(project(c, c->fc, 1, dmt));
        std::swap(Fold, Fnew);
    }
    c->solves++;
    // incremental adjoint -D~_t dlambda~ = dlambda~ * div~ v~ (Eq. 20), dlambda~(1) = -(2/s2) dm~(1)
    TRY(cube_axpby(dmt, (float)(-2.0 / c->p.sigma2), dmt, 0.f, nullptr, c->kc, c->st));
    for (int j = nt; j >= 0; --j) {
        TRY(include(c, dmt, 1, image_vals(c, j), n, -1, 0));
        TRY(image_term(c, j, image_vals(c, j), dvt, out));
        if (j > 0) {
            const float* src = image_vals(c, j);
            if (cubic(c)) {
                TRY(include(c, dmt, 1, c->fa, n, -1, 1));
                src = c->fa;
            }
            TRY(sl_gather_scale(c->sl, src, Dbstep(c, j - 1), gamstep(c, j - 1), 1, c->fd, c->st));
            TRY(project(c, c->fd, 1, dmt));
        }
    }
    c->solves++;
    return image_finish(c, dvt, out);
}

// device comparison of vt against the cached velocity: true if bitwise equal
__global__ void k_cube_neq(const float2* a, const float2* b, long n, int* flag) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float2 x = a[i], y = b[i];
        if (__float_as_uint(x.x) != __float_as_uint(y.x) || __float_as_uint(x.y) != __float_as_uint(y.y))
            *flag = 1;
    }
}

static int same_as_current(lddmm_ctx* c, const float2* vt, bool* same) {
    *same = false;
    if (!c->vel_valid) return LDDMM_OK;
    int* flag = reinterpret_cast<int*>(c->dsc + 8);
    LDDMM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->st));
    long n = nvec(c);
    {
        KTRACE("cube_neq", c->st, 16.0 * n, 0);
        k_cube_neq<<<(int)((n + 255) / 256), 256, 0, c->st>>>(vt, c->cv[lddmm_ctx::C_CUR], n, flag);
    }
    LDDMM_CHECK_LAUNCH();
    int h = 1;
    LDDMM_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    LDDMM_CUDA(cudaStreamSynchronize(c->st));
    *same = (h == 0);
    return LDDMM_OK;
}

// ------------------------------------------------------------------ graph-captured Hv
// H cv[C_P] -> cv[C_HP] at the current state. With graphs enabled, the first product runs
// eagerly (it settles kernel attributes), the second is captured into a CUDA graph and every
// later product (all PCG iterations of all Gauss-Newton updates: the buffers never move)
// replays it. Tracing forces the eager path so that kernels can be timed.
static int hessian_pcg(lddmm_ctx* c) {
    float2* pp = c->cv[lddmm_ctx::C_P];
    float2* Hp = c->cv[lddmm_ctx::C_HP];
    TRY(ensure_traj(c));
    if (has_u(c) && !c->warp_valid) TRY(data_term(c, nullptr));
    if (!c->use_graphs || c->graph_failed || tracing()) return hessian_impl(c, pp, Hp);
    if (c->hv_exec) {
        LDDMM_CUDA(cudaGraphLaunch(c->hv_exec, c->st));
        count_launches(c->hv_graph_launches);
        return LDDMM_OK;
    }
    if (c->hv_eager_runs++ == 0) return hessian_impl(c, pp, Hp);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graph_failed = true;
        return hessian_impl(c, pp, Hp);
    }
    capture_begin();
    int rc = hessian_impl(c, pp, Hp);
    long nl = capture_end();
    cudaError_t e = cudaStreamEndCapture(c->st, &graph);
    if (rc != LDDMM_OK || e != cudaSuccess || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        c->graph_failed = true;
        return hessian_impl(c, pp, Hp);
    }
    e = cudaGraphInstantiate(&c->hv_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->hv_exec = nullptr;
        c->graph_failed = true;
        return hessian_impl(c, pp, Hp);
    }
    c->hv_graph_launches = nl;
    LDDMM_CUDA(cudaGraphLaunch(c->hv_exec, c->st));
    count_launches(nl);
    return LDDMM_OK;
}

// ------------------------------------------------------------------ GN-Krylov driver
// <a, b> of velocity-shaped vectors (non-stationary: trapezoid-weighted over the nodes)
static double dot_host(lddmm_ctx* c, const float2* a, const float2* b, int* rc) {
    *rc = dot_f2_nodes(a, b, 3 * c->kc, nodes(c), c->dt, c->partials, c->dsc, c->st);
    if (*rc) return 0;
    *rc = read_scalars(c, 1);
    return c->hsc[0] * dscale(c);
}

// ------------------------------------------------------------------ two-level preconditioner
// The multi-level preconditioner named in Secs. 6-7 (that of the CLAIRE solver), read as: the
// same problem on the half grid with band Kc = 2 floor(K/4) and spectrally restricted images
// (the coarse context); P^{-1} r = E y + theta L~^{-1}(r - E R r), y from at most tl_inner PCG
// iterations (relative tolerance 0.1, preconditioner L~_c^{-1}) on H_c y = R r, H_c the coarse
// Gauss-Newton Hessian at R v~, theta = <R r, y> / <R r, L~_c^{-1} R r> (1 if R r = 0), which
// puts the modes above the coarse band on the scale of the coarse solve: with alpha = 0.0025 the
// data term, not L~, dominates H there. The outer Krylov method is then flexible PCG.
static const double kInnerTol = 0.1;
static bool two_level(const lddmm_ctx* c) { return c->coarse && c->tl_inner > 0; }

static int pcg_solve(lddmm_ctx* c, double bnorm, double eta, int maxit, int* its, int* inner_its);

// z = P^{-1} r (velocity-shaped vectors of c)
static int apply_precond(lddmm_ctx* c, const float2* r, float2* z, int* inner_its) {
    TRY(op_L(c, z, r, 1.f, 0.f, nullptr, 3 * nodes(c), -1));
    if (!two_level(c)) return LDDMM_OK;
    lddmm_ctx* q = c->coarse;
    float2* b = q->cv[lddmm_ctx::C_G];   // R r
    float2* y = q->cv[lddmm_ctx::C_X];
    float2* lb = q->cv[lddmm_ctx::C_Z];
    int rc = 0;
    TRY(cube_restrict(r, c->K, b, q->K, 3, c->st));
    LDDMM_CUDA(cudaMemcpyAsync(q->cv[lddmm_ctx::C_R], b, nvec(q) * sizeof(float2),
                               cudaMemcpyDeviceToDevice, c->st));
    const double bb = dot_host(q, b, b, &rc);
    TRY(rc);
    int its = 0;
    TRY(pcg_solve(q, std::sqrt(bb), kInnerTol, c->tl_inner, &its, nullptr));
    if (inner_its) *inner_its += its;
    TRY(op_L(q, lb, b, 1.f, 0.f, nullptr, 3, -1));
    const double by = dot_host(q, b, y, &rc);
    TRY(rc);
    const double bl = dot_host(q, b, lb, &rc);
    TRY(rc);
    const double theta = bl > 0.0 ? by / bl : 1.0;
    return cube_two_level(z, c->K, y, q->K, (float)theta, 3, c->st);
}

// PCG on H x = b from x = 0, b in cv[C_R] on entry (overwritten by the residual), x left in
// cv[C_X]; flexible (beta = <z', r' - r> / <z, r>) with the two-level preconditioner. Stops on
// ||r|| <= eta bnorm, after maxit products, or on non-positive curvature (at the first
// iteration x = P^{-1} b, the preconditioned steepest-descent direction).
static int pcg_solve(lddmm_ctx* c, double bnorm, double eta, int maxit, int* its, int* inner_its) {
    const long kc3 = nvec(c);
    float2 *r = c->cv[lddmm_ctx::C_R], *z = c->cv[lddmm_ctx::C_Z], *pp = c->cv[lddmm_ctx::C_P];
    float2 *Hp = c->cv[lddmm_ctx::C_HP], *x = c->cv[lddmm_ctx::C_X], *rp = c->cv[lddmm_ctx::C_RP];
    const bool flex = two_level(c);
    int rc = 0;
    *its = 0;
    LDDMM_CUDA(cudaMemsetAsync(x, 0, kc3 * sizeof(float2), c->st));
    TRY(apply_precond(c, r, z, inner_its));
    TRY(cube_axpby(pp, 1.f, z, 0.f, nullptr, kc3, c->st));
    double rz = dot_host(c, r, z, &rc);
    TRY(rc);
    for (int i = 0; i < maxit; ++i) {
        TRY(hessian_pcg(c));
        ++*its;
        const double pHp = dot_host(c, pp, Hp, &rc);
        TRY(rc);
        if (pHp <= 0.0) {
            if (i == 0)
                LDDMM_CUDA(cudaMemcpyAsync(x, z, kc3 * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
            break;
        }
        const double a = rz / pHp;
        TRY(cube_axpby(x, 1.f, x, (float)a, pp, kc3, c->st));
        if (flex)
            LDDMM_CUDA(cudaMemcpyAsync(rp, r, kc3 * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
        TRY(cube_axpby(r, 1.f, r, (float)-a, Hp, kc3, c->st));
        const double rn = std::sqrt(dot_host(c, r, r, &rc));
        TRY(rc);
        if (rn <= eta * bnorm) break;
        TRY(apply_precond(c, r, z, inner_its));
        const double rz2 = dot_host(c, r, z, &rc);
        TRY(rc);
        double num = rz2;
        if (flex) {
            num -= dot_host(c, rp, z, &rc);
            TRY(rc);
        }
        TRY(cube_axpby(pp, 1.f, z, (float)(num / rz), pp, kc3, c->st));
        rz = rz2;
    }
    return LDDMM_OK;
}

// The coarse Hessian of the next solve is taken at R v~ (v the current iterate).
static int coarse_prepare(lddmm_ctx* c, const float2* v) {
    lddmm_ctx* q = c->coarse;
    q->use_graphs = c->use_graphs;
    float2* vq = q->cv[lddmm_ctx::C_VT];
    TRY(cube_restrict(v, c->K, vq, q->K, 3, c->st));
    TRY(ensure_state(q, vq, false));
    return ensure_traj(q);
}

static int register_impl(lddmm_ctx* c, float2* v_io, const double* gref_in, lddmm_report* rep) {
    auto t0 = std::chrono::steady_clock::now();
    const long kc3 = nvec(c);             // float2 per velocity-shaped vector
    const int K = c->K;
    const int ncube = 3 * nodes(c);       // K^3 cubes per vector
    std::memset(rep, 0, sizeof(*rep));
    c->solves = 0;
    int rc = 0;
    float2* v = c->cv[lddmm_ctx::C_V];
    float2* vtr = c->cv[lddmm_ctx::C_VT];
    float2* g = c->cv[lddmm_ctx::C_G];
    float2 *r = c->cv[lddmm_ctx::C_R], *x = c->cv[lddmm_ctx::C_X];
    LDDMM_CUDA(cudaMemcpyAsync(v, v_io, kc3 * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
    if (!spatial(c)) TRY(cube_hermitian(v, K, ncube, c->st));

    double gref2, grefi;
    double E, Er, Ed;
    if (gref_in) {
        gref2 = gref_in[0];
        grefi = gref_in[1];
    } else {
        // reference: the gradient at v~ = 0 (cold start)
        TRY(max_abs(c, v, kc3, c->dsc));
        TRY(read_scalars(c, 1));
        if (c->hsc[0] != 0.0) {
            LDDMM_CUDA(cudaMemsetAsync(vtr, 0, kc3 * sizeof(float2), c->st));
            TRY(gradient_impl(c, vtr, false, g, nullptr, nullptr, nullptr));
            gref2 = std::sqrt(dot_host(c, g, g, &rc));
            TRY(rc);
            TRY(max_abs(c, g, kc3, c->dsc));
            TRY(read_scalars(c, 1));
            grefi = c->hsc[0];
        } else {
            gref2 = grefi = -1;  // filled from the first gradient below
        }
    }
    TRY(gradient_impl(c, v, false, g, &E, &Er, &Ed));
    double gn = std::sqrt(dot_host(c, g, g, &rc));
    TRY(rc);
    if (gref2 < 0) {
        gref2 = gn;
        TRY(max_abs(c, g, kc3, c->dsc));
        TRY(read_scalars(c, 1));
        grefi = c->hsc[0];
    }
    if (!(gref2 > 0)) gref2 = 1.0;
    if (!(grefi > 0)) grefi = 1.0;
    rep->E0 = E;
    c->hist.clear();
    auto record = [&](double Ecur) {
        // taken after the iterate's gradient norm reached the host, so the device is done
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        c->hist.push_back({t, gn / gref2, Ecur, (double)rep->pcg_iters_total, (double)c->solves});
    };
    record(E);
    int stop = LDDMM_STOP_MAXIT;
    int gn_iters = 0;
    for (int it = 0; it < c->p.max_gn; ++it) {
        if (gn / gref2 <= c->p.gtol) {
            stop = LDDMM_STOP_GTOL;
            break;
        }
        const double eta = std::min(0.5, std::sqrt(gn / gref2));
        // PCG on H x = -g from x0 = 0 (flexible PCG with the two-level preconditioner, whose
        // coarse Hessian is taken at the current iterate)
        if (two_level(c)) TRY(coarse_prepare(c, v));
        TRY(cube_axpby(r, -1.f, g, 0.f, nullptr, kc3, c->st));
        int its = 0, inner = 0;
        TRY(pcg_solve(c, gn, eta, c->p.max_pcg, &its, &inner));
        rep->pcg_iters_total += its;
        rep->pcg_inner_total += inner;
        // Armijo backtracking on eps
        const double slope = dot_host(c, g, x, &rc);
        TRY(rc);
        double eps = 1.0, Et = 0;
        bool ok = false;
        for (int ls = 0; ls <= 10; ++ls) {
            TRY(cube_axpby(vtr, 1.f, v, (float)eps, x, kc3, c->st));
            TRY(objective_impl(c, vtr, false, &Et, nullptr, nullptr));
            if (Et <= E + 1e-4 * eps * slope) {
                ok = true;
                break;
            }
            eps *= 0.5;
        }
        if (!ok) {
            stop = LDDMM_STOP_LINESEARCH;
            break;
        }
        LDDMM_CUDA(cudaMemcpyAsync(v, vtr, kc3 * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
        gn_iters = it + 1;
        // the accepted trial's state is current: the gradient reuses it
        TRY(gradient_impl(c, vtr, true, g, &E, &Er, &Ed));
        gn = std::sqrt(dot_host(c, g, g, &rc));
        TRY(rc);
        record(E);
    }
    if (stop == LDDMM_STOP_MAXIT && gn / gref2 <= c->p.gtol) stop = LDDMM_STOP_GTOL;
    // if the line search failed, the state in the buffers belongs to a rejected trial
    if (stop == LDDMM_STOP_LINESEARCH) TRY(objective_impl(c, v, false, &E, &Er, &Ed));
    // MSE_rel = ||m1 - I1||^2 / ||I0 - I1||^2
    const float* m1 = has_u(c) ? c->m1 : c->ms + (long)c->p.nt * c->n;
    TRY(sum_sq_diff(m1, c->I1, c->n, c->partials, c->dsc, c->st));
    TRY(sum_sq_diff(c->I0, c->I1, c->n, c->partials, c->dsc + 1, c->st));
    TRY(max_abs(c, g, kc3, c->dsc + 2));
    TRY(read_scalars(c, 3));
    rep->mse_rel = c->hsc[1] > 0 ? c->hsc[0] / c->hsc[1] : 0.0;
    rep->grad_rel_inf = c->hsc[2] / grefi;
    rep->grad_rel_l2 = gn / gref2;
    rep->E = E;
    rep->E_reg = Er;
    rep->E_data = Ed;
    rep->gn_iters = gn_iters;
    rep->stop_reason = stop;
    rep->solves = c->solves;
    LDDMM_CUDA(cudaMemcpyAsync(v_io, v, kc3 * sizeof(float2), cudaMemcpyDeviceToDevice, c->st));
    LDDMM_CUDA(cudaStreamSynchronize(c->st));
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return LDDMM_OK;
}

// ================================================================== the C ABI
static int ctx_alloc(lddmm_ctx* c) {
    const long n = c->n, kc3 = 3 * c->kc;
    const int nt = c->p.nt;
    const bool def = has_u(c), cub = cubic(c);
    if (spatial(c)) {
        TRY(spatial_fft_create(c->g, c->st, &c->fft));
    } else {
        float* twm = nullptr;
        TRY(dalloc_t(c, &twm, twiddle_floats(c->g, c->K)));
        TRY(twiddle_init(c->g, c->K, twm, c->tw, c->st));
    }
    TRY(dalloc_t(c, &c->I0, n));
    TRY(dalloc_t(c, &c->I1, n));
    if (cub) TRY(dalloc_t(c, &c->I0c, n));
    const size_t nodes_ = (size_t)nodes(c), steps = ns(c) ? (size_t)nt : 1;
    TRY(dalloc_t(c, &c->v, nodes_ * 3 * n));
    TRY(dalloc_t(c, &c->d, nodes_ * n));
    if (cub) {
        TRY(dalloc_t(c, &c->vc, nodes_ * 3 * n));
        TRY(dalloc_t(c, &c->dc, nodes_ * n));
    }
    TRY(dalloc_t(c, &c->Df, steps * 3 * n));
    TRY(dalloc_t(c, &c->Db, steps * 3 * n));
    TRY(dalloc_t(c, &c->gam, steps * n));
    if (def) {
        TRY(dalloc_t(c, &c->W, steps * 3 * n));
        TRY(dalloc_t(c, &c->ut, (size_t)(nt + 1) * kc3));
        TRY(dalloc_t(c, &c->Du, (size_t)(nt + 1) * 9 * n));
        if (jac_bf16(c))
            TRY(dalloc_t(c, reinterpret_cast<uint16_t**>(&c->Du16), (size_t)(nt + 1) * jac_bf16_stride(n)));
        TRY(dalloc_t(c, &c->G, 3 * n));
        TRY(dalloc_t(c, &c->m1, n));
    } else {
        TRY(dalloc_t(c, &c->ms, (size_t)(nt + 1) * n));
    }
    if (!def || state_eq(c)) TRY(dalloc_t(c, &c->Gm, (size_t)(nt + 1) * 3 * n));
    if (state_eq(c)) {
        TRY(dalloc_t(c, &c->Wb, steps * 3 * n));
        TRY(dalloc_t(c, &c->PJ, (size_t)(nt + 1) * 4 * n));
    }
    if (c->p.variant == LDDMM_V_DEFSTATE && !ns(c)) TRY(dalloc_t(c, &c->Rn, (size_t)(nt + 1) * 3 * n));
    if (c->p.variant != LDDMM_V_DEFSTATE && !ns(c)) TRY(dalloc_t(c, &c->Sn, (size_t)(nt + 1) * n));
    for (float** f : {&c->fa, &c->fb, &c->fc, &c->fd, &c->acc, &c->dvsp}) TRY(dalloc_t(c, f, 3 * n));
    if (!spatial(c)) {
        long se = spectral_scratch_elems(c->g, c->K, 3);
        TRY(dalloc_t(c, &c->s1, se));
        TRY(dalloc_t(c, &c->s2, se));
    }
    for (int i = 0; i < lddmm_ctx::C_NUM; ++i) {
        TRY(dalloc_t(c, &c->cv[i], nvec(c)));
        LDDMM_CUDA(cudaMemsetAsync(c->cv[i], 0, nvec(c) * sizeof(float2), c->st));
    }
    TRY(dalloc_t(c, &c->partials, 2 * kReduceBlocks));   // the Jacobian range uses two rows
    TRY(dalloc_t(c, &c->dsc, 16));
    LDDMM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&c->hsc), 16 * sizeof(double)));
    return LDDMM_OK;
}

static int check_ctx(lddmm_ctx* c) {
    if (!c) { set_error("context is NULL"); return LDDMM_EINVAL; }
    if (c->sticky != LDDMM_OK) {
        set_error("context is in an error state (" + std::to_string(c->sticky) + ")");
        return c->sticky;
    }
    return LDDMM_OK;
}

#define CTX_CALL(c, expr)                 \
    do {                                  \
        int rc0__ = check_ctx(c);         \
        if (rc0__) return rc0__;          \
        int rc1__ = (expr);               \
        if (rc1__) return fail(c, rc1__); \
        return LDDMM_OK;                  \
    } while (0)

static int after_images(lddmm_ctx* c);

// The coarse level's images: the spectral restriction of the context's images to the half grid.
static int coarse_images(lddmm_ctx* c) {
    lddmm_ctx* q = c->coarse;
    const float* in[2] = {c->I0, c->I1};
    float* out[2] = {q->I0, q->I1};
    TRY(spectral_restrict_half(c->g, in, q->g, out, 2, c->st));
    return after_images(q);
}

static int after_images(lddmm_ctx* c) {
    c->vel_valid = c->traj_valid = c->warp_valid = false;
    c->have_images = true;
    if (cubic(c)) TRY(bspline_prefilter(c->g, c->I0, 1, c->I0c, c->st));
    if (c->coarse) TRY(coarse_images(c));
    return LDDMM_OK;
}

// Creates the coarse level of the two-level preconditioner (half grid, band 2 floor(K/4), same
// variant, interpolation, nt, alpha, s, sigma^2 and precision form; stream shared).
static int make_coarse(lddmm_ctx* c) {
    if (spatial(c) || ns(c)) {
        set_error("the two-level preconditioner needs a band-limited stationary context");
        return LDDMM_EINVAL;
    }
    if (c->K < 8 || (c->g.nx & 1) || (c->g.ny & 1) || (c->g.nz & 1)) {
        set_error("the two-level preconditioner needs K >= 8 and even nx, ny, nz");
        return LDDMM_EINVAL;
    }
    lddmm_params cp = c->p;
    cp.nx /= 2;
    cp.ny /= 2;
    cp.nz /= 2;
    cp.K = 2 * (c->K / 4);
    lddmm_ctx* q = nullptr;
    TRY(lddmm_create(&cp, c->st, &q));
    c->coarse = q;
    if (c->have_images) {
        int rc = coarse_images(c);
        if (rc) {
            std::string msg = g_last_error;
            lddmm_destroy(q);
            c->coarse = nullptr;
            set_error(msg);
            return rc;
        }
    }
    return LDDMM_OK;
}

extern "C" {

const char* lddmm_last_error(void) { return g_last_error.c_str(); }

const char* lddmm_version(void) { return "lddmm-b300 0.1 sm_103a"; }

int lddmm_device_error(int* code) {
    if (!code) { set_error("code is NULL"); return LDDMM_EINVAL; }
    LDDMM_CUDA(cudaDeviceSynchronize());
    int conv = 0;
    TRY(tc_take_error(code));
    TRY(tc_conv_take_error(&conv));
    if (*code == LDDMM_OK) *code = conv;
    return LDDMM_OK;
}

int lddmm_selftest_wait(double seconds, int* status) { return wait_selftest(seconds, status); }

int lddmm_set_workspace_limit(long long bytes) {
    if (bytes < 0) { set_error("workspace limit must be >= 0 (0: none)"); return LDDMM_EINVAL; }
    g_ws_limit.store(bytes);
    return LDDMM_OK;
}

int lddmm_workspace_bytes(lddmm_ctx* c, long long* bytes) {
    if (!bytes) { set_error("bytes is NULL"); return LDDMM_EINVAL; }
    int rc = check_ctx(c);
    if (rc) return rc;
    *bytes = c->ws_bytes;
    return LDDMM_OK;
}

int lddmm_create(const lddmm_params* params, void* stream, lddmm_ctx** out) {
    if (!out) { set_error("out is NULL"); return LDDMM_EINVAL; }
    *out = nullptr;
    TRY(validate(params));
    lddmm_ctx* c = new lddmm_ctx();
    c->p = *params;
    c->g = Grid{params->nx, params->ny, params->nz};
    c->n = c->g.ntot();
    c->K = params->spatial ? 0 : params->K;
    // float2 per component of a velocity-shaped vector: K^3 coefficients, or a field of n
    // floats (n even: nx is) viewed as n/2 float2 in the spatial form
    c->kc = params->spatial ? c->n / 2 : (long)c->K * c->K * c->K;
    c->st = static_cast<cudaStream_t>(stream);
    c->dt = 1.0 / params->nt;
    c->to_vox[0] = (float)(params->nx / (2.0 * M_PI));
    c->to_vox[1] = (float)(params->ny / (2.0 * M_PI));
    c->to_vox[2] = (float)(params->nz / (2.0 * M_PI));
    c->sl = SLArgs{c->g, params->interp};
    int rc = ctx_alloc(c);
    if (rc) {
        std::string msg = g_last_error;
        lddmm_destroy(c);
        set_error(msg);
        return rc;
    }
    *out = c;
    return LDDMM_OK;
}

int lddmm_destroy(lddmm_ctx* c) {
    if (!c) return LDDMM_OK;
    cudaStreamSynchronize(c->st);   // also for the legacy default stream (st == NULL)
    if (c->hv_exec) cudaGraphExecDestroy(c->hv_exec);
    lddmm_destroy(c->coarse);
    spatial_fft_destroy(c->fft);
    for (void* p : c->allocs) cudaFree(p);
    if (c->hsc) cudaFreeHost(c->hsc);
    delete c;
    return LDDMM_OK;
}

int lddmm_set_images(lddmm_ctx* c, const float* I0, const float* I1) {
    if (!I0 || !I1) { set_error("image pointer is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        LDDMM_CUDA(cudaMemcpyAsync(c->I0, I0, c->n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
        LDDMM_CUDA(cudaMemcpyAsync(c->I1, I1, c->n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
        return after_images(c);
    })());
}

int lddmm_set_images_host(lddmm_ctx* c, const float* I0, const float* I1) {
    if (!I0 || !I1) { set_error("image pointer is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        LDDMM_CUDA(cudaMemcpyAsync(c->I0, I0, c->n * sizeof(float), cudaMemcpyHostToDevice, c->st));
        LDDMM_CUDA(cudaMemcpyAsync(c->I1, I1, c->n * sizeof(float), cudaMemcpyHostToDevice, c->st));
        return after_images(c);
    })());
}

int lddmm_objective(lddmm_ctx* c, const float* v, double* E, double* Er, double* Ed) {
    if (!v) { set_error("v is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, objective_impl(c, reinterpret_cast<const float2*>(v), false, E, Er, Ed));
}

int lddmm_gradient(lddmm_ctx* c, const float* v, float* g, double* E, double* Er, double* Ed) {
    if (!v || !g) { set_error("v or g is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, gradient_impl(c, reinterpret_cast<const float2*>(v), false,
                              reinterpret_cast<float2*>(g), E, Er, Ed));
}

int lddmm_hessian_matvec(lddmm_ctx* c, const float* v, const float* dv, float* Hdv) {
    if (!v || !dv || !Hdv) { set_error("v, dv or Hdv is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        const float2* vt = reinterpret_cast<const float2*>(v);
        bool same = false;
        TRY(same_as_current(c, vt, &same));
        if (!same) TRY(ensure_state(c, vt, false));
        return hessian_impl(c, reinterpret_cast<const float2*>(dv), reinterpret_cast<float2*>(Hdv));
    })());
}

int lddmm_register(lddmm_ctx* c, float* v_inout, const double* g_ref_norms, lddmm_report* rep) {
    if (!v_inout || !rep) { set_error("v_inout or report is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, register_impl(c, reinterpret_cast<float2*>(v_inout), g_ref_norms, rep));
}

int lddmm_get_history(lddmm_ctx* c, double* out, int cap, int* count) {
    if (!c) { set_error("context is NULL"); return LDDMM_EINVAL; }
    if (!count || cap < 0 || (cap > 0 && !out)) {
        set_error("get_history: null count, cap < 0, or null out with cap > 0");
        return LDDMM_EINVAL;
    }
    const int n = (int)c->hist.size();
    for (int i = 0; i < std::min(n, cap); ++i)
        for (int k = 0; k < 5; ++k) out[5 * i + k] = c->hist[i][k];
    *count = n;
    return LDDMM_OK;
}

int lddmm_jacobian_det(lddmm_ctx* c, const float* v, float* J, double* range) {
    if (!v || !range) { set_error("jacobian_det: v or range is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        if (!has_u(c)) {
            set_error("jacobian_det: deformation-state or state-equation contexts only");
            return LDDMM_EINVAL;
        }
        const float2* vt = reinterpret_cast<const float2*>(v);
        bool same = false;
        TRY(same_as_current(c, vt, &same));
        TRY(ensure_state(c, vt, same));
        TRY(ensure_traj(c));
        double* pmin = c->partials;
        double* pmax = c->partials + kReduceBlocks;
        TRY(jacobian_det(c->g, c->Du + (long)c->p.nt * 9 * c->n, J, pmin, pmax, c->st));
        std::vector<double> h(2 * kReduceBlocks);
        LDDMM_CUDA(cudaMemcpyAsync(h.data(), c->partials, h.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->st));
        LDDMM_CUDA(cudaStreamSynchronize(c->st));
        range[0] = *std::min_element(h.begin(), h.begin() + kReduceBlocks);
        range[1] = *std::max_element(h.begin() + kReduceBlocks, h.end());
        return LDDMM_OK;
    })());
}

int lddmm_max_displacement(lddmm_ctx* c, const float* v, double* vox) {
    if (!v || !vox) { set_error("max_displacement: v or vox is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        if (!has_u(c)) {
            set_error("max_displacement: deformation-state or state-equation contexts only");
            return LDDMM_EINVAL;
        }
        const float2* vt = reinterpret_cast<const float2*>(v);
        bool same = false;
        TRY(same_as_current(c, vt, &same));
        TRY(ensure_state(c, vt, same));
        // |phi(1)(x) - x| = |iota(u~(1))(x)|, in voxels per axis
        TRY(include(c, c->ut + (long)c->p.nt * 3 * c->kc, 3, c->fa, c->n, -1, 0));
        TRY(max_norm3(c->fa, c->n, c->to_vox, c->partials, c->dsc, c->st));
        TRY(read_scalars(c, 1));
        *vox = c->hsc[0];
        return LDDMM_OK;
    })());
}

int lddmm_get_warped(lddmm_ctx* c, float* m1) {
    if (!m1) { set_error("m1 is NULL"); return LDDMM_EINVAL; }
    CTX_CALL(c, ([&]() -> int {
        if (!c->vel_valid) { set_error("no state solved yet"); return LDDMM_EINVAL; }
        if (has_u(c)) TRY(data_term(c, nullptr));
        const float* src = has_u(c) ? c->m1 : c->ms + (long)c->p.nt * c->n;
        LDDMM_CUDA(cudaMemcpyAsync(m1, src, c->n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
        return LDDMM_OK;
    })());
}

}  // extern "C"

// ------------------------------------------------------------------ stand-alone operators
// Scratch comes from CUDA's stream-ordered pool and is released on the same stream.
struct PoolScratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit PoolScratch(cudaStream_t s) : st(s) {}
    ~PoolScratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <class T>
    int get(T** p, size_t count) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), st);
        if (e != cudaSuccess) {
            set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            *p = nullptr;
            return LDDMM_ENOMEM;
        }
        ptrs.push_back(*p);
        return LDDMM_OK;
    }
};

namespace lddmm {

int check_grid(int nx, int ny, int nz) {
    if (nx < 2 || ny < 2 || nz < 2 || nx > 1024 || ny > 1024 || nz > 4096) {
        set_error("grid must be 2..1024 (x, y) and 2..4096 (z) voxels per axis");
        return LDDMM_EINVAL;
    }
    if ((long)nx * ny * nz > 0x7fffffffL / 3) {
        set_error("grid too large: nx*ny*nz must stay below 2^31/3 voxels");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

// band accepted by the stand-alone spectral operators (the rule the partial-DFT stages
// apply), checked before any scratch is taken or any twiddle table is built
int check_band(int nx, int ny, int nz, int K) {
    if (K < 4 || (K & 1) || K > 64 || K > nx || K > ny || K > nz) {
        set_error("spectral: need even 4 <= K <= min(64, nx, ny, nz)");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

// precision forms accepted by the stand-alone spectral operators
int check_spectral_precision(int precision) {
    if (precision != LDDMM_PREC_FP32 && precision != LDDMM_PREC_BF16X3 &&
        precision != LDDMM_PREC_FP32_SIMT) {
        set_error("spectral precision must be LDDMM_PREC_FP32, LDDMM_PREC_BF16X3 or LDDMM_PREC_FP32_SIMT");
        return LDDMM_EINVAL;
    }
    return LDDMM_OK;
}

}  // namespace lddmm

extern "C" {

int lddmm_bl_project(int nx, int ny, int nz, int K, const float* f, int ncomp, float* c,
                     int precision, void* stream) {
    TRY(check_grid(nx, ny, nz));
    TRY(check_band(nx, ny, nz, K));
    TRY(check_spectral_precision(precision));
    if (!f || !c || ncomp < 1) { set_error("bl_project: null pointer or ncomp < 1"); return LDDMM_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Grid g{nx, ny, nz};
    PoolScratch ps(st);
    float* twm;
    float2 *s1, *s2;
    TRY(ps.get(&twm, twiddle_floats(g, K)));
    long se = spectral_scratch_elems(g, K, ncomp);
    TRY(ps.get(&s1, se));
    TRY(ps.get(&s2, se));
    Twiddles tw;
    TRY(twiddle_init(g, K, twm, tw, st));
    return bl_project(g, tw, f, g.ntot(), ncomp, reinterpret_cast<float2*>(c), s1, s2, precision, st);
}

int lddmm_bl_include(int nx, int ny, int nz, int K, const float* c, int ncomp, float* f,
                     int deriv_axis, int bspline, int precision, void* stream) {
    TRY(check_grid(nx, ny, nz));
    TRY(check_band(nx, ny, nz, K));
    TRY(check_spectral_precision(precision));
    if (!f || !c || ncomp < 1) { set_error("bl_include: null pointer or ncomp < 1"); return LDDMM_EINVAL; }
    if (deriv_axis < -1 || deriv_axis > 2) { set_error("bl_include: deriv_axis must be -1..2"); return LDDMM_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Grid g{nx, ny, nz};
    PoolScratch ps(st);
    float* twm;
    float2 *s1, *s2;
    TRY(ps.get(&twm, twiddle_floats(g, K)));
    long se = spectral_scratch_elems(g, K, ncomp);
    TRY(ps.get(&s1, se));
    TRY(ps.get(&s2, se));
    Twiddles tw;
    TRY(twiddle_init(g, K, twm, tw, st));
    return bl_include(g, tw, reinterpret_cast<const float2*>(c), ncomp, f, g.ntot(), deriv_axis,
                      bspline ? 1 : 0, s1, s2, precision, st);
}

int lddmm_sl_characteristics(int nx, int ny, int nz, const float* vel, double dt, int direction,
                             int interp, float* offsets, void* stream) {
    TRY(check_grid(nx, ny, nz));
    if (!vel || !offsets) { set_error("sl_characteristics: null pointer"); return LDDMM_EINVAL; }
    if (interp != 1 && interp != 3) { set_error("interp must be 1 or 3"); return LDDMM_EINVAL; }
    if (direction != 1 && direction != -1) { set_error("direction must be +1 or -1"); return LDDMM_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Grid g{nx, ny, nz};
    SLArgs a{g, interp};
    const float one[3] = {1.f, 1.f, 1.f};
    const float* vsrc = vel;
    PoolScratch ps(st);
    if (interp == 3) {
        float* vc;
        TRY(ps.get(&vc, 3 * g.ntot()));
        TRY(bspline_prefilter(g, vel, 3, vc, st));
        vsrc = vc;
    }
    return sl_characteristics(a, vsrc, vel, one, direction > 0 ? -dt : dt, offsets, st);
}

int lddmm_sl_transport(int nx, int ny, int nz, int nt, int interp, const float* vel,
                       const float* field, int ncomp, int direction, float* out, void* stream) {
    TRY(check_grid(nx, ny, nz));
    if (!vel || !field || !out || ncomp < 1) { set_error("sl_transport: null pointer or ncomp < 1"); return LDDMM_EINVAL; }
    if (nt < 1) { set_error("sl_transport: nt must be >= 1"); return LDDMM_EINVAL; }
    if (interp != 1 && interp != 3) { set_error("interp must be 1 or 3"); return LDDMM_EINVAL; }
    if (direction != 1 && direction != -1) { set_error("direction must be +1 or -1"); return LDDMM_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Grid g{nx, ny, nz};
    const long n = g.ntot();
    SLArgs a{g, interp};
    PoolScratch ps(st);
    float *D, *tmp, *coef = nullptr;
    TRY(ps.get(&D, 3 * n));
    TRY(ps.get(&tmp, (size_t)ncomp * n));
    const float one[3] = {1.f, 1.f, 1.f};
    const double dt = 1.0 / nt;
    const float* vsrc = vel;
    if (interp == 3) {
        TRY(ps.get(&coef, (size_t)std::max(ncomp, 3) * n));
        TRY(bspline_prefilter(g, vel, 3, coef, st));
        vsrc = coef;
    }
    TRY(sl_characteristics(a, vsrc, vel, one, direction > 0 ? -dt : dt, D, st));
    // ping-pong between out and tmp so that the last step lands in out
    const float* cur = field;
    for (int j = 0; j < nt; ++j) {
        const bool last_to_out = ((nt - 1 - j) % 2) == 0;
        float* dst = last_to_out ? out : tmp;
        const float* src = cur;
        if (interp == 3) {
            TRY(bspline_prefilter(g, cur, ncomp, coef, st));
            src = coef;
        } else if (src == dst) {
            LDDMM_CUDA(cudaMemcpyAsync(tmp == dst ? out : tmp, cur, (size_t)ncomp * n * sizeof(float),
                                       cudaMemcpyDeviceToDevice, st));
            src = tmp == dst ? out : tmp;
        }
        TRY(sl_gather(a, src, D, ncomp, dst, st));
        cur = dst;
    }
    return LDDMM_OK;
}


// ------------------------------------------------------------------ options, autotuning
int lddmm_set_option(lddmm_ctx* c, int option, long value) {
    int rc = check_ctx(c);
    if (rc) return rc;
    switch (option) {
        case LDDMM_OPT_GRAPHS:
            c->use_graphs = value != 0;
            return LDDMM_OK;
        case LDDMM_OPT_BLOCK_X: {
            if (value < 1 || value > 256 || 256 % value != 0) {
                set_error("block x must divide 256");
                return LDDMM_EINVAL;
            }
            c->sl.bx = (int)value;
            c->sl.by = 256 / (int)value;
            return LDDMM_OK;
        }
        case LDDMM_OPT_GATHER_ZT: {
            if (value < 0 || value > 16) {
                set_error("gather z planes per thread must be 0 (by grid size) .. 16");
                return LDDMM_EINVAL;
            }
            c->sl.zt = (int)value;
            return LDDMM_OK;
        }
        case LDDMM_OPT_TWO_LEVEL: {
            if (value < 0 || value > 1000) {
                set_error("two-level inner iterations must be 0 (off) .. 1000");
                return LDDMM_EINVAL;
            }
            if (value == 0) {
                lddmm_destroy(c->coarse);
                c->coarse = nullptr;
                c->tl_inner = 0;
                return LDDMM_OK;
            }
            if (!c->coarse) {
                rc = make_coarse(c);
                if (rc) return rc;
            }
            c->tl_inner = (int)value;
            return LDDMM_OK;
        }
        default:
            set_error("unknown option");
            return LDDMM_EINVAL;
    }
}

}  // extern "C"

namespace {

std::string tune_key(const lddmm_ctx* c) {
    return std::to_string(c->g.nx) + "x" + std::to_string(c->g.ny) + "x" + std::to_string(c->g.nz) +
           "/i" + std::to_string(c->p.interp);
}

// The cache is a flat JSON object {"<nx>x<ny>x<nz>/i<interp>": <block x>, ...}.
std::vector<std::pair<std::string, int>> read_tune_cache(const char* path) {
    std::vector<std::pair<std::string, int>> out;
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    fclose(f);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
        size_t end = text.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = text.substr(pos + 1, end - pos - 1);
        size_t colon = text.find(':', end);
        if (colon == std::string::npos) break;
        int v = atoi(text.c_str() + colon + 1);
        out.emplace_back(key, v);
        pos = colon + 1;
    }
    return out;
}

void write_tune_cache(const char* path, const std::vector<std::pair<std::string, int>>& kv) {
    FILE* f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{");
    for (size_t i = 0; i < kv.size(); ++i)
        fprintf(f, "%s\n \"%s\": %d", i ? "," : "", kv[i].first.c_str(), kv[i].second);
    fprintf(f, "\n}\n");
    fclose(f);
}

}  // namespace

extern "C" {

// Times the SL voxel kernels of this context's grid for each 256-thread block shape and
// keeps the fastest; with cache_path, reuses / records the choice there.
int lddmm_autotune(lddmm_ctx* c, const char* cache_path, int* block_x_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    const std::string key = tune_key(c);
    auto kv = read_tune_cache(cache_path);
    for (auto& e : kv)
        if (e.first == key && e.second > 0 && 256 % e.second == 0) {
            c->sl.bx = e.second;
            c->sl.by = 256 / e.second;
            if (block_x_out) *block_x_out = e.second;
            return LDDMM_OK;
        }
    // candidates; inputs are the context's own buffers (zeroed offsets: no data dependence
    // of the timing beyond the access pattern of a zero displacement)
    const int cand[] = {32, 64, 128, 256, 16};
    const long n = c->n;
    LDDMM_CUDA(cudaMemsetAsync(c->Df, 0, 3 * n * sizeof(float), c->st));
    cudaEvent_t e0, e1;
    LDDMM_CUDA(cudaEventCreate(&e0));
    LDDMM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_bx = c->sl.bx;
    for (int bx : cand) {
        SLArgs a = c->sl;
        a.bx = bx;
        a.by = 256 / bx;
        float tot = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            LDDMM_CUDA(cudaEventRecord(e0, c->st));
            rc = sl_gather_scale(a, c->fa, c->Df, c->gam, 3, c->fb, c->st);
            if (rc == LDDMM_OK && has_u(c) && c->Du)
                rc = sl_inc_defstate(a, c->fa, c->Df, c->fb, jac(c, 0, true), jac_bf16(c), c->dvsp, c->dt,
                                     c->fc, c->fd, c->st);
            LDDMM_CUDA(cudaEventRecord(e1, c->st));
            LDDMM_CUDA(cudaEventSynchronize(e1));
            if (rc) break;
            float ms = 0.f;
            LDDMM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;  // first repetition warms up
        }
        if (rc) break;
        if (tot < best) {
            best = tot;
            best_bx = bx;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return fail(c, rc);
    c->sl.bx = best_bx;
    c->sl.by = 256 / best_bx;
    c->vel_valid = c->traj_valid = c->warp_valid = false;  // the offsets were overwritten
    if (block_x_out) *block_x_out = best_bx;
    if (cache_path) {
        kv.emplace_back(key, best_bx);
        write_tune_cache(cache_path, kv);
    }
    return LDDMM_OK;
}

// ------------------------------------------------------------------ batched registration
int lddmm_register_batch(lddmm_ctx* const* ctxs, float* const* v_inout, int n,
                         const double* g_ref_norms, lddmm_report* reports, int max_threads) {
    if (n < 0 || (n > 0 && (!ctxs || !v_inout || !reports))) {
        set_error("register_batch: null arrays or n < 0");
        return LDDMM_EINVAL;
    }
    // one worker thread per pair owns its context (host fields, buffers, graph, stream): the
    // same context twice would be driven by two threads at once. Compared as pointers, before
    // any context is read (NULL entries are left to the context check below).
    if (n > 1) {
        std::vector<const lddmm_ctx*> sorted;
        for (int i = 0; i < n; ++i)
            if (ctxs[i]) sorted.push_back(ctxs[i]);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            set_error("register_batch: the same context appears more than once");
            return LDDMM_EINVAL;
        }
    }
    for (int i = 0; i < n; ++i) {
        int rc = check_ctx(ctxs[i]);
        if (rc) return rc;
        if (!v_inout[i]) {
            set_error("register_batch: null velocity");
            return LDDMM_EINVAL;
        }
    }
    if (n == 0) return LDDMM_OK;  // an empty batch: nothing to register, no device work
    int dev = 0;
    LDDMM_CUDA(cudaGetDevice(&dev));
    const int nthreads = std::max(1, std::min(n, max_threads > 0 ? max_threads : 8));
    std::atomic<int> next{0};
    std::atomic<int> first_rc{LDDMM_OK};
    std::string first_msg;
    std::mutex msg_mu;
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= n) break;
            lddmm_ctx* c = ctxs[i];
            const bool g = c->use_graphs;
            c->use_graphs = true;
            int rc = register_impl(c, reinterpret_cast<float2*>(v_inout[i]),
                                   g_ref_norms ? g_ref_norms + 2 * i : nullptr, &reports[i]);
            c->use_graphs = g;
            if (rc != LDDMM_OK) {
                fail(c, rc);
                int expect = LDDMM_OK;
                if (first_rc.compare_exchange_strong(expect, rc)) {
                    std::lock_guard<std::mutex> lk(msg_mu);
                    first_msg = "pair " + std::to_string(i) + ": " + g_last_error;
                }
            }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    if (first_rc.load() != LDDMM_OK) set_error(first_msg);
    return first_rc.load();
}

}  // extern "C"
