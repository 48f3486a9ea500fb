/*
 * lddmm.h -- C ABI of the B300 (sm_103a) library for band-limited PDE-constrained LDDMM
 * with Gauss-Newton-Krylov optimisation and Semi-Lagrangian Runge-Kutta (SL-RK)
 * integration (arxiv 2006.06823).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Grid      nx, ny, nz voxels; scalar fields are float[nz][ny][nx] (x fastest); vector
 *            fields are float[3][nz][ny][nx] with component 0 = x, 1 = y, 2 = z.
 *  Domain    Omega = [0, 2 pi)^3, periodic; voxel j_a sits at x_a = 2 pi j_a / n_a.
 *  Band      K even, 4 <= K <= min(nx, ny, nz). Coefficient cubes are interleaved complex
 *            float[ncomp][K][K][K][2] indexed [comp][jz][jy][jx][re/im]; slot j holds
 *            wavenumber k = j - K/2. Slot j = 0 (k = -K/2) is always zero, so the retained
 *            set is S = {|k_a| <= K/2 - 1} (Sec. 2.2, truncated Fourier domain).
 *            Cubes describing real fields are Hermitian (c_{-k} = conj c_k); the library
 *            reads only the kx >= 0 half of an input cube and writes full, Hermitian cubes.
 *  pi / iota pi(f)_k = (1/N_tot) sum_x f(x) e^{-i k.x};  iota(c)(x) = sum_{k in S} c_k e^{i k.x}.
 *  Units     Band-limited velocities and displacements are physical (per [0, 2 pi)); spatial
 *            velocities handed to the SL entry points are in voxels per unit time.
 *  Pointers  Field and cube pointers are DEVICE pointers owned by the caller, unless a
 *            parameter says "host". The library owns only a context's workspace and the
 *            scratch of the stand-alone calls (taken from CUDA's stream-ordered pool).
 *  Streams   `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *            asynchronous on it, except those returning host scalars or reports, which
 *            synchronise that stream before returning.
 *  Errors    Every call returns an lddmm_status; nothing is thrown across the ABI. The
 *            message of the calling thread's most recent failure is in lddmm_last_error().
 *            A context records its first error and refuses further work (sticky).
 */
#ifndef LDDMM_H
#define LDDMM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDDMM_OK = 0,
    LDDMM_EINVAL = -1,      /* bad argument, shape or parameter */
    LDDMM_ENOMEM = -2,      /* device allocation failed or workspace cap exceeded */
    LDDMM_ECUDA = -3,       /* a CUDA runtime error (message kept) */
    LDDMM_ENONFINITE = -4,  /* NaN/Inf met in an energy or inner product */
    LDDMM_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
    LDDMM_ELINESEARCH = -6  /* no acceptable update length (returned in reports only) */
} lddmm_status;

/* Variant (Sec. 2.3). IMAGE: transported image m and adjoint lambda (Sec. 2.3.1).
 * STATE: m(t) = I0 o phi(t), lambda(t) = J(t) lambda(1) o psi(t) with phi = id - iota(u~)
 * from the deformation state equation and psi = id - iota(nu~), J = 1 - iota(U~) from two
 * backward equations (Sec. 2.3.2); gradient and Gauss-Newton Hessian of Eqs. 15-16 with
 * dlambda(t) = J(t) dlambda(1) o psi(t) (stationary velocity only). DEFSTATE: displacement
 * u~ and adjoint rho~ (Sec. 2.3.3). STATE and DEFSTATE share the energy (the same phi(1)). */
enum { LDDMM_V_IMAGE = 1, LDDMM_V_STATE = 2, LDDMM_V_DEFSTATE = 3 };
enum { LDDMM_INTERP_LINEAR = 1, LDDMM_INTERP_CUBIC = 3 };  /* Sec. 3.1, Sec. 4.2 */
/* Precision form. FP32: FP32-accurate results; the x stages of pi and iota run on the
 * tensor cores as split TF32 products (hi + lo, three products, FP32 accumulation) where the
 * shape allows (K a multiple of 16, nx a multiple of 4, nx <= 256 for iota), else as FP32
 * SIMT. BF16X3: split BF16 products (lower precision, stated error). FP32_SIMT: never the
 * tensor cores (the plain FP32 reference form). BF16X3_JBF16 (contexts only): BF16X3 plus
 * BF16 storage of the trajectory Jacobians D iota(u~_j) that the Gauss-Newton Hessian-vector
 * products read (halving their largest stream); the gradient keeps FP32 Jacobians. */
enum { LDDMM_PREC_FP32 = 0, LDDMM_PREC_BF16X3 = 1, LDDMM_PREC_FP32_SIMT = 2,
       LDDMM_PREC_BF16X3_JBF16 = 3 };
enum { LDDMM_FORWARD = 1, LDDMM_BACKWARD = -1 };           /* SL time direction */
enum { LDDMM_STOP_GTOL = 1, LDDMM_STOP_MAXIT = 2, LDDMM_STOP_LINESEARCH = 3 };

/* Problem parameters. Paper values (Sec. 4.3): alpha = 0.0025, s = 2, at most 10 Gauss-
 * Newton iterations with at most 5 PCG iterations, nt = 5 for SL-RK. */
typedef struct {
    int nx, ny, nz;    /* grid */
    int K;             /* band (cube edge), even */
    int nt;            /* time steps on [0, 1] */
    int variant;       /* LDDMM_V_IMAGE, LDDMM_V_STATE or LDDMM_V_DEFSTATE */
    int interp;        /* LDDMM_INTERP_LINEAR or LDDMM_INTERP_CUBIC */
    double alpha;      /* L = (Id - alpha Laplacian)^s, Eq. 1 */
    int s;
    double sigma2;     /* data weight 1/sigma^2 of Eq. 10 */
    int max_gn;        /* Gauss-Newton updates */
    int max_pcg;       /* PCG iterations per update */
    double gtol;       /* stop when ||g|| / ||g(v=0)|| <= gtol */
    int precision;     /* LDDMM_PREC_* form */
    int nonstationary; /* 0: one cube v~ for all t (the default); 1: v~_j at every node t_j =
                          j/nt (any variant, either domain). Every velocity argument of a
                          non-stationary context is then the stack float[nt+1][3][K][K][K][2];
                          norms and inner products of such stacks weight node j by the
                          trapezoid weight w_j (R11), and the gradient / Hessian at node j is
                          the integrand of Eq. 32 / 33 (15 / 16 for IMAGE and STATE) at t_j. */
    int spatial;       /* 0: band-limited (the default; Sec. 2.2-2.3). 1: spatial domain (Sec. 2.1
                          with SL-RK in Omega, the paper's "PDE-LDDMM ... SL" methods): every
                          velocity argument is a field float[3][nz][ny][nx] (physical
                          units); K is ignored, pi and iota are the identity, and L, L^{-1}
                          and the derivatives grad m,
                          D u, div v are spectral on the full grid (cuFFT). Inner products and
                          E_reg use the voxel mean. nx must be even. A non-stationary
                          spatial velocity is float[nt+1][3][nz][ny][nx]. */
} lddmm_params;

/* Outcome of lddmm_register. */
typedef struct {
    int gn_iters;         /* accepted Gauss-Newton updates */
    int pcg_iters_total;  /* Hessian-vector products spent in PCG */
    int stop_reason;      /* LDDMM_STOP_* */
    int solves;           /* PDE solves of nt steps (state, adjoint, incremental) */
    double E0, E, E_reg, E_data;   /* energy at v0 and at the result (Eq. 10) */
    double grad_rel_l2;   /* ||g(v)||_2 / ||g(0)||_2 at the result */
    double grad_rel_inf;  /* ||g(v)||_inf / ||g(0)||_inf (Sec. 5.1.1) */
    double mse_rel;       /* ||m(1) - I1||^2 / ||I0 - I1||^2 (Sec. 5.1.1) */
    double seconds;       /* wall time inside the call */
    int pcg_inner_total;  /* coarse-level Hessian-vector products of the two-level
                             preconditioner (LDDMM_OPT_TWO_LEVEL; 0 without it) */
} lddmm_report;

typedef struct lddmm_ctx lddmm_ctx;

/* ---------------------------------------------------------------- context lifecycle */

/* Validates *params, allocates the context's device workspace on the current device and
 * binds the context to `stream`. *out receives the handle (NULL on failure). The workspace
 * grows with nt: the stationary deformation-state form keeps, per voxel, 36 (nt + 1) bytes of
 * trajectory Jacobians and 12 (nt + 1) bytes of per-node adjoint values besides about 150
 * bytes of fields; lddmm_workspace_bytes reports a context's total.
 * Errors: EINVAL (shape, band, variant, interp, nt, sigma2 <= 0), ENOMEM, ECUDA. */
int lddmm_create(const lddmm_params* params, void* stream, lddmm_ctx** out);

/* Frees the workspace (after synchronising the context's stream). NULL is accepted. */
int lddmm_destroy(lddmm_ctx* ctx);

/* Copies the source image I0 (moving, m(0) = I0) and the target I1 (fixed) into the
 * context, device-to-device (float[nz][ny][nx] each). Eq. 10, Eq. 17. */
int lddmm_set_images(lddmm_ctx* ctx, const float* I0, const float* I1);

/* Same, from HOST buffers (pageable or pinned); the copies run on the context's stream. */
int lddmm_set_images_host(lddmm_ctx* ctx, const float* I0_host, const float* I1_host);

/* ------------------------------------------------------------------ the optimiser */

/* Energy of Eq. 10 at the band-limited velocity v (cube float[3][K][K][K][2]) under the
 * context's variant: solves the state equation (Eq. 17, or Eq. 34 for STATE and DEFSTATE). Writes host doubles
 * (any pointer may be NULL). Synchronises. */
int lddmm_objective(lddmm_ctx* ctx, const float* v, double* E, double* E_reg, double* E_data);

/* Gradient g~ at v (Eq. 15 for IMAGE and STATE, Eq. 32 for DEFSTATE) into g (device cube
 * float[3][K][K][K][2]); also leaves the state trajectory of v cached for
 * lddmm_hessian_matvec. Energies as in lddmm_objective (host, may be NULL). Synchronises. */
int lddmm_gradient(lddmm_ctx* ctx, const float* v, float* g, double* E, double* E_reg,
                   double* E_data);

/* Gauss-Newton Hessian-vector product H(v) dv (Eq. 16 for IMAGE and STATE, Eq. 33 read as
 * the Gauss-Newton operator for DEFSTATE) into Hdv (device cubes). Recomputes the state of
 * v when it is not the cached one. Asynchronous. */
int lddmm_hessian_matvec(lddmm_ctx* ctx, const float* v, const float* dv, float* Hdv);

/* Gauss-Newton-Krylov registration (Eqs. 13-14): v_inout (device cube) holds the
 * initial velocity (zeros for a cold start) and receives the result; PCG with
 * preconditioner L~^{-1}, Armijo update length, stop on grad ratio or max_gn.
 * g_ref_norms (host, may be NULL): {||g(0)||_2, ||g(0)||_inf} of the cold start, so that a
 * warm start is measured against the cold-start reference; NULL computes them here.
 * *report (host) receives the outcome. Synchronises. */
int lddmm_register(lddmm_ctx* ctx, float* v_inout, const double* g_ref_norms,
                   lddmm_report* report);

/* BF16-storage form of the scalar transport (the mixed-precision variant of the state sweep
 * D_t m = 0, Table 1 row 1; trilinear SL-RK, Sec. 3.1): the departure offsets are computed in
 * FP32 exactly as lddmm_sl_transport does, then stored in BF16 (offsets_bf16 = 1) or kept FP32
 * (0); the field is stored in BF16 between steps (rounded to nearest even after each step);
 * every interpolation is evaluated in FP32. vel: device [3][nz][ny][nx] in voxels per unit
 * time; field, out: device [nz][ny][nx] FP32 (out must not be field). Bytes per voxel-step 10
 * (BF16 offsets) or 16, against 20 for FP32 storage; the error against FP32 storage is that of
 * the BF16 roundings (about 2^-9 relative per step). Scratch from the stream-ordered pool;
 * asynchronous on stream. EINVAL before any device work for bad grids, NULL pointers, nt < 1,
 * a bad direction or flag, or field == out. */
int lddmm_sl_transport_bf16(int nx, int ny, int nz, int nt, const float* vel, const float* field,
                            int direction, int offsets_bf16, float* out, void* stream);

/* Persistent batched transport (the batched form; no counterpart in the paper's text): the
 * state sweep D_t m = 0 (Table 1 row 1; SL-RK characteristics Eqs. 40-42 with trilinear
 * interpolation, Sec. 3.1) of n independent pairs with their own grids, all in ONE cooperative
 * kernel launch: blocks take 256-voxel tiles from one work list spanning every active pair,
 * first the departure points of every pair, then nt steps, with a grid-wide barrier between
 * steps. Per pair p: dims[3p..3p+2] = (nx, ny, nz) (host array), vel[p] a device [3][nz][ny][nx]
 * velocity in voxels per unit time, field[p] the device [nz][ny][nx] field transported, out[p]
 * the device result (must not be field[p]); vel, field and out are host arrays of device
 * pointers. active: NULL (all pairs) or a device int[n], nonzero = transport this pair (the
 * others' out is left untouched; read once, synchronously, before the launch). direction +1
 * forward, -1 backward. Each pair's result equals lddmm_sl_transport(..., interp = 1, ...)
 * bit for bit. wait_seconds bounds every barrier wait (0: 1 s; at most 10 s); on expiry the
 * kernel records LDDMM_ETIMEOUT and returns, and so does this call (the outputs are then
 * incomplete; the device stays usable). A negative value -s is a self-test: the barrier
 * expects one block more than the launch has, so every wait runs out after s seconds.
 * Scratch (4 floats per voxel) comes from the stream-ordered pool. Synchronises. n = 0: OK
 * without device work; n < 0 or > 256, NULL arrays, bad grids (the stand-alone operators'
 * limits), nt < 1, a bad direction or field[p] == out[p]: EINVAL before any device work. */
int lddmm_sl_transport_batch(int n, const int* dims, int nt, int direction,
                             const float* const* vel, const float* const* field,
                             float* const* out, const int* active, double wait_seconds,
                             void* stream);

/* Convergence history of the last lddmm_register (or of this context's pair in
 * lddmm_register_batch): one record per Gauss-Newton iterate n = 0 .. gn_iters, five
 * doubles each: {seconds since the call began (host clock, read once the iterate's gradient
 * norm is on the host, i.e. after its device work finished), ||g_n||_2 / ||g_ref||_2 (the
 * residual of the stopping test, Sec. 4.3), E(v~_n), PCG iterations so far, PDE solves so
 * far}. The time-to-residual of a threshold is the first record at or below it. Writes
 * min(cap, available) records to out (host, 5 * cap doubles) and the number available to
 * *count (0 before the first registration). NULL ctx or count, cap < 0, or NULL out with
 * cap > 0: EINVAL. Host-only; never touches the device. */
int lddmm_get_history(lddmm_ctx* ctx, double* out, int cap, int* count);

/* Batched form (no counterpart in the paper's text; it serves many independent pairs).
 * Registers n pairs, each with its own context (created on the current device, ideally each
 * bound to its own stream so that their kernels overlap), from up to max_threads host
 * threads (<= 0: 8). Each pair runs lddmm_register with its Hessian-vector product captured
 * once into a CUDA graph and replayed for every PCG iteration. g_ref_norms: NULL or n pairs
 * of {||g(0)||_2, ||g(0)||_inf}. reports[i] receives pair i's outcome. Returns the first
 * failure (message names the pair); the other pairs still complete. Synchronises.
 * The n contexts must be distinct (each is driven by one thread at a time): a context that
 * appears twice is EINVAL before any device work.
 * n = 0 returns OK without touching the device; n < 0, or NULL arrays with n > 0, EINVAL. */
int lddmm_register_batch(lddmm_ctx* const* ctxs, float* const* v_inout, int n,
                         const double* g_ref_norms, lddmm_report* reports, int max_threads);

enum { LDDMM_OPT_GRAPHS = 1, LDDMM_OPT_BLOCK_X = 2, LDDMM_OPT_GATHER_ZT = 3,
       LDDMM_OPT_TWO_LEVEL = 4 };

/* Context options: LDDMM_OPT_GRAPHS (0/1) captures the PCG Hessian-vector product into a
 * CUDA graph on its second use and replays it (lddmm_register); LDDMM_OPT_BLOCK_X sets the
 * x extent of the 256-thread blocks of the SL voxel kernels (must divide 256);
 * LDDMM_OPT_GATHER_ZT (0..16) the number of consecutive z planes one thread of the
 * 3-component trilinear gathers and incremental deformation-state steps handles (1: one voxel
 * per thread; more: the next plane's offsets are loaded while the current taps are in
 * flight; 0, the default: 4 or 2 when the grid still fills the GPU, else 1). Results do not
 * depend on it. LDDMM_OPT_TWO_LEVEL (0..1000) replaces the preconditioner L~^{-1} of
 * lddmm_register's PCG by a two-level one (the multi-level preconditioner Secs. 6-7 name as
 * future work; value = the cap on its coarse PCG iterations per application, 0 = off): a
 * coarse context on the half grid with band Kc = 2 floor(K/4) and the images restricted
 * spectrally (modes with 2|k_a| < N_a/2 kept) solves H_c y = R r to relative tolerance 0.1
 * (R: the coefficients of the coarse band, H_c: its Gauss-Newton Hessian at R v~), and
 * P^{-1} r = E y + theta L~^{-1}(r - E R r), theta = <R r, y> / <R r, L~_c^{-1} R r>; the
 * outer PCG becomes flexible PCG. Needs a band-limited stationary context, K >= 8 and even
 * nx, ny, nz; the coarse context is allocated by this call (freed by value 0 or
 * lddmm_destroy) and its images follow lddmm_set_images. EINVAL for other values or
 * contexts; ENOMEM, ECUDA. */
int lddmm_set_option(lddmm_ctx* ctx, int option, long value);

/* Autotuner: times the SL voxel kernels of the context's grid for block shapes
 * 16x16, 32x8, 64x4, 128x2 and 256x1 and keeps the fastest (written to *block_x_out if not
 * NULL). cache_path (may be NULL): JSON object {"<nx>x<ny>x<nz>/i<interp>": block_x}; an
 * existing entry is used without timing, a new one is added. Overwrites the context's
 * departure offsets (the next objective/gradient recomputes them). Synchronises. */
int lddmm_autotune(lddmm_ctx* ctx, const char* cache_path, int* block_x_out);

/* Jacobian determinant of the deformation phi(1) = id - iota(u~(1)) for the velocity v
 * (device cube): J = det(I - D iota(u~(1))) per voxel (Sec. 5.1.1 reports its minimum and
 * maximum; J < 0 flags a fold). J: device float[nz][ny][nx] or NULL; range (host): {min J,
 * max J} over the volume. Solves the state for v unless it is the context's current one.
 * DEFSTATE and STATE contexts only (EINVAL for IMAGE). Synchronises. */
int lddmm_jacobian_det(lddmm_ctx* ctx, const float* v, float* J, double* range);

/* *vox = max over voxels of |phi(1)(x) - x| = |iota(u~(1))(x)| in voxels (per-axis voxel
 * units, FP64 reduction): the largest displacement of the deformation for the velocity v
 * (device, the context's velocity layout). Solves the state for v unless it is the context's
 * current one. DEFSTATE and STATE contexts only (EINVAL for IMAGE). Synchronises. */
int lddmm_max_displacement(lddmm_ctx* ctx, const float* v, double* vox);

/* Warp m(1) = I0 o phi(1) of the last state solved in the context into m1 (device,
 * float[nz][ny][nx]). DEFSTATE, STATE: phi(1) = id - iota(u~(1)); IMAGE: m(nt). */
int lddmm_get_warped(lddmm_ctx* ctx, float* m1);

/* ----------------------------------------------- stand-alone operators of the hot path */

/* pi: ncomp real fields f (float[ncomp][nz][ny][nx]) -> cubes c (float[ncomp][K][K][K][2]).
 * Sec. 2.2. precision: LDDMM_PREC_FP32 (FP32 arithmetic) or LDDMM_PREC_BF16X3 (tensor-core
 * split products, FP32 accumulation). Scratch from the stream-ordered pool.
 * Errors: EINVAL (shape, K, ncomp < 1), ENOMEM, ECUDA. */
int lddmm_bl_project(int nx, int ny, int nz, int K, const float* f, int ncomp, float* c,
                     int precision, void* stream);

/* lddmm_bl_project without any allocation. The paper has no counterpart: this exists for
 * callers that cannot let a library allocate device memory -- a host framework that owns
 * all device memory through its own pool, a service held to a memory budget reserved up
 * front, or a latency-critical loop that cannot afford the allocator. It computes what
 * lddmm_bl_project computes, with the same kernels, but its scratch is one fixed 24 MiB
 * device array inside the library (held by every GPU that loads the library until the
 * process exits) instead of the stream-ordered pool. It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 * Limit: the scratch needed, about ncomp * nz * max(ny, K) * K * 4 bytes plus the twiddle
 * tables, must fit in 24 MiB (3 components of 192 x 224 x 192 at K = 32 take about 19 MiB);
 * larger problems return EINVAL and should use lddmm_bl_project.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and caches it; make that first call before any stream
 * capture. All calls on a device share the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller. Arguments and errors as
 * lddmm_bl_project. */
int lddmm_bl_project_noalloc(int nx, int ny, int nz, int K, const float* f, int ncomp, float* c,
                             int precision, void* stream);

/* iota: cubes c (float[ncomp][K][K][K][2], Hermitian) -> real fields f.
 * deriv_axis = -1: iota(c); 0/1/2: iota(i k_axis c), the spectral derivative along x/y/z.
 * bspline = 1: iota(c / B^(k)) with B^(k) = prod_a (2 + cos(2 pi k_a / n_a)) / 3, i.e. the
 * periodic cubic B-spline coefficients of iota(c) (the prefilter of Sec. 4.2 done exactly in
 * Fourier). Sec. 2.2. Errors as lddmm_bl_project. */
int lddmm_bl_include(int nx, int ny, int nz, int K, const float* c, int ncomp, float* f,
                     int deriv_axis, int bspline, int precision, void* stream);

/* Departure-point offsets D = X - x (voxels, float[3][nz][ny][nx]) of one SL step of length
 * dt for the stationary voxel-unit velocity vel (float[3][nz][ny][nx]) by Eqs. 40-42:
 * direction FORWARD: X* = x - dt v, X = x - dt/2 (v(X*) + v); BACKWARD: the same along -v.
 * interp LINEAR or CUBIC (cubic prefilters vel internally). Errors: EINVAL, ENOMEM, ECUDA. */
int lddmm_sl_characteristics(int nx, int ny, int nz, const float* vel, double dt,
                             int direction, int interp, float* offsets, void* stream);

/* nt SL steps of D_t u = 0 (Table 1 row 1) for ncomp fields with the stationary voxel-unit
 * velocity vel: characteristics once (as above, dt = 1/nt), then u^{j+1} = u^j o X.
 * direction BACKWARD integrates -D_t u = 0 from t = 1 to 0. field and out are
 * float[ncomp][nz][ny][nx] and may alias. This is the unit of the voxel-steps/s figure.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int lddmm_sl_transport(int nx, int ny, int nz, int nt, int interp, const float* vel,
                       const float* field, int ncomp, int direction, float* out,
                       void* stream);

/* ------------------------------------------------------- learned Gauss-Newton warm start */
/* No counterpart in the paper (its solver always starts from v = 0). A 3-D convolutional
 * encoder-decoder maps the image pair, band-limited and resampled to D^3, to a velocity on
 * the (D/2)^3 grid; its band-limited projection is an initial velocity for lddmm_register,
 * which then finishes the registration and measures the prediction by its own residual.
 * Architecture (base c channels): D^3: conv 2->c, c->c; pool; (D/2)^3: c->2c, 2c->2c;
 * pool; (D/4)^3: 2c->4c, 4c->4c; pool; (D/8)^3: 4c->8c, 8c->8c; upsample; (D/4)^3:
 * [8c up | 4c skip] -> 4c, 4c->4c; upsample; (D/2)^3: [4c up | 2c skip] -> 2c, 2c->2c,
 * 2c->3. Convolutions 3x3x3 (zero padding, stride 1) with ReLU except the last; pooling is
 * the 2x2x2 mean; upsampling repeats each voxel 2x2x2. Weights and activations are stored
 * BF16 (LDDMM_NET_FP32: FP32), master weights, gradients and Adam moments FP32, all sums
 * accumulate in FP32.
 * Network tensors are device float arrays: input x [B][2][D][D][D] (channel 0 = I0, the
 * template, channel 1 = I1, the reference), output y [B][3][D/2][D/2][D/2] (physical
 * velocity components x, y, z). Parameters: one flat float vector, per convolution in
 * forward order its weights W[cout][cin][27] (tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)) then
 * its biases b[cout]. The network object owns all its device memory; calls run on its
 * stream, are not thread-safe on one object, and are asynchronous unless stated. */
typedef struct lddmm_net lddmm_net;

/* Storage of the network's weights and activations and the kernels of its convolutions.
 * LDDMM_NET_BF16 (the default form): BF16 storage; the 3x3x3 convolutions (forward, input
 * gradient, weight gradient) run on the tensor cores as implicit GEMMs (tcgen05 kind::tf32,
 * FP32 accumulation; BF16 operands enter exactly, FP32 gradients split hi + lo), except the
 * weight gradient of layers narrower than 32 voxels per axis (FP32 SIMT kernel).
 * LDDMM_NET_FP32: FP32 storage with the FP32 SIMT convolutions, the reference form for
 * checking the BF16 one. LDDMM_NET_BF16_SIMT: BF16 storage with the FP32 SIMT convolutions
 * (the reference for the tensor-core ones, which sum in another order). LDDMM_NET_FP32_TC:
 * FP32 storage with the tensor-core convolutions, every FP32 operand split hi + lo (products
 * within about 2^-21 relative of FP32's), to check those kernels against FP32 arithmetic. */
enum { LDDMM_NET_BF16 = 0, LDDMM_NET_FP32 = 1, LDDMM_NET_BF16_SIMT = 2, LDDMM_NET_FP32_TC = 3 };

/* D a power of two in 8..128, base_channels 1..64, batch_max 1..64 (largest B of later
 * calls), storage one of the four LDDMM_NET_* forms. Weights He-initialised (normal, std
 * sqrt(2 / (27 cin))) from `seed`, biases 0. Synchronises. Errors: EINVAL, ENOMEM, ECUDA. */
int lddmm_net_create(int D, int base_channels, int batch_max, int storage,
                     unsigned long long seed, void* stream, lddmm_net** out);
int lddmm_net_destroy(lddmm_net* net);
/* Length of the flat parameter vector (0 for NULL). */
long lddmm_net_num_params(const lddmm_net* net);
/* Copy the FP32 parameters to / from dst / src (host or device, num_params floats).
 * set_params also resets the Adam state. Both synchronise. */
int lddmm_net_get_params(lddmm_net* net, float* dst);
int lddmm_net_set_params(lddmm_net* net, const float* src);
/* y = net(x) for B samples (device pointers). Errors: EINVAL (B outside 1..batch_max,
 * NULL), ECUDA. */
int lddmm_net_forward(lddmm_net* net, const float* x, int B, float* y);
/* grads (device, num_params floats) = gradient of sum(dy * net(x)) over the parameters,
 * layout as the parameter vector. Errors as lddmm_net_forward. */
int lddmm_net_gradients(lddmm_net* net, const float* x, const float* dy, int B, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr > 0) on the mean squared
 * error mean((net(x) - target)^2) of B samples (target [B][3][D/2]^3, device). The loss of
 * the step's forward pass goes to *loss (host, FP64) if loss is not NULL, which
 * synchronises. Errors as lddmm_net_forward, EINVAL for lr <= 0. */
int lddmm_net_train_step(lddmm_net* net, const float* x, const float* target, int B, float lr,
                         double* loss);
/* Network input of one pair: x[c] = iota_{D^3}(pi_D(I_c)), each image (device,
 * float[nz][ny][nx], nx, ny, nz >= D) band-limited to D^3 modes and evaluated on the D^3
 * grid of the same domain (spectral resampling, Sec. 2.2 operators). x: device
 * float[2][D][D][D]. Errors: EINVAL, ENOMEM, ECUDA. */
int lddmm_net_input(lddmm_net* net, int nx, int ny, int nz, const float* I0, const float* I1,
                    float* x);
/* Warm start: vtilde (device cube float[3][K][K][K][2]) = pi_K(net(input(I0, I1))), the
 * exact band-limited projection of the predicted (D/2)^3 velocity (K <= D/2). Pass it as
 * the initial velocity of lddmm_register. Errors: EINVAL, ENOMEM, ECUDA. */
int lddmm_net_warm_start(lddmm_net* net, int nx, int ny, int nz, const float* I0,
                         const float* I1, int K, float* vtilde);

/* ---------------------------------------------------------------------- diagnostics */

/* Kernel tracing (no counterpart in the paper; profiling support). The library counts
 * every kernel it launches (process-wide, always on). With tracing enabled it also records
 * a CUDA event pair around each launch on the launch's stream, with the launch's
 * algorithmic bytes and flops; lddmm_trace_read synchronises those events and returns a
 * JSON object {kernel: {launches, ms, bytes, flops}} summed since the last reset into
 * buf (len bytes). With buf == NULL it returns the size needed; EINVAL if len is short. */
long lddmm_launch_count(void);
int lddmm_trace_enable(int on);
int lddmm_trace_reset(void);
int lddmm_trace_read(char* buf, int len);

/* Message of the calling thread's most recent failure ("" if none). Never NULL. */
const char* lddmm_last_error(void);

/* Reads and clears the device error word set by the library's kernels when a bounded
 * device-side wait gives up (*code = LDDMM_ETIMEOUT; 0 if none). Synchronises the device. */
int lddmm_device_error(int* code);

/* Self-test of the device-side wait bound: a one-thread kernel waits, through the routine the
 * tensor-core kernels use, on an mbarrier phase that nothing completes, with the bound set to
 * `seconds`; it gives up, records LDDMM_ETIMEOUT in the device error word (see
 * lddmm_device_error) and returns, and *status receives LDDMM_ETIMEOUT. The wait is bounded by
 * %globaltimer and by an iteration count: no fault, trap or hang, and the CUDA context stays
 * usable. Synchronises. EINVAL unless 0 < seconds <= 1 and status != NULL. */
int lddmm_selftest_wait(double seconds, int* status);

/* Caps the device memory that each context may allocate for its workspace (bytes, process-
 * wide, applies to contexts created afterwards and to later allocations of existing ones,
 * e.g. the coarse context of LDDMM_OPT_TWO_LEVEL, which counts on its own; 0 = no cap, the
 * default). An allocation beyond the cap fails with LDDMM_ENOMEM before calling cudaMalloc
 * (lddmm_create then frees what it holds). cuFFT's plan work areas are not counted. EINVAL for
 * a negative value. */
int lddmm_set_workspace_limit(long long bytes);

/* *bytes = the device bytes the context's workspace holds (its own allocations). */
int lddmm_workspace_bytes(lddmm_ctx* ctx, long long* bytes);

/* Library version string, e.g. "lddmm-b300 0.1 sm_103a". */
const char* lddmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LDDMM_H */
