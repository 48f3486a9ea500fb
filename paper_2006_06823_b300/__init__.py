"""B300 (sm_103a) band-limited PDE-constrained LDDMM with SL-RK integration.

Thin Python binding of the C ABI declared in ``include/lddmm.h`` (``liblddmm.so``, built
in-tree by ``python -m paper_2006_06823_b300.build``). Every function here only marshals
arguments: tensors are passed as device pointers with the current torch CUDA stream, and
all arithmetic runs in the library's CUDA kernels. There is no CPU fallback: if the
library is missing, the first call raises.

Names follow the C entry points without their ``lddmm_`` prefix:
``bl_project``, ``bl_include``, ``sl_characteristics``, ``sl_transport``,
``sl_transport_bf16``, ``sl_transport_batch``, ``register_batch``,
``device_error``, ``selftest_wait``, ``set_workspace_limit``, the context methods
``set_images``, ``objective``, ``gradient``, ``hessian_matvec``, ``register``,
``get_warped``, ``history``, ``jacobian_det``, ``max_displacement``, ``set_option``, ``autotune``,
``workspace_bytes``, and the warm-start network ``Net``.

Conventions (see the header): images float32 ``[nz, ny, nx]``; vector fields float32
``[3, nz, ny, nx]`` (component 0 = x); band-limited cubes complex64 ``[C, K, K, K]``
indexed ``[comp, jz, jy, jx]`` with wavenumber ``k = j - K/2``.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblddmm.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "lddmm.h")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ELINESEARCH = 0, -1, -2, -3, -4, -5, -6
V_IMAGE, V_STATE, V_DEFSTATE = 1, 2, 3
INTERP_LINEAR, INTERP_CUBIC = 1, 3
PREC_FP32, PREC_BF16X3, PREC_FP32_SIMT, PREC_BF16X3_JBF16 = 0, 1, 2, 3
FORWARD, BACKWARD = 1, -1
STOP_GTOL, STOP_MAXIT, STOP_LINESEARCH = 1, 2, 3
OPT_GRAPHS, OPT_BLOCK_X, OPT_GATHER_ZT, OPT_TWO_LEVEL = 1, 2, 3, 4
NET_BF16, NET_FP32, NET_BF16_SIMT, NET_FP32_TC = 0, 1, 2, 3


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("K", ctypes.c_int), ("nt", ctypes.c_int), ("variant", ctypes.c_int),
                ("interp", ctypes.c_int), ("alpha", ctypes.c_double), ("s", ctypes.c_int),
                ("sigma2", ctypes.c_double), ("max_gn", ctypes.c_int),
                ("max_pcg", ctypes.c_int), ("gtol", ctypes.c_double),
                ("precision", ctypes.c_int), ("nonstationary", ctypes.c_int),
                ("spatial", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int), ("pcg_iters_total", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("solves", ctypes.c_int),
                ("E0", ctypes.c_double), ("E", ctypes.c_double), ("E_reg", ctypes.c_double),
                ("E_data", ctypes.c_double), ("grad_rel_l2", ctypes.c_double),
                ("grad_rel_inf", ctypes.c_double), ("mse_rel", ctypes.c_double),
                ("seconds", ctypes.c_double), ("pcg_inner_total", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LddmmError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"lddmm error {code}: {message}")
        self.code = code


_lib = None
_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double


def _declare(lib):
    sig = {
        "lddmm_create": (_I, [ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
        "lddmm_destroy": (_I, [_P]),
        "lddmm_set_images": (_I, [_P, _P, _P]),
        "lddmm_set_images_host": (_I, [_P, _P, _P]),
        "lddmm_objective": (_I, [_P, _P, _P, _P, _P]),
        "lddmm_gradient": (_I, [_P, _P, _P, _P, _P, _P]),
        "lddmm_hessian_matvec": (_I, [_P, _P, _P, _P]),
        "lddmm_register": (_I, [_P, _P, _P, ctypes.POINTER(Report)]),
        "lddmm_get_warped": (_I, [_P, _P]),
        "lddmm_jacobian_det": (_I, [_P, _P, _P, ctypes.POINTER(_D)]),
        "lddmm_get_history": (_I, [_P, ctypes.POINTER(_D), _I, ctypes.POINTER(_I)]),
        "lddmm_max_displacement": (_I, [_P, _P, ctypes.POINTER(_D)]),
        "lddmm_bl_project": (_I, [_I, _I, _I, _I, _P, _I, _P, _I, _P]),
        "lddmm_bl_project_noalloc": (_I, [_I, _I, _I, _I, _P, _I, _P, _I, _P]),
        "lddmm_bl_include": (_I, [_I, _I, _I, _I, _P, _I, _P, _I, _I, _I, _P]),
        "lddmm_sl_characteristics": (_I, [_I, _I, _I, _P, _D, _I, _I, _P, _P]),
        "lddmm_sl_transport": (_I, [_I, _I, _I, _I, _I, _P, _P, _I, _I, _P, _P]),
        "lddmm_sl_transport_bf16": (_I, [_I, _I, _I, _I, _P, _P, _I, _I, _P, _P]),
        "lddmm_sl_transport_batch": (_I, [_I, ctypes.POINTER(_I), _I, _I, ctypes.POINTER(_P),
                                          ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _D, _P]),
        "lddmm_register_batch": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P,
                                      ctypes.POINTER(Report), _I]),
        "lddmm_set_option": (_I, [_P, _I, ctypes.c_long]),
        "lddmm_autotune": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_I)]),
        "lddmm_net_create": (_I, [_I, _I, _I, _I, ctypes.c_ulonglong, _P, ctypes.POINTER(_P)]),
        "lddmm_net_destroy": (_I, [_P]),
        "lddmm_net_num_params": (ctypes.c_long, [_P]),
        "lddmm_net_get_params": (_I, [_P, _P]),
        "lddmm_net_set_params": (_I, [_P, _P]),
        "lddmm_net_forward": (_I, [_P, _P, _I, _P]),
        "lddmm_net_gradients": (_I, [_P, _P, _P, _I, _P]),
        "lddmm_net_train_step": (_I, [_P, _P, _P, _I, ctypes.c_float,
                                      ctypes.POINTER(_D)]),
        "lddmm_net_input": (_I, [_P, _I, _I, _I, _P, _P, _P]),
        "lddmm_net_warm_start": (_I, [_P, _I, _I, _I, _P, _P, _I, _P]),
        "lddmm_launch_count": (ctypes.c_long, []),
        "lddmm_trace_enable": (_I, [_I]),
        "lddmm_trace_reset": (_I, []),
        "lddmm_trace_read": (_I, [ctypes.c_char_p, _I]),
        "lddmm_device_error": (_I, [ctypes.POINTER(_I)]),
        "lddmm_selftest_wait": (_I, [_D, ctypes.POINTER(_I)]),
        "lddmm_set_workspace_limit": (_I, [ctypes.c_longlong]),
        "lddmm_workspace_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
        "lddmm_last_error": (ctypes.c_char_p, []),
        "lddmm_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def load():
    """Loads ``liblddmm.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2006_06823_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        _declare(lib)
        _lib = lib
    return _lib


def header_functions():
    """Names of the functions declared in include/lddmm.h."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lddmm_[a-z_]+)\s*\(", text)))


def _check(rc):
    if rc != 0:
        raise LddmmError(rc, load().lddmm_last_error().decode())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    # the library launches on the current device's stream (and the projection's scratch and
    # tensor maps belong to that device): a tensor of another device would be a peer pointer
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"tensor on {t.device}, but the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t):
    import torch
    return _ptr(t, torch.float32)


def _sized(t, numel, name):
    """t after checking that it holds exactly ``numel`` elements: the C call reads or writes
    that many through its pointer, so a smaller tensor would be overrun on the device."""
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()} "
                         f"(shape {tuple(t.shape)})")
    return t


def _c64(t):
    import torch
    return _ptr(t, torch.complex64)


# ------------------------------------------------------------------ stand-alone operators

def bl_project(f, K, precision=PREC_FP32, out=None):
    """pi (Sec. 2.2): real fields ``[C, nz, ny, nx]`` -> Hermitian cubes ``[C, K, K, K]``."""
    import torch
    if f.dim() == 3:
        f = f.unsqueeze(0)
    C, nz, ny, nx = f.shape
    if out is None:
        out = torch.empty((C, K, K, K), dtype=torch.complex64, device=f.device)
    _sized(out, C * K ** 3, "bl_project: out")
    _check(load().lddmm_bl_project(nx, ny, nz, K, _f32(f), C, _c64(out), precision, _stream()))
    return out


def bl_project_noalloc(f, K, out, precision=PREC_FP32):
    """pi without allocations inside the library (lddmm_bl_project_noalloc): for callers
    that cannot let the library allocate device memory. ``out`` must be given; the
    library's fixed 24 MiB scratch bounds the problem size, and concurrent calls race."""
    if f.dim() == 3:
        f = f.unsqueeze(0)
    C, nz, ny, nx = f.shape
    _sized(out, C * K ** 3, "bl_project_noalloc: out")
    _check(load().lddmm_bl_project_noalloc(nx, ny, nz, K, _f32(f), C, _c64(out), precision,
                                           _stream()))
    return out


def bl_include(c, shape, deriv_axis=-1, bspline=False, precision=PREC_FP32, out=None):
    """iota (Sec. 2.2): cubes ``[C, K, K, K]`` -> real fields ``[C, nz, ny, nx]``.

    deriv_axis 0/1/2 synthesises the spectral derivative along x/y/z; bspline=True the
    periodic cubic B-spline coefficients of the field.
    """
    import torch
    if c.dim() == 3:
        c = c.unsqueeze(0)
    C, K = c.shape[0], c.shape[-1]
    nz, ny, nx = shape
    if out is None:
        out = torch.empty((C, nz, ny, nx), dtype=torch.float32, device=c.device)
    _sized(c, C * K ** 3, "bl_include: c")
    _sized(out, C * nz * ny * nx, "bl_include: out")
    _check(load().lddmm_bl_include(nx, ny, nz, K, _c64(c), C, _f32(out), deriv_axis,
                                   1 if bspline else 0, precision, _stream()))
    return out


def sl_characteristics(vel, dt, direction=FORWARD, interp=INTERP_LINEAR, out=None):
    """Departure offsets (voxels) of one SL step for a voxel-unit velocity (Eqs. 40-42)."""
    import torch
    _, nz, ny, nx = vel.shape
    if out is None:
        out = torch.empty_like(vel)
    _sized(vel, 3 * nz * ny * nx, "sl_characteristics: vel")
    _sized(out, 3 * nz * ny * nx, "sl_characteristics: out")
    _check(load().lddmm_sl_characteristics(nx, ny, nz, _f32(vel), float(dt), direction, interp,
                                           _f32(out), _stream()))
    return out


def sl_transport(vel, field, nt, direction=FORWARD, interp=INTERP_LINEAR, out=None):
    """nt SL steps of D_t u = 0 (Table 1 row 1) for fields ``[C, nz, ny, nx]``."""
    import torch
    squeeze = field.dim() == 3
    if squeeze:
        field = field.unsqueeze(0)
    C, nz, ny, nx = field.shape
    if out is None:
        out = torch.empty_like(field)
    _sized(vel, 3 * nz * ny * nx, "sl_transport: vel")
    _sized(out, C * nz * ny * nx, "sl_transport: out")
    _check(load().lddmm_sl_transport(nx, ny, nz, nt, interp, _f32(vel), _f32(field), C,
                                     direction, _f32(out), _stream()))
    return out[0] if squeeze else out


# ------------------------------------------------------------------ the optimiser

class Context:
    """One registration problem on the current CUDA device and stream (lddmm_create)."""

    def __init__(self, nx, ny, nz, K, nt=10, variant=V_DEFSTATE, interp=INTERP_LINEAR,
                 alpha=0.0025, s=2, sigma2=0.01, max_gn=10, max_pcg=20, gtol=1e-3,
                 precision=PREC_FP32, nonstationary=False, spatial=False):
        self.params = Params(nx, ny, nz, K, nt, variant, interp, alpha, s, sigma2, max_gn,
                             max_pcg, gtol, precision, 1 if nonstationary else 0,
                             1 if spatial else 0)
        self.shape = (nz, ny, nx)
        self.K = K
        self.nt = nt
        self.nonstationary = bool(nonstationary)
        self.spatial = bool(spatial)
        # velocity-shaped arguments: complex64 cubes, or float32 fields in the spatial form,
        # (nt + 1) of them in the non-stationary form
        self._vec_ptr = _f32 if spatial else _c64
        self._vec_len = ((nt + 1) if nonstationary else 1) * 3 * (
            nx * ny * nz if spatial else K ** 3)
        self._h = ctypes.c_void_p()
        _check(load().lddmm_create(ctypes.byref(self.params), _stream(), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            load().lddmm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _vec(self, t):
        return self._vec_ptr(_sized(t, self._vec_len, "velocity-shaped argument"))

    def _field(self, t, name):
        nz, ny, nx = self.shape
        return _f32(_sized(t, nx * ny * nz, name))

    def zeros_cube(self):
        """A zero velocity: [3, K, K, K] complex64 ([3, nz, ny, nx] float32 in the spatial
        form), with a leading nt + 1 for a non-stationary context."""
        import torch
        lead = (self.nt + 1, 3) if self.nonstationary else (3,)
        if self.spatial:
            return torch.zeros(lead + self.shape, dtype=torch.float32, device="cuda")
        return torch.zeros(lead + (self.K, self.K, self.K), dtype=torch.complex64, device="cuda")

    def set_images(self, I0, I1):
        if I0.is_cuda:
            _check(load().lddmm_set_images(self._h, self._field(I0, "set_images: I0"),
                                           self._field(I1, "set_images: I1")))
        else:
            import torch
            nz, ny, nx = self.shape
            a = _sized(I0.to(torch.float32).contiguous(), nx * ny * nz, "set_images: I0")
            b = _sized(I1.to(torch.float32).contiguous(), nx * ny * nz, "set_images: I1")
            _check(load().lddmm_set_images_host(self._h, ctypes.c_void_p(a.data_ptr()),
                                                ctypes.c_void_p(b.data_ptr())))

    def objective(self, v):
        E, Er, Ed = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().lddmm_objective(self._h, self._vec(v), ctypes.byref(E), ctypes.byref(Er),
                                      ctypes.byref(Ed)))
        return E.value, Er.value, Ed.value

    def gradient(self, v, out=None):
        import torch
        g = torch.empty_like(v) if out is None else out
        E, Er, Ed = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().lddmm_gradient(self._h, self._vec(v), self._vec(g), ctypes.byref(E),
                                     ctypes.byref(Er), ctypes.byref(Ed)))
        return (E.value, Er.value, Ed.value), g

    def hessian_matvec(self, v, dv, out=None):
        import torch
        h = torch.empty_like(dv) if out is None else out
        _check(load().lddmm_hessian_matvec(self._h, self._vec(v), self._vec(dv), self._vec(h)))
        return h

    def register(self, v=None, g_ref_norms=None):
        """GN-Krylov registration; v (complex64 [3,K,K,K], device) is updated in place."""
        v = self.zeros_cube() if v is None else v
        rep = Report()
        ref = None
        if g_ref_norms is not None:
            ref = (ctypes.c_double * 2)(*g_ref_norms)
        _check(load().lddmm_register(self._h, self._vec(v), ref, ctypes.byref(rep)))
        return v, rep.as_dict()

    def history(self):
        """Convergence history of the last registration (lddmm_get_history): a list of dicts
        per Gauss-Newton iterate with ``t`` (seconds since the call began), ``residual``
        (||g||_2 / ||g_ref||_2), ``E``, ``pcg`` and ``solves`` (cumulative)."""
        n = ctypes.c_int(0)
        _check(load().lddmm_get_history(self._h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_double * (5 * max(n.value, 1)))()
        _check(load().lddmm_get_history(self._h, buf, n.value, ctypes.byref(n)))
        keys = ("t", "residual", "E", "pcg", "solves")
        return [{k: buf[5 * i + j] for j, k in enumerate(keys)} for i in range(n.value)]

    def set_option(self, option, value):
        _check(load().lddmm_set_option(self._h, option, int(value)))

    def workspace_bytes(self):
        """Device bytes of the context's own workspace (lddmm_workspace_bytes)."""
        b = ctypes.c_longlong(0)
        _check(load().lddmm_workspace_bytes(self._h, ctypes.byref(b)))
        return b.value

    def autotune(self, cache_path=None):
        """Picks the fastest SL voxel-kernel block shape for this grid (lddmm_autotune)."""
        bx = ctypes.c_int(0)
        path = cache_path.encode() if cache_path else None
        _check(load().lddmm_autotune(self._h, path, ctypes.byref(bx)))
        return bx.value

    def jacobian_det(self, v, out=None, field=False):
        """(min J, max J) of J = det D phi(1) for velocity v (lddmm_jacobian_det); with
        field=True also the per-voxel J (float32 [nz, ny, nx])."""
        import torch
        J = None
        if field:
            J = torch.empty(self.shape, dtype=torch.float32, device="cuda") if out is None else out
        rng = (ctypes.c_double * 2)()
        _check(load().lddmm_jacobian_det(self._h, self._vec(v),
                                         self._field(J, "jacobian_det: out") if J is not None else None,
                                         rng))
        return (rng[0], rng[1]), J

    def max_displacement(self, v):
        """max |phi(1)(x) - x| in voxels for velocity v (lddmm_max_displacement)."""
        d = ctypes.c_double(0)
        _check(load().lddmm_max_displacement(self._h, self._vec(v), ctypes.byref(d)))
        return d.value

    def get_warped(self, out=None):
        import torch
        m = torch.empty(self.shape, dtype=torch.float32, device="cuda") if out is None else out
        _check(load().lddmm_get_warped(self._h, self._field(m, "get_warped: out")))
        return m


def sl_transport_bf16(vel, field, nt, direction=FORWARD, offsets_bf16=True, out=None):
    """Scalar SL transport with BF16 storage of the field between steps (and of the departure
    offsets with ``offsets_bf16``), FP32 arithmetic (lddmm_sl_transport_bf16)."""
    import torch
    nz, ny, nx = field.shape
    if out is None:
        out = torch.empty_like(field)
    _sized(vel, 3 * field.numel(), "sl_transport_bf16: velocity")
    _sized(out, field.numel(), "sl_transport_bf16: out")
    _check(load().lddmm_sl_transport_bf16(nx, ny, nz, nt, _f32(vel), _f32(field), direction,
                                          1 if offsets_bf16 else 0, _f32(out), _stream()))
    return out


def sl_transport_batch(vels, fields, nt, direction=FORWARD, outs=None, active=None,
                       wait_seconds=0.0):
    """Scalar SL transport of many pairs of different grids in one persistent launch
    (lddmm_sl_transport_batch): vels[p] float32 [3, nz, ny, nx] (voxel units), fields[p]
    float32 [nz, ny, nx]; returns the transported fields. ``active`` (int32 device tensor
    [n], optional) selects the pairs to transport."""
    import torch
    n = len(vels)
    if len(fields) != n:
        raise ValueError("sl_transport_batch: one field per velocity")
    if outs is None:
        outs = [torch.empty_like(f) for f in fields]
    if len(outs) != n:
        raise ValueError("sl_transport_batch: one output per velocity")
    dims = (ctypes.c_int * (3 * max(n, 1)))()
    vp, fp, op = ((_P * max(n, 1))() for _ in range(3))
    for v, f, o in zip(vels, fields, outs):   # every size before any device check
        _sized(v, 3 * f.numel(), "sl_transport_batch: velocity")
        _sized(o, f.numel(), "sl_transport_batch: out")
    for p, (v, f, o) in enumerate(zip(vels, fields, outs)):
        nz, ny, nx = f.shape
        dims[3 * p], dims[3 * p + 1], dims[3 * p + 2] = nx, ny, nz
        vp[p], fp[p], op[p] = _f32(v).value, _f32(f).value, _f32(o).value
    act = None
    if active is not None:
        act = _ptr(_sized(active, n, "sl_transport_batch: active"), torch.int32)
    _check(load().lddmm_sl_transport_batch(n, dims, nt, direction, vp, fp, op, act,
                                           float(wait_seconds), _stream()))
    return outs


# ------------------------------------------------------------------ learned warm start

class Net:
    """The warm-start encoder-decoder (lddmm_net_*): input ``[B, 2, D, D, D]`` float32
    (template, reference), output ``[B, 3, D/2, D/2, D/2]`` float32 velocity. Runs on the
    torch CUDA stream current at construction."""

    def __init__(self, D=64, base_channels=16, batch_max=8, seed=0, storage=NET_BF16):
        import torch
        self.D, self.c, self.batch_max, self.storage = D, base_channels, batch_max, storage
        self._stream = torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        _check(load().lddmm_net_create(D, base_channels, batch_max, storage, seed,
                                       ctypes.c_void_p(self._stream.cuda_stream),
                                       ctypes.byref(self._h)))
        self.num_params = int(load().lddmm_net_num_params(self._h))

    def close(self):
        if self._h:
            load().lddmm_net_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import torch
        p = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _check(load().lddmm_net_get_params(self._h, _f32(p)))
        return p

    def set_params(self, p):
        import torch
        p = torch.as_tensor(p, dtype=torch.float32).contiguous()
        if p.numel() != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {p.numel()}")
        _check(load().lddmm_net_set_params(self._h, ctypes.c_void_p(p.data_ptr())))

    def forward(self, x, out=None):
        import torch
        B, d = x.shape[0], self.D // 2
        y = torch.empty((B, 3, d, d, d), dtype=torch.float32, device=x.device) if out is None else out
        _sized(x, B * 2 * self.D ** 3, "net forward: x")
        _sized(y, B * 3 * d ** 3, "net forward: out")
        _check(load().lddmm_net_forward(self._h, _f32(x), B, _f32(y)))
        return y

    def gradients(self, x, dy, out=None):
        import torch
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device) if out is None else out
        B, d = x.shape[0], self.D // 2
        _sized(x, B * 2 * self.D ** 3, "net gradients: x")
        _sized(dy, B * 3 * d ** 3, "net gradients: dy")
        _sized(g, self.num_params, "net gradients: out")
        _check(load().lddmm_net_gradients(self._h, _f32(x), _f32(dy), x.shape[0], _f32(g)))
        return g

    def train_step(self, x, target, lr, want_loss=True):
        loss = ctypes.c_double(0.0)
        B, d = x.shape[0], self.D // 2
        _sized(x, B * 2 * self.D ** 3, "net train_step: x")
        _sized(target, B * 3 * d ** 3, "net train_step: target")
        _check(load().lddmm_net_train_step(self._h, _f32(x), _f32(target), x.shape[0],
                                           float(lr), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def input(self, I0, I1, out=None):
        import torch
        nz, ny, nx = I0.shape
        x = torch.empty((2, self.D, self.D, self.D), dtype=torch.float32, device=I0.device) \
            if out is None else out
        _sized(I1, nx * ny * nz, "net input: I1")
        _sized(x, 2 * self.D ** 3, "net input: out")
        _check(load().lddmm_net_input(self._h, nx, ny, nz, _f32(I0), _f32(I1), _f32(x)))
        return x

    def warm_start(self, I0, I1, K, out=None):
        import torch
        nz, ny, nx = I0.shape
        v = torch.empty((3, K, K, K), dtype=torch.complex64, device=I0.device) \
            if out is None else out
        _sized(I1, nx * ny * nz, "net warm_start: I1")
        _sized(v, 3 * K ** 3, "net warm_start: out")
        _check(load().lddmm_net_warm_start(self._h, nx, ny, nz, _f32(I0), _f32(I1), K, _c64(v)))
        return v


# ------------------------------------------------------------------ tracing

def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(load().lddmm_launch_count())


def trace_enable(on=True):
    _check(load().lddmm_trace_enable(1 if on else 0))


def trace_reset():
    _check(load().lddmm_trace_reset())


def trace_read():
    """Per-kernel {launches, ms, bytes, flops} since the last reset (synchronises)."""
    import json
    lib = load()
    size = lib.lddmm_trace_read(None, 0)
    buf = ctypes.create_string_buffer(size + 64)
    _check(lib.lddmm_trace_read(buf, size + 64))
    return json.loads(buf.value.decode())


def device_error():
    """Reads and clears the library's device error word (0 if no bounded wait gave up)."""
    code = ctypes.c_int(0)
    _check(load().lddmm_device_error(ctypes.byref(code)))
    return code.value


def selftest_wait(seconds):
    """Runs the bounded-wait self-test (lddmm_selftest_wait): a device wait that nothing
    completes gives up after `seconds`; returns the status it reported (ETIMEOUT)."""
    status = ctypes.c_int(0)
    _check(load().lddmm_selftest_wait(float(seconds), ctypes.byref(status)))
    return status.value


def set_workspace_limit(nbytes):
    """Caps the device bytes each context may allocate (0: no cap; lddmm_set_workspace_limit)."""
    _check(load().lddmm_set_workspace_limit(int(nbytes)))


def register_batch(contexts, velocities, g_ref_norms=None, max_threads=8):
    """Registers many pairs concurrently (lddmm_register_batch). ``contexts``: Context objects
    (each best created under its own torch CUDA stream); ``velocities``: complex64
    [3, K, K, K] device cubes updated in place. Returns the list of report dicts."""
    n = len(contexts)
    if len(velocities) != n:
        raise ValueError("register_batch: one velocity per context")
    if g_ref_norms is not None and (len(g_ref_norms) != n or any(len(p) != 2 for p in g_ref_norms)):
        raise ValueError("register_batch: g_ref_norms needs one (l2, inf) norm pair per context")
    hs = (_P * n)(*[c._h for c in contexts])
    vs = (_P * n)(*[ctypes.c_void_p(c._vec(v).value) for c, v in zip(contexts, velocities)])
    reps = (Report * n)()
    ref = None
    if g_ref_norms is not None:
        flat = [float(x) for pair in g_ref_norms for x in pair]
        ref = (ctypes.c_double * (2 * n))(*flat)
    _check(load().lddmm_register_batch(hs, vs, n, ref, reps, max_threads))
    return [r.as_dict() for r in reps]

