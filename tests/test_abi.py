"""The C-ABI library loads and exports every declared entry point; host-side argument
validation answers without touching a GPU."""
import ctypes

import pytest

import paper_2006_06823_b300 as L


def test_library_exports_every_declared_function():
    lib = L.load()
    names = L.header_functions()
    assert "lddmm_register" in names and "lddmm_bl_project" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_version_and_empty_error():
    lib = L.load()
    assert b"sm_103a" in lib.lddmm_version()
    assert isinstance(lib.lddmm_last_error(), bytes)


@pytest.mark.parametrize("field,value", [("K", 7), ("K", 2), ("K", 40), ("nt", 0),
                                         ("variant", 4), ("interp", 2), ("sigma2", 0.0),
                                         ("nx", 3), ("precision", 5), ("max_pcg", 0)])
def test_create_rejects_bad_parameters_before_any_device_work(field, value):
    lib = L.load()
    p = L.Params(32, 32, 32, 16, 10, L.V_DEFSTATE, L.INTERP_LINEAR, 0.0025, 2, 0.01, 5, 10,
                 1e-3, L.PREC_FP32)
    setattr(p, field, value)
    h = ctypes.c_void_p(123)
    rc = lib.lddmm_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == L.EINVAL
    assert h.value is None
    assert len(lib.lddmm_last_error()) > 0


def test_standalone_calls_reject_bad_shapes_before_any_device_work():
    lib = L.load()
    assert lib.lddmm_bl_project(1, 8, 8, 4, ctypes.c_void_p(16), 1, ctypes.c_void_p(16), 0, None) == L.EINVAL
    assert lib.lddmm_bl_include(8, 8, 8, 4, None, 1, None, -1, 0, 0, None) == L.EINVAL
    assert lib.lddmm_sl_transport(8, 8, 8, 0, 1, ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 1,
                                  ctypes.c_void_p(16), None) == L.EINVAL
    assert lib.lddmm_sl_characteristics(8, 8, 8, ctypes.c_void_p(16), 0.1, 2, 1,
                                        ctypes.c_void_p(16), None) == L.EINVAL
    assert lib.lddmm_destroy(None) == L.OK


@pytest.mark.parametrize("fn", ["lddmm_bl_project", "lddmm_bl_project_noalloc"])
def test_projections_reject_the_same_oversized_grid(fn):
    """1024^3 voxels exceed the 2^31/3 voxel limit of the projection; the allocation-free
    form would otherwise fit its scratch at K = 4, so both must return EINVAL before any
    device work (on a machine without a GPU any device call would give ECUDA instead)."""
    lib = L.load()
    p = ctypes.c_void_p(256)
    assert getattr(lib, fn)(1024, 1024, 1024, 4, p, 1, p, 0, None) == L.EINVAL
    assert b"too large" in lib.lddmm_last_error()


@pytest.mark.parametrize("K", [-2, 0, 2, 5, 66, 18])
def test_spectral_calls_reject_a_bad_band_before_any_device_work(K):
    """The band must be even with 4 <= K <= min(64, nx, ny, nz) (18 > 16 here): EINVAL from
    the projection, its allocation-free form and the inclusion before any scratch is taken
    (on a machine without a GPU any device call would give ECUDA or ENOMEM instead)."""
    lib = L.load()
    p = ctypes.c_void_p(256)
    assert lib.lddmm_bl_project(16, 16, 16, K, p, 1, p, 0, None) == L.EINVAL
    assert b"K" in lib.lddmm_last_error()
    assert lib.lddmm_bl_project_noalloc(16, 16, 16, K, p, 1, p, 0, None) == L.EINVAL
    assert lib.lddmm_bl_include(16, 16, 16, K, p, 1, p, -1, 0, 0, None) == L.EINVAL
    assert b"K" in lib.lddmm_last_error()


@pytest.mark.parametrize("prec", [3, 7, -1])
def test_standalone_spectral_calls_reject_unknown_precision(prec):
    """The stand-alone operators take FP32, BF16X3 or FP32_SIMT (BF16X3_JBF16 is a context
    form); anything else is EINVAL before any device work."""
    lib = L.load()
    p = ctypes.c_void_p(256)
    assert lib.lddmm_bl_project(16, 16, 16, 8, p, 1, p, prec, None) == L.EINVAL
    assert lib.lddmm_bl_include(16, 16, 16, 8, p, 1, p, -1, 0, prec, None) == L.EINVAL
    assert lib.lddmm_bl_project_noalloc(16, 16, 16, 8, p, 1, p, prec, None) == L.EINVAL
    assert b"precision" in lib.lddmm_last_error()


def test_register_batch_validates_its_arrays_and_accepts_an_empty_batch():
    """An empty batch is OK with no device work; a negative count, NULL arrays for a
    non-empty batch or a NULL context among them are EINVAL, all before any device call."""
    lib = L.load()
    P = ctypes.c_void_p
    assert lib.lddmm_register_batch(None, None, 0, None, None, 1) == L.OK
    assert lib.lddmm_register_batch(None, None, -1, None, None, 1) == L.EINVAL
    assert lib.lddmm_register_batch(None, None, 2, None, None, 1) == L.EINVAL
    arr = (P * 2)(None, None)
    reps = (L.Report * 2)()
    assert lib.lddmm_register_batch(arr, arr, 2, None, reps, 1) == L.EINVAL
    assert b"NULL" in lib.lddmm_last_error()


def test_register_batch_rejects_a_context_given_twice():
    """Each pair's context is driven by one worker thread; the same handle twice in one batch
    is EINVAL, decided on the pointers alone before any context is read or device call made
    (the fake handles here are never dereferenced)."""
    lib = L.load()
    P = ctypes.c_void_p
    a, b = P(0x1000), P(0x2000)
    ctxs = (P * 3)(a, b, a)
    vs = (P * 3)(P(256), P(512), P(768))
    reps = (L.Report * 3)()
    assert lib.lddmm_register_batch(ctxs, vs, 3, None, reps, 2) == L.EINVAL
    assert b"more than once" in lib.lddmm_last_error()


def test_null_context_is_rejected():
    lib = L.load()
    rep = L.Report()
    assert lib.lddmm_register(None, ctypes.c_void_p(16), None, ctypes.byref(rep)) == L.EINVAL
    assert lib.lddmm_objective(None, ctypes.c_void_p(16), None, None, None) == L.EINVAL


@pytest.mark.parametrize("D,c,B,st", [(48, 4, 1, 0), (4, 4, 1, 0), (256, 4, 1, 0), (64, 0, 1, 0),
                                      (64, 65, 1, 0), (64, 16, 0, 0), (64, 16, 65, 0),
                                      (64, 16, 8, 4), (64, 16, 8, -1)])
def test_net_create_rejects_bad_shapes_before_any_device_work(D, c, B, st):
    lib = L.load()
    h = ctypes.c_void_p(123)
    rc = lib.lddmm_net_create(D, c, B, st, 0, None, ctypes.byref(h))
    assert rc == L.EINVAL
    assert h.value is None
    assert b"net_create" in lib.lddmm_last_error()


def test_net_calls_reject_null_network():
    lib = L.load()
    assert lib.lddmm_net_forward(None, None, 1, None) == L.EINVAL
    assert lib.lddmm_net_train_step(None, None, None, 1, 1e-3, None) == L.EINVAL
    assert lib.lddmm_net_warm_start(None, 64, 64, 64, None, None, 32, None) == L.EINVAL
    assert lib.lddmm_net_num_params(None) == 0
    assert lib.lddmm_net_destroy(None) == L.OK


def test_nonstationary_flag_is_validated_before_any_device_work():
    lib = L.load()
    for variant, flag in ((L.V_IMAGE, 2), (L.V_STATE, -1), (L.V_DEFSTATE, 2)):
        p = L.Params(32, 32, 32, 16, 10, variant, L.INTERP_LINEAR, 0.0025, 2, 0.01, 5, 10,
                     1e-3, L.PREC_FP32, flag)
        h = ctypes.c_void_p(123)
        assert lib.lddmm_create(ctypes.byref(p), None, ctypes.byref(h)) == L.EINVAL
        assert b"nonstationary" in lib.lddmm_last_error() or b"non-stationary" in lib.lddmm_last_error()


def test_spatial_flag_is_validated_before_any_device_work():
    lib = L.load()
    for nx, spatial, nonst in ((32, 2, 0), (33, 1, 0), (32, -1, 1)):
        p = L.Params(nx, 32, 32, 16, 10, L.V_DEFSTATE, L.INTERP_LINEAR, 0.0025, 2, 0.01, 5, 10,
                     1e-3, L.PREC_FP32, nonst, spatial)
        h = ctypes.c_void_p(123)
        assert lib.lddmm_create(ctypes.byref(p), None, ctypes.byref(h)) == L.EINVAL
        assert h.value is None


def _header_text():
    import os
    return open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "include",
                             "lddmm.h")).read()


def test_report_struct_of_the_binding_follows_the_header():
    """lddmm_report is filled by the library through the binding's ctypes mirror: same fields,
    same order (the two-level preconditioner's pcg_inner_total last)."""
    import re
    text = _header_text()
    body = text[text.index("/* Outcome of lddmm_register. */"):text.index("} lddmm_report;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split("{", 1)[1].split(";"):
        decl = decl.strip()
        if decl:
            names += [n.strip() for n in decl.split(None, 1)[1].split(",")]
    assert names == [n for n, _ in L.Report._fields_]
    assert names[-1] == "pcg_inner_total"


def test_network_storage_codes_of_the_binding_follow_the_header():
    import re
    codes = dict(re.findall(r"LDDMM_NET_(\w+) = (\d+)", _header_text()))
    assert {k: int(v) for k, v in codes.items()} == {
        "BF16": L.NET_BF16, "FP32": L.NET_FP32, "BF16_SIMT": L.NET_BF16_SIMT,
        "FP32_TC": L.NET_FP32_TC}


def test_option_codes_of_the_binding_follow_the_header():
    import re
    text = _header_text()
    codes = dict(re.findall(r"LDDMM_OPT_(\w+) = (\d+)", text))
    assert {k: int(v) for k, v in codes.items()} == {
        "GRAPHS": L.OPT_GRAPHS, "BLOCK_X": L.OPT_BLOCK_X, "GATHER_ZT": L.OPT_GATHER_ZT,
        "TWO_LEVEL": L.OPT_TWO_LEVEL}


_SCALARS = {"int": ctypes.c_int, "long": ctypes.c_long, "long long": ctypes.c_longlong,
            "unsigned long long": ctypes.c_ulonglong, "double": ctypes.c_double,
            "float": ctypes.c_float, "char": ctypes.c_char}
_STRUCTS = {"lddmm_params": L.Params, "lddmm_report": L.Report}


def _header_prototypes():
    """(return type, name, [parameter types]) of every function declared in the header."""
    import re
    text = re.sub(r"/\*.*?\*/", "", _header_text(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = []
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(lddmm_[a-z_]+)\s*\(([^)]*)\)\s*;", text):
        params = [] if m.group(3).strip() == "void" else [
            re.sub(r"\b[A-Za-z_]\w*\s*$", "", p).strip() for p in m.group(3).split(",")]
        out.append((" ".join(m.group(1).split()), m.group(2), params))
    return out


def _type_matches(ctype_decl, t):
    """Whether the ctypes type t passes a C parameter of type ctype_decl without conversion
    loss: scalars exactly, pointers as c_void_p, c_char_p (char only) or a POINTER to the
    pointee's own type (c_void_p for a pointer to a pointer)."""
    stars = ctype_decl.count("*")
    base = " ".join(ctype_decl.replace("*", " ").replace("const", " ").split())
    if stars == 0:
        return t is _SCALARS[base]
    if t is ctypes.c_void_p:
        return True
    if t is ctypes.c_char_p:
        return base == "char" and stars == 1
    pointee = getattr(t, "_type_", None)
    if not isinstance(pointee, type):
        return False
    if stars >= 2:
        return pointee is ctypes.c_void_p
    return pointee is _SCALARS.get(base, _STRUCTS.get(base))


def test_binding_signatures_follow_the_header_prototypes():
    """Every declared function has a ctypes signature in the binding whose arity and argument
    types match the C prototype: an undeclared or mistyped argument would pass a truncated
    pointer or a misread scalar without any error."""
    lib = L.load()
    protos = _header_prototypes()
    assert sorted(n for _, n, _ in protos) == L.header_functions()
    bad = []
    for ret, name, params in protos:
        fn = getattr(lib, name)
        args = fn.argtypes
        if args is None or len(args) != len(params):
            bad.append((name, "arity", params, args))
            continue
        bad += [(name, i, p, a) for i, (p, a) in enumerate(zip(params, args))
                if not _type_matches(p, a)]
        if not _type_matches(ret, fn.restype):
            bad.append((name, "return", ret, fn.restype))
    assert bad == []


def test_signature_check_catches_a_mistyped_argument():
    """The comparison above is not vacuous: a double where the header has int, an int where
    it has a pointer and a pointer to the wrong struct are each rejected."""
    assert _type_matches("int", ctypes.c_int) and not _type_matches("int", ctypes.c_double)
    assert not _type_matches("const float*", ctypes.c_int)
    assert _type_matches("lddmm_report*", ctypes.POINTER(L.Report))
    assert not _type_matches("lddmm_report*", ctypes.POINTER(L.Params))
    assert _type_matches("lddmm_ctx**", ctypes.POINTER(ctypes.c_void_p))
    assert not _type_matches("double*", ctypes.POINTER(ctypes.c_int))


C_CONSUMER = r"""
#include <stdio.h>
#include "lddmm.h"
int main(void) {
    lddmm_params p = {0};
    p.nx = p.ny = p.nz = 32; p.K = 7; p.nt = 10; p.variant = LDDMM_V_DEFSTATE;
    p.interp = LDDMM_INTERP_LINEAR; p.alpha = 0.0025; p.s = 2; p.sigma2 = 0.01;
    p.max_gn = 5; p.max_pcg = 10; p.gtol = 1e-3;
    lddmm_ctx* c = (lddmm_ctx*)0x1;
    int rc = lddmm_create(&p, NULL, &c);
    printf("%s|%d|%d|%s\n", lddmm_version(), rc, c == NULL, lddmm_last_error());
    return rc == LDDMM_EINVAL && c == NULL ? 0 : 1;
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    """The boundary needs no C++ or Python: a C99 program (-pedantic, warnings as errors)
    includes include/lddmm.h, links liblddmm.so and gets EINVAL for an odd band before any
    device work."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")
    libdir = os.path.dirname(os.path.abspath(L.LIB_PATH))
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(root, "include"), str(src), "-L", libdir, "-llddmm",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    version, rc, null, msg = out.stdout.strip().split("|", 3)
    assert "sm_103a" in version and int(rc) == L.EINVAL and null == "1" and "band" in msg


def test_every_context_call_rejects_a_null_context_before_any_device_work():
    lib = L.load()
    p = ctypes.c_void_p(256)                 # never dereferenced: the context check comes first
    d = ctypes.c_double(0)
    rep = L.Report()
    calls = [
        lambda: lib.lddmm_set_images(None, p, p),
        lambda: lib.lddmm_set_images_host(None, p, p),
        lambda: lib.lddmm_objective(None, p, ctypes.byref(d), None, None),
        lambda: lib.lddmm_gradient(None, p, p, None, None, None),
        lambda: lib.lddmm_hessian_matvec(None, p, p, p),
        lambda: lib.lddmm_register(None, p, None, ctypes.byref(rep)),
        lambda: lib.lddmm_jacobian_det(None, p, None, ctypes.byref(d)),
        lambda: lib.lddmm_max_displacement(None, p, ctypes.byref(d)),
        lambda: lib.lddmm_get_warped(None, p),
        lambda: lib.lddmm_get_history(None, None, 0, ctypes.byref(ctypes.c_int(0))),
        lambda: lib.lddmm_set_option(None, L.OPT_TWO_LEVEL, 2),
        lambda: lib.lddmm_autotune(None, None, None),
    ]
    for call in calls:
        assert call() == L.EINVAL
        assert b"NULL" in lib.lddmm_last_error()
    ctxs = (ctypes.c_void_p * 1)(None)
    vs = (ctypes.c_void_p * 1)(p)
    reps = (L.Report * 1)()
    assert lib.lddmm_register_batch(ctxs, vs, 1, None, reps, 1) == L.EINVAL


def test_workspace_limit_gives_enomem_before_any_device_work():
    lib = L.load()
    p = L.Params(32, 32, 32, 16, 10, L.V_DEFSTATE, L.INTERP_LINEAR, 0.0025, 2, 0.01, 5, 10,
                 1e-3, L.PREC_FP32)
    h = ctypes.c_void_p(123)
    try:
        assert lib.lddmm_set_workspace_limit(1) == L.OK
        assert lib.lddmm_create(ctypes.byref(p), None, ctypes.byref(h)) == L.ENOMEM
        assert h.value is None
        assert b"workspace limit" in lib.lddmm_last_error()
    finally:
        lib.lddmm_set_workspace_limit(0)
    assert lib.lddmm_set_workspace_limit(-1) == L.EINVAL


@pytest.mark.parametrize("seconds", [0.0, -1.0, 1.5])
def test_wait_selftest_validates_its_bound_before_any_device_work(seconds):
    lib = L.load()
    st = ctypes.c_int(7)
    assert lib.lddmm_selftest_wait(seconds, ctypes.byref(st)) == L.EINVAL
    assert st.value == 7
    assert lib.lddmm_selftest_wait(0.01, None) == L.EINVAL


def test_binding_rejects_undersized_and_mismatched_tensors_before_calling_the_library():
    """The wrappers check every tensor's element count against what the C call reads or
    writes through its pointer (an undersized ``out`` would be overrun on the device). The
    check runs before the device check, so CPU tensors exercise it without a GPU."""
    import torch
    f = torch.zeros((1, 8, 8, 8))
    with pytest.raises(ValueError, match="bl_project: out"):
        L.bl_project(f, 4, out=torch.empty((1, 4, 4, 3), dtype=torch.complex64))
    with pytest.raises(ValueError, match="bl_project_noalloc: out"):
        L.bl_project_noalloc(f, 4, out=torch.empty((2, 4, 4), dtype=torch.complex64))
    with pytest.raises(ValueError, match="bl_include: c"):
        L.bl_include(torch.zeros((3, 4, 4, 2), dtype=torch.complex64), (8, 8, 8))
    with pytest.raises(ValueError, match="bl_include: out"):
        L.bl_include(torch.zeros((3, 4, 4, 4), dtype=torch.complex64), (8, 8, 8),
                     out=torch.empty((3, 8, 8, 7)))
    vel = torch.zeros((3, 8, 8, 8))
    with pytest.raises(ValueError, match="sl_characteristics: vel"):
        L.sl_characteristics(torch.zeros((2, 8, 8, 8)), 0.1)
    with pytest.raises(ValueError, match="sl_characteristics: out"):
        L.sl_characteristics(vel, 0.1, out=torch.empty((3, 8, 8)))
    with pytest.raises(ValueError, match="sl_transport: vel"):
        L.sl_transport(torch.zeros((3, 8, 8, 4)), f, 2)
    with pytest.raises(ValueError, match="sl_transport: out"):
        L.sl_transport(vel, torch.zeros((2, 8, 8, 8)), 2, out=torch.empty((1, 8, 8, 8)))
    with pytest.raises(ValueError, match="one velocity per context"):
        L.register_batch([object(), object()], [None])
    with pytest.raises(ValueError, match="norm pair per context"):
        L.register_batch([object()], [None], g_ref_norms=[(1.0,)])
    field = torch.zeros((8, 8, 8))
    with pytest.raises(ValueError, match="one field per velocity"):
        L.sl_transport_batch([vel, vel], [field], 2)
    with pytest.raises(ValueError, match="one output per velocity"):
        L.sl_transport_batch([vel, vel], [field, field], 2, outs=[field])
    with pytest.raises(ValueError, match="sl_transport_batch: velocity"):
        L.sl_transport_batch([torch.zeros((2, 8, 8, 8))], [field], 2)
    with pytest.raises(ValueError, match="sl_transport_batch: out"):
        L.sl_transport_batch([vel], [field], 2, outs=[torch.empty((8, 8, 7))])
    with pytest.raises(ValueError, match="sl_transport_bf16: out"):
        L.sl_transport_bf16(vel, field, 2, out=torch.empty((8, 8, 7)))
    # a context's velocity-shaped arguments: (nt + 1) cubes in the non-stationary form
    ctx = object.__new__(L.Context)
    ctx._vec_ptr, ctx._vec_len = L._c64, 5 * 3 * 4 ** 3
    with pytest.raises(ValueError, match="velocity-shaped"):
        ctx._vec(torch.zeros((3, 4, 4, 4), dtype=torch.complex64))
    # the right count reaches the device check (no GPU here)
    with pytest.raises(ValueError, match="CUDA tensor"):
        ctx._vec(torch.zeros((5, 3, 4, 4, 4), dtype=torch.complex64))
    ctx._h = None


def test_set_images_checks_both_images_against_the_grid():
    """Host images are copied by the library for nx*ny*nz floats each: a smaller array would
    be over-read on the host, so the binding refuses it; the right size reaches the library
    (here a NULL context, so EINVAL)."""
    import torch
    ctx = object.__new__(L.Context)
    ctx.shape, ctx._h = (4, 5, 6), None
    with pytest.raises(ValueError, match="set_images: I1"):
        ctx.set_images(torch.zeros((4, 5, 6)), torch.zeros((4, 5, 5)))
    with pytest.raises(ValueError, match="set_images: I0"):
        ctx.set_images(torch.zeros(100, dtype=torch.float64), torch.zeros((4, 5, 6)))
    with pytest.raises(L.LddmmError) as e:
        ctx.set_images(torch.zeros((4, 5, 6)), torch.zeros((4, 5, 6), dtype=torch.float64))
    assert e.value.code == L.EINVAL


def test_batched_transport_rejects_bad_arguments_before_any_device_work():
    lib = L.load()
    P = ctypes.c_void_p
    dims = (ctypes.c_int * 6)(16, 16, 16, 8, 8, 8)
    a, b, c = P(256), P(512), P(768)
    vel = (P * 2)(a, a)
    fld = (P * 2)(b, b)
    out = (P * 2)(c, P(1024))
    ok_args = dict(n=2, dims=dims, nt=4, direction=1, vel=vel, field=fld, out=out)

    def call(**kw):
        k = dict(ok_args, **kw)
        return lib.lddmm_sl_transport_batch(k["n"], k["dims"], k["nt"], k["direction"], k["vel"],
                                            k["field"], k["out"], None, kw.get("wait", 0.0), None)

    assert lib.lddmm_sl_transport_batch(0, None, 1, 1, None, None, None, None, 0.0, None) == L.OK
    assert call(n=-1) == L.EINVAL
    assert call(n=257) == L.EINVAL
    assert call(dims=None) == L.EINVAL
    assert call(nt=0) == L.EINVAL
    assert call(direction=0) == L.EINVAL
    assert call(wait=11.0) == L.EINVAL
    assert call(dims=(ctypes.c_int * 6)(16, 16, 16, 1, 8, 8)) == L.EINVAL     # a grid below 2
    assert call(out=(P * 2)(c, b)) == L.EINVAL                                # out = field
    assert b"same buffer" in lib.lddmm_last_error()
    assert call(vel=(P * 2)(a, None)) == L.EINVAL


def test_bf16_transport_rejects_bad_arguments_before_any_device_work():
    lib = L.load()
    p, q, r = ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(768)
    ok = (16, 16, 16, 4, p, q, 1, 1, r, None)
    for bad in [(1, 16, 16, 4, p, q, 1, 1, r, None), (16, 16, 16, 0, p, q, 1, 1, r, None),
                (16, 16, 16, 4, p, q, 0, 1, r, None), (16, 16, 16, 4, p, q, 1, 2, r, None),
                (16, 16, 16, 4, None, q, 1, 1, r, None), (16, 16, 16, 4, p, q, 1, 1, q, None)]:
        assert lib.lddmm_sl_transport_bf16(*bad) == L.EINVAL
    assert ok[5] != ok[8]
