"""GPU parity of the non-stationary forms (velocity per node) of the three variants against
the FP64 oracle (oracle/variants.py: ProblemNS), through the C ABI."""
import numpy as np
import pytest

from oracle import gnk
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import blob_pair, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def devc(c):
    return torch.as_tensor(np.ascontiguousarray(c).astype(np.complex64), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def problem(shape, K, order, nt, variant=Vn.DEFSTATE):
    I0, I1 = blob_pair(shape, K, seed=0, order=order)
    p = Vn.Params(K=K, nt=nt, order=order, variant=variant)
    return Vn.ProblemNS(I0, I1, p), Vn.Problem(I0, I1, p)


def context(prob, **kw):
    nz, ny, nx = prob.shape
    p = prob.p
    ctx = L.Context(nx, ny, nz, p.K, nt=p.nt, variant=p.variant, interp=p.order, alpha=p.alpha,
                    s=p.s, sigma2=p.sigma2, nonstationary=True, **kw)
    ctx.set_images(torch.as_tensor(prob.I0, dtype=torch.float32, device="cuda"),
                   torch.as_tensor(prob.I1, dtype=torch.float32, device="cuda"))
    return ctx


def stack(K, nt, seed, scale):
    return np.stack([synth.random_velocity_coeffs(K, K, seed=seed + j) * scale for j in range(nt + 1)])


CASES = [((16, 16, 16), 8, 1), ((16, 16, 16), 8, 3), ((24, 20, 32), 16, 1)]


@pytest.mark.parametrize("variant", [Vn.DEFSTATE, Vn.IMAGE, Vn.STATE])
@pytest.mark.parametrize("shape,K,order", CASES)
def test_objective_gradient_hessian_match_oracle(shape, K, order, variant):
    nt = 4
    prob, _ = problem(shape, K, order, nt, variant)
    vts = stack(K, nt, 3, 0.4)
    dvs = stack(K, nt, 40, 0.05)
    E, Er, Ed, g = prob.gradient(vts)
    H = prob.hessian_matvec(vts, dvs)
    with context(prob) as ctx:
        Eg, Erg, _ = ctx.objective(devc(vts))
        assert Eg == pytest.approx(E, rel=1e-5) and Erg == pytest.approx(Er, rel=1e-6)
        (E2, _, _), gg = ctx.gradient(devc(vts))
        assert E2 == pytest.approx(E, rel=1e-5)
        assert rel_l2(host(gg), g) < 1e-4
        Hg = ctx.hessian_matvec(devc(vts), devc(dvs))
        assert rel_l2(host(Hg), H) < 1e-4


@pytest.mark.parametrize("variant", [Vn.DEFSTATE, Vn.IMAGE, Vn.STATE])
def test_equal_nodes_reproduce_the_stationary_context(variant):
    """All nodes equal: same energy, and the weighted sum of the node gradients is the
    stationary gradient (GPU against GPU)."""
    shape, K, nt = (16, 16, 16), 8, 4
    prob, st = problem(shape, K, 1, nt, variant)
    vt = synth.random_velocity_coeffs(K, K, seed=7) * 0.5
    w = Vn.trapezoid_weights(nt)
    with context(prob) as ctx:
        (En, _, _), gn = ctx.gradient(devc(np.stack([vt] * (nt + 1))))
        gn = host(gn)
    nz, ny, nx = shape
    with L.Context(nx, ny, nz, K, nt=nt, variant=variant, interp=1) as cs:
        cs.set_images(torch.as_tensor(st.I0, dtype=torch.float32, device="cuda"),
                      torch.as_tensor(st.I1, dtype=torch.float32, device="cuda"))
        (Es, _, _), gs = cs.gradient(devc(vt))
        gs = host(gs)
    assert En == pytest.approx(Es, rel=1e-6)
    assert rel_l2(sum(wj * gj for wj, gj in zip(w, gn)), gs) < 1e-5


@pytest.mark.parametrize("variant", [Vn.DEFSTATE, Vn.IMAGE, Vn.STATE])
def test_registration_matches_oracle(variant):
    prob, _ = problem((16, 16, 16), 8, 1, 4, variant)
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=5)
    with context(prob, max_gn=3, max_pcg=5) as ctx:
        v, rep = ctx.register()
    assert v.shape == (5, 3, 8, 8, 8)
    assert rep["gn_iters"] == rep_o.gn_iters
    assert rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
    assert rel_l2(host(v), v_o) < 1e-3


def test_nonstationary_flag_must_be_zero_or_one():
    p = L.Params(16, 16, 16, 8, 4, L.V_IMAGE, L.INTERP_LINEAR, 0.0025, 2, 0.01, 5, 10, 1e-3,
                 L.PREC_FP32, 3, 0)
    import ctypes
    h = ctypes.c_void_p()
    assert L.load().lddmm_create(ctypes.byref(p), None, ctypes.byref(h)) == L.EINVAL
