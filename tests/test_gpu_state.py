"""GPU parity of the state-equation variant (Sec. 2.3.2: m = I0 o phi, lambda = J lambda(1) o psi)
against the FP64 oracle, through the C ABI (lddmm_create with LDDMM_V_STATE)."""
import numpy as np
import pytest

from oracle import gnk
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def devc(c):
    return torch.as_tensor(np.ascontiguousarray(c).astype(np.complex64), device="cuda")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def gpu_context(prob, variant=None, **kw):
    nz, ny, nx = prob.shape
    p = prob.p
    ctx = L.Context(nx, ny, nz, p.K, nt=p.nt, variant=variant or p.variant, interp=p.order,
                    alpha=p.alpha, s=p.s, sigma2=p.sigma2, **kw)
    ctx.set_images(dev(prob.I0), dev(prob.I1))
    return ctx


CASES = [((16, 16, 16), 8, 1), ((16, 16, 16), 8, 3), ((20, 24, 28), 10, 1),
         # K = 16 with nx = 32: the x stages of pi and iota run on the tensor cores
         ((24, 20, 32), 16, 1), ((24, 20, 32), 16, 3)]


@pytest.mark.parametrize("shape,K,order", CASES)
def test_objective_gradient_hessian_match_oracle(shape, K, order):
    prob = oracle_problem(shape, K, Vn.STATE, order, nt=5)
    vt = synth.random_velocity_coeffs(K, K, seed=3) * 0.5
    E, Er, Ed, g = prob.gradient(vt)
    dv = synth.random_coeffs(K, seed=4) * 0.1
    Hdv = prob.hessian_matvec(vt, dv)
    with gpu_context(prob) as ctx:
        Eg, Erg, Edg = ctx.objective(devc(vt))
        assert Eg == pytest.approx(E, rel=1e-5)
        assert Erg == pytest.approx(Er, rel=1e-6)
        (E2, _, _), gg = ctx.gradient(devc(vt))
        assert E2 == pytest.approx(E, rel=1e-5)
        assert rel_l2(host(gg), g) < 1e-4
        Hg = ctx.hessian_matvec(devc(vt), devc(dv))
        assert rel_l2(host(Hg), Hdv) < 1e-4


def test_bf16_jacobian_form_against_oracle():
    """LDDMM_PREC_BF16X3_JBF16: the incremental deformation state of the Hessian reads BF16
    Jacobians (relative error <= 2^-9 per entry): bound 1e-2, as for the deformation state."""
    prob = oracle_problem((20, 24, 28), 10, Vn.STATE, 1, nt=5)
    vt = synth.random_velocity_coeffs(10, 10, seed=3) * 0.5
    E, Er, Ed, g = prob.gradient(vt)
    dv = synth.random_coeffs(10, seed=4) * 0.1
    Hdv = prob.hessian_matvec(vt, dv)
    with gpu_context(prob, precision=L.PREC_BF16X3_JBF16) as ctx:
        (E2, _, _), gg = ctx.gradient(devc(vt))
        assert E2 == pytest.approx(E, rel=1e-4)
        assert rel_l2(host(gg), g) < 1e-3
        err = rel_l2(host(ctx.hessian_matvec(devc(vt), devc(dv))), Hdv)
        assert 0 < err < 1e-2, err


def test_shares_the_energy_and_the_jacobian_with_the_deformation_state():
    prob = oracle_problem((20, 24, 28), 10, Vn.STATE, 1, nt=5)
    vt = devc(synth.random_velocity_coeffs(10, 10, seed=5))
    with gpu_context(prob) as cs, gpu_context(prob, variant=L.V_DEFSTATE) as cd:
        assert cs.objective(vt) == cd.objective(vt)             # same kernels, same phi(1)
        rs, Js = cs.jacobian_det(vt, field=True)
        rd, Jd = cd.jacobian_det(vt, field=True)
        assert rs == rd and torch.equal(Js, Jd)
        m_s, m_d = torch.empty_like(Js), torch.empty_like(Jd)
        cs.get_warped(m_s)
        cd.get_warped(m_d)
        assert torch.equal(m_s, m_d)


def test_zero_velocity_gradient_is_the_image_variant_gradient():
    # v = 0: phi = psi = id, J = 1, so lambda(t) = lambda(1) and m(t) = I0 in both variants
    prob = oracle_problem((24, 20, 32), 16, Vn.STATE, 1, nt=5)
    z = devc(np.zeros((3, 16, 16, 16), complex))
    with gpu_context(prob) as cs, gpu_context(prob, variant=L.V_IMAGE) as ci:
        gs = host(cs.gradient(z)[1])
        gi = host(ci.gradient(z)[1])
    assert rel_l2(gs, gi) < 1e-5


def test_hessian_recomputes_state_for_a_new_velocity():
    prob = oracle_problem((16, 16, 16), 8, Vn.STATE, 3, nt=4)
    v1 = synth.random_velocity_coeffs(8, 8, seed=5) * 0.5
    v2 = synth.random_velocity_coeffs(8, 8, seed=6) * 0.5
    dv = synth.random_coeffs(8, seed=7) * 0.1
    with gpu_context(prob) as ctx:
        ctx.gradient(devc(v1))
        H = ctx.hessian_matvec(devc(v2), devc(dv))
    assert rel_l2(host(H), prob.hessian_matvec(v2, dv)) < 1e-4


@pytest.mark.parametrize("order", [1, 3])
def test_live_registration_matches_oracle(order):
    prob = oracle_problem((16, 16, 16), 8, Vn.STATE, order, nt=5)
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=5)
    with gpu_context(prob, max_gn=3, max_pcg=5) as ctx:
        v, rep = ctx.register()
    assert rep["gn_iters"] == rep_o.gn_iters
    assert rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
    assert rep["mse_rel"] == pytest.approx(rep_o.mse_rel, rel=1e-3)
    assert rel_l2(host(v), v_o) < 1e-3


def test_graph_replayed_hessian_matches_eager():
    prob = oracle_problem((24, 20, 32), 16, Vn.STATE, 1, nt=5)
    with gpu_context(prob, max_gn=2, max_pcg=6) as ca, gpu_context(prob, max_gn=2, max_pcg=6) as cb:
        cb.set_option(L.OPT_GRAPHS, 1)
        va, ra = ca.register()
        vb, rb = cb.register()
    assert ra["pcg_iters_total"] == rb["pcg_iters_total"]
    assert rel_l2(host(vb), host(va)) < 1e-6


def test_full_size_state_variant_properties():
    """192 x 224 x 192, K = 32, nt = 10: energies shared with the deformation state, the v = 0
    gradient equal to the image variant's, and two Gauss-Newton updates lower the energy."""
    shape = (192, 224, 192)
    nz, ny, nx = shape
    I1 = synth.gaussian_blobs_device(shape, 0, "cuda")
    vt = synth.random_velocity_coeffs(32, 8, seed=1)
    v = L.bl_include(devc(vt), shape)
    V = v * (torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1)
             / (2 * np.pi))
    V *= 4.0 / V.pow(2).sum(0).sqrt().max()
    I0 = L.sl_transport(V, I1, 10, L.FORWARD, L.INTERP_LINEAR)
    kw = dict(nt=10, interp=L.INTERP_LINEAR, max_gn=2, max_pcg=5, gtol=0.0)
    z = torch.zeros((3, 32, 32, 32), dtype=torch.complex64, device="cuda")
    with L.Context(nx, ny, nz, 32, variant=L.V_STATE, **kw) as cs, \
            L.Context(nx, ny, nz, 32, variant=L.V_IMAGE, **kw) as ci:
        cs.set_images(I0, I1)
        ci.set_images(I0, I1)
        assert rel_l2(host(cs.gradient(z)[1]), host(ci.gradient(z)[1])) < 2e-5
        v, rep = cs.register()
    assert rep["gn_iters"] == 2 and rep["E"] < 0.9 * rep["E0"]
    assert np.isfinite(host(v)).all()
