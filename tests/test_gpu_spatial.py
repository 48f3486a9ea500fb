"""GPU parity of the spatial-domain variants (Sec. 2.1 with SL-RK in Omega: velocity on the
grid, spectral derivatives and L on the full grid) against the FP64 oracle, through the C ABI
(lddmm_params.spatial = 1)."""
import numpy as np
import pytest

from oracle import gnk
from oracle import spatial as Sp
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import blob_pair, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def spatial_problem(shape, variant, order, nt=5, seed=0):
    I0, I1 = blob_pair(shape, 8, seed=seed, order=order)
    return Sp.SpatialProblem(I0, I1, Vn.Params(K=0, nt=nt, order=order, variant=variant,
                                               sigma2=0.01))


def field(shape, seed, scale):
    """A smooth velocity-shaped field: iota of random low-frequency coefficients."""
    return S.include(synth.random_velocity_coeffs(8, 8, seed), shape) * scale


def gpu_context(prob, **kw):
    nz, ny, nx = prob.shape
    p = prob.p
    ctx = L.Context(nx, ny, nz, 0, nt=p.nt, variant=p.variant, interp=p.order, alpha=p.alpha,
                    s=p.s, sigma2=p.sigma2, spatial=True, **kw)
    ctx.set_images(dev(prob.I0), dev(prob.I1))
    return ctx


CASES = [((16, 16, 16), Vn.DEFSTATE, 1), ((16, 16, 16), Vn.DEFSTATE, 3),
         ((16, 16, 16), Vn.IMAGE, 1), ((16, 16, 16), Vn.IMAGE, 3),
         ((16, 16, 16), Vn.STATE, 1), ((16, 16, 16), Vn.STATE, 3),
         ((20, 24, 28), Vn.DEFSTATE, 1), ((20, 24, 28), Vn.IMAGE, 1), ((20, 24, 28), Vn.STATE, 1),
         ((21, 18, 32), Vn.DEFSTATE, 3)]


@pytest.mark.parametrize("shape,variant,order", CASES)
def test_objective_gradient_hessian_match_oracle(shape, variant, order):
    prob = spatial_problem(shape, variant, order)
    v = field(shape, 3, 1.0)
    v *= 2.0 / np.abs(v * prob.tv).max()
    dv = field(shape, 4, 0.1)
    E, Er, Ed, g = prob.gradient(v)
    Hdv = prob.hessian_matvec(v, dv)
    with gpu_context(prob) as ctx:
        Eg, Erg, Edg = ctx.objective(dev(v))
        assert Eg == pytest.approx(E, rel=1e-5)
        assert Erg == pytest.approx(Er, rel=1e-5)
        (E2, _, _), gg = ctx.gradient(dev(v))
        assert E2 == pytest.approx(E, rel=1e-5)
        assert rel_l2(host(gg), g) < 1e-4
        Hg = ctx.hessian_matvec(dev(v), dev(dv))
        assert rel_l2(host(Hg), Hdv) < 1e-4


@pytest.mark.parametrize("variant,order", [(Vn.DEFSTATE, 1), (Vn.IMAGE, 3), (Vn.STATE, 1)])
def test_live_registration_matches_oracle(variant, order):
    prob = spatial_problem((16, 16, 16), variant, order)
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=5)
    with gpu_context(prob, max_gn=3, max_pcg=5) as ctx:
        v, rep = ctx.register()
    assert rep["gn_iters"] == rep_o.gn_iters
    assert rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
    assert rep["mse_rel"] == pytest.approx(rep_o.mse_rel, rel=1e-3)
    assert rel_l2(host(v), v_o) < 1e-3


def test_graph_replayed_hessian_matches_eager():
    prob = spatial_problem((20, 24, 28), Vn.DEFSTATE, 1)
    with gpu_context(prob, max_gn=2, max_pcg=6) as ca, gpu_context(prob, max_gn=2, max_pcg=6) as cb:
        cb.set_option(L.OPT_GRAPHS, 1)
        va, ra = ca.register()
        vb, rb = cb.register()
    assert ra["pcg_iters_total"] == rb["pcg_iters_total"]
    assert rel_l2(host(vb), host(va)) < 1e-6


def test_full_size_zero_velocity_gradient_sampled():
    """192 x 224 x 192: at v = 0 the deformation-state gradient is rho(1) = -(2/sigma^2)
    (I0 - I1) G with G the trilinear derivative of I0 at the grid points (the forward
    difference), computed voxel by voxel here; and two Gauss-Newton updates lower the energy."""
    shape = (192, 224, 192)
    nz, ny, nx = shape
    I1 = synth.gaussian_blobs_device(shape, 0, "cuda")
    vt = synth.random_velocity_coeffs(32, 8, seed=1)
    V = L.bl_include(torch.as_tensor(vt.astype(np.complex64), device="cuda"), shape)
    V = V * (torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1)
             / (2 * np.pi))
    V *= 4.0 / V.pow(2).sum(0).sqrt().max()
    I0 = L.sl_transport(V, I1, 10, L.FORWARD, L.INTERP_LINEAR)
    with L.Context(nx, ny, nz, 0, nt=10, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR, max_gn=2,
                   max_pcg=5, gtol=0.0, spatial=True) as ctx:
        ctx.set_images(I0, I1)
        g = host(ctx.gradient(ctx.zeros_cube())[1])
        v, rep = ctx.register()
    a, b = host(I0), host(I1)
    rng = synth.rng(5)
    idx = np.stack([rng.integers(0, n, 2000) for n in shape], 1)
    for z, y, x in idx:
        gx = (a[z, y, (x + 1) % nx] - a[z, y, x]) * nx / (2 * np.pi)
        gy = (a[z, (y + 1) % ny, x] - a[z, y, x]) * ny / (2 * np.pi)
        gz = (a[(z + 1) % nz, y, x] - a[z, y, x]) * nz / (2 * np.pi)
        r = -(2 / 0.01) * (a[z, y, x] - b[z, y, x])
        ref = np.array([r * gx, r * gy, r * gz])
        assert np.abs(g[:, z, y, x] - ref).max() <= 1e-4 * (np.abs(ref).max() + 1.0)
    assert rep["gn_iters"] == 2 and rep["E"] < 0.9 * rep["E0"]


@pytest.mark.parametrize("variant,order", [(Vn.DEFSTATE, 1), (Vn.IMAGE, 3), (Vn.STATE, 1)])
def test_nonstationary_spatial_form_matches_oracle(variant, order):
    """One field per node (lddmm_params.spatial = nonstationary = 1) against SpatialProblemNS:
    energy, node gradients and Hessian-vector products, then a short registration."""
    shape, nt = (16, 16, 16), 4
    I0, I1 = blob_pair(shape, 8, seed=0, order=order)
    p = Vn.Params(K=0, nt=nt, order=order, variant=variant, sigma2=0.01)
    prob = Sp.SpatialProblemNS(I0, I1, p)
    base = field(shape, 3, 1.0)
    base *= 2.0 / np.abs(base * prob.tv).max()
    vs = np.stack([base * (0.5 + 0.1 * j) for j in range(nt + 1)])
    dvs = np.stack([field(shape, 20 + j, 0.1) for j in range(nt + 1)])
    E, Er, Ed, g = prob.gradient(vs)
    H = prob.hessian_matvec(vs, dvs)
    with gpu_context(prob, nonstationary=True, max_gn=3, max_pcg=5) as ctx:
        (Eg, Erg, _), gg = ctx.gradient(dev(vs))
        assert Eg == pytest.approx(E, rel=1e-5) and Erg == pytest.approx(Er, rel=1e-5)
        assert rel_l2(host(gg), g) < 1e-4
        assert rel_l2(host(ctx.hessian_matvec(dev(vs), dev(dvs))), H) < 1e-4
        v, rep = ctx.register()
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=5)
    assert v.shape == (nt + 1, 3) + shape
    assert rep["gn_iters"] == rep_o.gn_iters and rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
