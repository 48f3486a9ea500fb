"""Gradient and Gauss-Newton Hessian-vector parity against the FP64 oracle on a medium grid
that runs the benchmark's launch paths: 96 x 112 x 96 voxels (nx a multiple of 16, so the x
stages of pi and iota run on the tensor cores), band K = 32, four z planes per thread in the
pipelined SL kernels (the depth the paper-scale grid gets by default), and the paper-scale
input recipe scaled to this grid: the ellipsoid phantom warped by a random band-limited
velocity (4 voxels max displacement, the oracle's transport) with N(0, 0.01) noise on both
images. Trilinear and cubic B-spline interpolation (Sec. 4.2), deformation-state variant
(Sec. 2.3.3). The oracle's time steps are kept few (nt = 3 / 2) so that its FP64 sweeps
over the million voxels finish in about a minute."""
import numpy as np
import pytest

from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import rel_l2, scaled_velocity, voxel_velocity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

SHAPE = (96, 112, 96)   # nz, ny, nx
K = 32


def phantom_problem(order, nt, noisy=True):
    nz, ny, nx = SHAPE
    fixed = synth.ellipsoid_phantom(SHAPE)
    vt = scaled_velocity(K, K, 1, SHAPE, 8.0 * nx / 192)
    moving = SL.sl_transport(fixed, voxel_velocity(vt, SHAPE), 10, +1, 1)
    I0 = synth.add_noise(moving, seed=2) if noisy else moving
    I1 = synth.add_noise(fixed, seed=3) if noisy else fixed
    return Vn.Problem(I0, I1, Vn.Params(K=K, nt=nt, order=order, variant=Vn.DEFSTATE, sigma2=0.01))


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _devc(c):
    return torch.as_tensor(np.ascontiguousarray(c).astype(np.complex64), device="cuda")


# Tolerances (relative L2). Trilinear interpolation of a noisy image has a gradient that jumps
# across cell faces, and the gradient and Gauss-Newton product use it at the deformed points
# (G = grad I0 o phi(1)): FP32 rounding of a departure point moves some points across a face.
# The oracle's own FP64 gradient on the noisy trilinear case moves by 5.7e-4 when the velocity
# cube is perturbed by 6e-8 relative (FP32 rounding size), and by 8.5e-8 on the same phantom
# without noise, so the FP32 path is held to 1e-4 where the data are smooth (noise-free
# trilinear; cubic B-splines, whose gradient is continuous) and to 5e-3 on noisy trilinear.
@pytest.mark.parametrize("order,nt,noisy,tol", [(1, 3, False, 1e-4), (1, 3, True, 5e-3),
                                                (3, 2, True, 1e-4)])
def test_gradient_and_hessian_on_the_bench_launch_path(order, nt, noisy, tol):
    prob = phantom_problem(order, nt, noisy)
    vt = scaled_velocity(K, K, 5, SHAPE, 2.0)
    E, Er, Ed, g = prob.gradient(vt)
    # the first PCG direction of a Gauss-Newton step, L~^{-1}(-g), as the product's argument
    p = S.apply_Linv(-g, prob.p.alpha, prob.p.s)
    Hp = prob.hessian_matvec(vt, p)
    nz, ny, nx = SHAPE
    with L.Context(nx, ny, nz, K, nt=nt, variant=L.V_DEFSTATE, interp=order, alpha=prob.p.alpha,
                   s=prob.p.s, sigma2=prob.p.sigma2) as ctx:
        ctx.set_option(L.OPT_GATHER_ZT, 4)
        ctx.set_images(_dev(prob.I0), _dev(prob.I1))
        (Eg, _, _), gg = ctx.gradient(_devc(vt))
        Hg = ctx.hessian_matvec(_devc(vt), _devc(p))
        gg = gg.cpu().numpy().astype(np.complex128)
        Hg = Hg.cpu().numpy().astype(np.complex128)
    assert Eg == pytest.approx(E, rel=1e-5)
    assert rel_l2(gg, g) < tol
    assert rel_l2(Hg, Hp) < tol
    # the curvature PCG tests first (its sign decides a negative-curvature stop)
    assert S.inner(p, Hg) == pytest.approx(S.inner(p, Hp), rel=tol)
    assert S.inner(p, Hp) > 0


def small_phantom_problem(order, nt, shape=(32, 32, 32), K_=16):
    nz, ny, nx = shape
    fixed = synth.ellipsoid_phantom(shape)
    vt = scaled_velocity(K_, K_, 1, shape, 8.0 * nx / 192)
    moving = SL.sl_transport(fixed, voxel_velocity(vt, shape), 10, +1, 1)
    I0 = synth.add_noise(moving, seed=2)
    I1 = synth.add_noise(fixed, seed=3)
    return Vn.Problem(I0, I1, Vn.Params(K=K_, nt=nt, order=order, variant=Vn.DEFSTATE, sigma2=0.01))


@pytest.mark.parametrize("order", [1, 3])
def test_noisy_phantom_registration_follows_the_oracle_iterate_by_iterate(order):
    """Gauss-Newton on the noisy ellipsoid phantom (the paper-scale recipe at 32^3): the GPU's
    PCG iteration counts, stop reason, and per-iterate energy and relative residual follow the
    oracle's. With cubic interpolation both take only one to three PCG iterations per
    Gauss-Newton step (a single conjugate-gradient step already meets the forcing term 0.5)
    and the residual falls slowly, as the cubic form does at the paper grid."""
    from oracle import gnk
    prob = small_phantom_problem(order, nt=4)
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=20)
    nz, ny, nx = prob.I0.shape
    with L.Context(nx, ny, nz, prob.p.K, nt=prob.p.nt, variant=L.V_DEFSTATE, interp=order,
                   alpha=prob.p.alpha, s=prob.p.s, sigma2=prob.p.sigma2, max_gn=3,
                   max_pcg=20) as ctx:
        ctx.set_images(_dev(prob.I0), _dev(prob.I1))
        _, rep = ctx.register()
        hist = ctx.history()
    assert rep["gn_iters"] == rep_o.gn_iters
    assert rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["stop_reason"] == rep_o.stop_reason
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
    assert rep["grad_rel_l2"] == pytest.approx(rep_o.grad_rel_l2, rel=1e-2)
    # the history: one record per iterate, the oracle's (E, residual) before each update
    assert len(hist) == rep["gn_iters"] + 1
    for h, (E_o, res_o) in zip(hist, rep_o.history):
        assert h["E"] == pytest.approx(E_o, rel=1e-3)
        assert h["residual"] == pytest.approx(res_o, rel=1e-2)
    assert hist[-1]["residual"] == pytest.approx(rep["grad_rel_l2"], rel=1e-12)
    assert hist[-1]["pcg"] == rep["pcg_iters_total"]
    assert all(b["t"] >= a["t"] for a, b in zip(hist, hist[1:]))
