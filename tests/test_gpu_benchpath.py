"""Gradient and Gauss-Newton Hessian-vector parity against the FP64 oracle on a medium grid
that runs the benchmark's launch paths: 96 x 112 x 96 voxels (nx a multiple of 16, so the x
stages of pi and iota run on the tensor cores), band K = 32, four z planes per thread in the
pipelined SL kernels (the depth the paper-scale grid gets by default), and the paper-scale
input recipe scaled to this grid: the ellipsoid phantom warped by a random band-limited
velocity (4 voxels max displacement, the oracle's transport) with N(0, 0.01) noise on both
images. Trilinear and cubic B-spline interpolation (Sec. 4.2), deformation-state variant
(Sec. 2.3.3). The oracle's time steps are kept few (nt = 3 / 2). The inputs are rebuilt here
from the seeded generator and the oracle's transport; the oracle's gradient, Gauss-Newton
product and registration reports, which take minutes of host time at this size, are read
from ``tests/golden/`` as written by ``tests/golden/make_benchpath.py`` (oracle calls only;
``tests/test_golden_benchpath.py`` checks them against the live oracle where that is cheap)."""
import json
import os

import numpy as np
import pytest

from _problems import BENCH_K, BENCH_SHAPE, bench_phantom_problem, bench_velocity, \
    first_direction, rel_l2, small_phantom_problem
from oracle import spectral as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _devc(c):
    return torch.as_tensor(np.ascontiguousarray(c).astype(np.complex64), device="cuda")


def _stored(order, nt, noisy):
    kind = "noisy" if noisy else "clean"
    return np.load(os.path.join(GOLDEN, f"benchpath_o{order}_nt{nt}_{kind}.npz"))


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
    prob = bench_phantom_problem(order, nt, noisy)
    ref = _stored(order, nt, noisy)
    E, g, Hp, pHp = float(ref["E"]), ref["g"], ref["Hp"], float(ref["pHp"])
    # the first PCG direction of a Gauss-Newton step, L~^{-1}(-g), as the product's argument
    p = first_direction(g, prob.p.alpha, prob.p.s)
    vt = bench_velocity()
    nz, ny, nx = BENCH_SHAPE
    with L.Context(nx, ny, nz, BENCH_K, nt=nt, variant=L.V_DEFSTATE, interp=order,
                   alpha=prob.p.alpha, s=prob.p.s, sigma2=prob.p.sigma2) as ctx:
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
    assert S.inner(p, Hg) == pytest.approx(pHp, rel=tol)
    assert pHp > 0


@pytest.mark.parametrize("order", [1, 3])
def test_noisy_phantom_registration_follows_the_oracle_iterate_by_iterate(order):
    """Gauss-Newton on the noisy ellipsoid phantom (the paper-scale recipe at 32^3): the GPU's
    PCG iteration counts, stop reason, and per-iterate energy and relative residual follow the
    oracle's. With cubic interpolation both take only one to three PCG iterations per
    Gauss-Newton step (a single conjugate-gradient step already meets the forcing term 0.5)
    and the residual falls slowly, as the cubic form does at the paper grid."""
    with open(os.path.join(GOLDEN, f"benchpath_registration_o{order}.json")) as f:
        rep_o = json.load(f)
    cfg = rep_o["config"]
    prob = small_phantom_problem(order, nt=cfg["nt"])
    nz, ny, nx = prob.I0.shape
    with L.Context(nx, ny, nz, prob.p.K, nt=prob.p.nt, variant=L.V_DEFSTATE, interp=order,
                   alpha=prob.p.alpha, s=prob.p.s, sigma2=prob.p.sigma2, max_gn=cfg["max_gn"],
                   max_pcg=cfg["max_pcg"]) as ctx:
        ctx.set_images(_dev(prob.I0), _dev(prob.I1))
        _, rep = ctx.register()
        hist = ctx.history()
    assert rep["gn_iters"] == rep_o["gn_iters"]
    assert rep["pcg_iters_total"] == rep_o["pcg_iters_total"]
    assert rep["stop_reason"] == rep_o["stop_reason"]
    assert rep["E"] == pytest.approx(rep_o["E"], rel=1e-3)
    assert rep["grad_rel_l2"] == pytest.approx(rep_o["grad_rel_l2"], rel=1e-2)
    # the history: one record per iterate, the oracle's (E, residual) before each update
    assert len(hist) == rep["gn_iters"] + 1
    for h, (E_o, res_o) in zip(hist, rep_o["history"]):
        assert h["E"] == pytest.approx(E_o, rel=1e-3)
        assert h["residual"] == pytest.approx(res_o, rel=1e-2)
    assert hist[-1]["residual"] == pytest.approx(rep["grad_rel_l2"], rel=1e-12)
    assert hist[-1]["pcg"] == rep["pcg_iters_total"]
    assert all(b["t"] >= a["t"] for a, b in zip(hist, hist[1:]))
