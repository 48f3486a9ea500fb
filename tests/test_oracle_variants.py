"""Pins of the oracle's energy, gradient and GN Hessian (Sec. 2.3.1, 2.3.3).

The gradient is derived optimise-then-discretise, so it matches finite differences of the
discrete energy only up to discretisation error: the tolerances below are measured ones.
"""
import numpy as np
import pytest

from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import oracle_problem

N = 16
K = 8


def _problem(variant, order, nt=10, zero_residual=False):
    shape = (N, N, N)
    I1 = synth.gaussian_blobs(shape, seed=0)
    p = Vn.Params(K=K, nt=nt, order=order, variant=variant, sigma2=0.01)
    vgen = synth.random_velocity_coeffs(K, 8, seed=1)
    base = Vn.Problem(I1, I1, p)
    _, V, _ = base.velocity(vgen)
    sc = 2.0 / np.abs(V).max()
    I0 = I1 if zero_residual else SL.sl_transport(I1, V * sc, 10, +1, order)
    return Vn.Problem(I0, I1, p), vgen * sc


def _fd(prob, vt, dvt, h=1e-3):
    return (prob.objective(vt + h * dvt)[0] - prob.objective(vt - h * dvt)[0]) / (2 * h)


def test_zero_velocity_and_equal_images_give_zero_energy():
    prob, _ = _problem(Vn.DEFSTATE, 1, zero_residual=True)
    E, Er, Ed, m1 = prob.objective(np.zeros((3, K, K, K), complex))
    assert E == 0.0 and Er == 0.0 and Ed == 0.0


def test_regularisation_energy_closed_form_single_mode():
    prob, _ = _problem(Vn.DEFSTATE, 1, zero_residual=True)
    vt = np.zeros((3, K, K, K), complex)
    h = K // 2
    vt[1, h + 2, h - 1, h + 3] = 0.4 + 0.1j
    vt[1, h - 2, h + 1, h - 3] = 0.4 - 0.1j
    w = (1 + 0.0025 * (4 + 1 + 9)) ** 2
    assert prob.energy_reg(vt) == pytest.approx(0.5 * w * 2 * (0.16 + 0.01), rel=1e-14)


def test_data_energy_at_zero_velocity_is_the_image_mse():
    for variant in (Vn.IMAGE, Vn.DEFSTATE):
        prob, _ = _problem(variant, 1)
        E, Er, Ed, m1 = prob.objective(np.zeros((3, K, K, K), complex))
        assert Ed == pytest.approx(np.mean((prob.I0 - prob.I1) ** 2) / 0.01, rel=1e-13)


@pytest.mark.parametrize("variant", [Vn.IMAGE, Vn.DEFSTATE])
def test_constant_images_reduce_gradient_and_hessian_to_L(variant):
    shape = (N, N, N)
    c = np.full(shape, 0.4)
    prob = Vn.Problem(c, c, Vn.Params(K=K, nt=5, variant=variant))
    vt = synth.random_coeffs(K, seed=2) * 0.05
    E, Er, Ed, g = prob.gradient(vt)
    assert Ed < 1e-28
    np.testing.assert_allclose(g, S.apply_L(vt, 0.0025, 2), atol=1e-14)
    dv = synth.random_coeffs(K, seed=3)
    np.testing.assert_allclose(prob.hessian_matvec(vt, dv), S.apply_L(dv, 0.0025, 2), atol=1e-13)


@pytest.mark.parametrize("order,tol", [(1, 1e-2), (3, 1e-3)])
def test_defstate_gradient_matches_central_differences(order, tol):
    prob, vt = _problem(Vn.DEFSTATE, order)
    vt = vt * 0.3
    g = prob.gradient(vt)[3]
    for seed in (5, 6, 7):
        dvt = synth.random_coeffs(K, seed) * 0.05
        fd = _fd(prob, vt, dvt)
        assert abs(fd - S.inner(g, dvt)) <= tol * abs(fd), (fd, S.inner(g, dvt))


def test_image_variant_gradient_matches_central_differences_with_cubic():
    prob, vt = _problem(Vn.IMAGE, 3)
    vt = vt * 0.3
    g = prob.gradient(vt)[3]
    for seed in (5, 6):
        dvt = synth.random_coeffs(K, seed) * 0.05
        fd = _fd(prob, vt, dvt)
        assert abs(fd - S.inner(g, dvt)) <= 5e-2 * abs(fd)


@pytest.mark.parametrize("variant", [Vn.IMAGE, Vn.DEFSTATE])
def test_negative_gradient_is_a_descent_direction(variant):
    prob, vt = _problem(variant, 1)
    vt = vt * 0.3
    E, _, _, g = prob.gradient(vt)
    step = 1e-3 / np.sqrt(S.inner(g, g))
    assert prob.objective(vt - step * g)[0] < E


@pytest.mark.parametrize("variant,order,tol", [(Vn.DEFSTATE, 1, 1e-2), (Vn.DEFSTATE, 3, 1e-3),
                                               (Vn.IMAGE, 1, 3e-2), (Vn.IMAGE, 3, 1e-2)])
def test_gauss_newton_hessian_is_symmetric_positive(variant, order, tol):
    prob, vt = _problem(variant, order)
    vt = vt * 0.3
    x = synth.random_coeffs(K, 7) * 0.05
    y = synth.random_coeffs(K, 8) * 0.05
    Hx, Hy = prob.hessian_matvec(vt, x), prob.hessian_matvec(vt, y)
    a, b = S.inner(y, Hx), S.inner(x, Hy)
    assert abs(a - b) <= tol * max(abs(a), abs(b))
    assert S.inner(x, Hx) > S.inner(x, S.apply_L(x, 0.0025, 2))
    assert S.inner(y, Hy) > S.inner(y, S.apply_L(y, 0.0025, 2))


def test_defstate_hessian_matches_gradient_differences_at_zero_residual():
    prob, _ = _problem(Vn.DEFSTATE, 3, zero_residual=True)
    vt = np.zeros((3, K, K, K), complex)
    d = synth.random_coeffs(K, 9) * 0.05
    h = 1e-3
    fd = (prob.gradient(vt + h * d)[3] - prob.gradient(vt - h * d)[3]) / (2 * h)
    Hd = prob.hessian_matvec(vt, d)
    assert np.linalg.norm(fd - Hd) <= 1e-3 * np.linalg.norm(Hd)


def _single_mode(K, comp, axis, amp):
    """Cube of u with u_comp = amp sin(x_axis) (wavenumber 1 along axis), other comps zero."""
    c = np.zeros((3, K, K, K), dtype=np.complex128)
    idx_p = [K // 2] * 3
    idx_m = [K // 2] * 3
    ax = 2 - axis                      # cube index order [jz][jy][jx]
    idx_p[ax] += 1
    idx_m[ax] -= 1
    c[(comp,) + tuple(idx_p)] = -0.5j * amp      # sin = (e^{ix} - e^{-ix}) / 2i
    c[(comp,) + tuple(idx_m)] = 0.5j * amp
    return c


def test_jacobian_determinant_closed_forms():
    """det(I - Du): u = (a sin x, 0, 0) gives 1 - a cos x; u = (a sin y, 0, 0) is a shear,
    det 1; zero velocity gives the identity map, det 1 exactly."""
    shape, K, a = (8, 10, 12), 6, 0.3
    nz, ny, nx = shape
    x = 2 * np.pi * np.arange(nx) / nx
    J = Vn.Problem.jacobian_determinant_of(_single_mode(K, 0, 0, a), shape)
    np.testing.assert_allclose(J, np.broadcast_to(1 - a * np.cos(x), shape), atol=1e-12)
    J = Vn.Problem.jacobian_determinant_of(_single_mode(K, 0, 1, a), shape)
    np.testing.assert_allclose(J, 1.0, atol=1e-12)
    # two components: u = (a sin x, b sin y, 0) -> (1 - a cos x)(1 - b cos y)
    c = _single_mode(K, 0, 0, a) + _single_mode(K, 1, 1, 0.2)
    y = 2 * np.pi * np.arange(ny) / ny
    J = Vn.Problem.jacobian_determinant_of(c, shape)
    ref = (1 - a * np.cos(x))[None, None, :] * (1 - 0.2 * np.cos(y))[None, :, None]
    np.testing.assert_allclose(J, np.broadcast_to(ref, shape), atol=1e-12)
    prob = oracle_problem((8, 8, 8), 4, Vn.DEFSTATE, 1, nt=3)
    assert np.array_equal(prob.jacobian_determinant(np.zeros((3, 4, 4, 4), complex)), np.ones((8, 8, 8)))


def _smooth_pair(N, shift=0.3):
    """Three periodic Gaussian blobs defined on [0, 2 pi)^3 (so every grid samples the same
    functions): the fixed image and a copy shifted by `shift` rad along y (and shift/2 along x)."""
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")

    def blobs(s_):
        f = np.zeros((N, N, N))
        for cz, cy, cx, w, a in [(2.0, 3.0, 2.5, 0.7, 1.0), (4.0, 2.0, 4.2, 0.9, 0.6),
                                 (3.5, 4.5, 1.5, 0.6, 0.8)]:
            d2 = sum(np.angle(np.exp(1j * (C - c))) ** 2
                     for C, c in ((Z, cz), (Y, cy + s_), (X, cx + 0.5 * s_)))
            f += a * np.exp(-d2 / (2 * w * w))
        return f

    return blobs(shift), blobs(0.0)


@pytest.mark.parametrize("order,min_ratio", [(1, 1.5), (3, 8.0)])
def test_defstate_gradient_gap_shrinks_under_refinement(order, min_ratio):
    """Optimise-then-discretise: the adjoint gradient is the derivative of the discrete energy
    only up to the discretisation error, so the gap to central differences must shrink when the
    grid and the time step are refined together (N, nt) = (12, 4) -> (24, 8) at a fixed band:
    at least linearly for trilinear SL (measured 4.2x and 1.7x on two directions), much faster
    for cubic (measured 12x and 19x)."""
    K = 8
    vt = synth.random_velocity_coeffs(K, 6, seed=3)
    dvs = [synth.random_coeffs(K, seed) * 0.05 for seed in (5, 6)]
    gaps = {}
    for N, nt in ((12, 4), (24, 8)):
        I0, I1 = _smooth_pair(N)
        prob = Vn.Problem(I0, I1, Vn.Params(K=K, nt=nt, order=order, variant=Vn.DEFSTATE))
        v = vt * (0.15 / np.abs(S.include(vt, (N, N, N))).max())
        g = prob.gradient(v)[3]
        fds = [_fd(prob, v, dv) for dv in dvs]
        gaps[N] = [abs(fd - S.inner(g, dv)) / abs(fd) for fd, dv in zip(fds, dvs)]
    for coarse, fine in zip(gaps[12], gaps[24]):
        assert fine * min_ratio <= coarse, gaps
