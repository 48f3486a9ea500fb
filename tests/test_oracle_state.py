"""Pins of the oracle's state-equation variant (Sec. 2.3.2): m = I0 o phi, lambda = J lambda(1) o psi.

Closed forms (translations, a single cosine), the identities that tie its two backward
equations to the adjoint of Eq. 18, inverse consistency of phi(1) and psi(0), and finite
differences of the discrete energy (the gradient is optimise-then-discretise, so those agree
up to a measured discretisation error).
"""
import numpy as np
import pytest

from oracle import interp as I
from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth

N = 16
K = 8


def _problem(order, nt=10, zero_residual=False, variant=Vn.STATE, K_=K):
    shape = (N, N, N)
    I1 = synth.gaussian_blobs(shape, seed=0)
    p = Vn.Params(K=K_, nt=nt, order=order, variant=variant, sigma2=0.01)
    vgen = synth.random_velocity_coeffs(K_, 8, seed=1)
    base = Vn.Problem(I1, I1, p)
    _, V, _ = base.velocity(vgen)
    sc = 2.0 / np.abs(V).max()
    I0 = I1 if zero_residual else SL.sl_transport(I1, V * sc, 10, +1, order)
    return Vn.Problem(I0, I1, p), vgen * sc


def _xgrid(n=N):
    return 2 * np.pi * np.arange(n) / n


def _translation_problem(variant, a, nt):
    """I0 = cos x, I1 = cos(x - a) on N^3, stationary velocity c along x (k = 0 only)."""
    x = _xgrid()
    I0 = np.broadcast_to(np.cos(x), (N, N, N)).copy()
    I1 = np.broadcast_to(np.cos(x - a), (N, N, N)).copy()
    return Vn.Problem(I0, I1, Vn.Params(K=K, nt=nt, order=3, variant=variant, sigma2=0.01))


@pytest.mark.parametrize("variant", [Vn.IMAGE, Vn.STATE, Vn.DEFSTATE])
def test_translation_gradient_and_hessian_closed_form(variant):
    # v = c e_x moving c dt N / (2 pi) = 1 voxel per step: with the interpolating cubic spline
    # every characteristic, composition and source integral is exact, m(t) = cos(x - t c),
    # J = 1, E(c) = c^2 / 2 + (1 - cos(a - c)) / sigma^2 and dE/dc = c - sin(a - c) / sigma^2.
    # Where the derivative of the interpolant of I0 enters (G), it is the spline's: at the
    # nodes a mode of step h is differentiated with the symbol mu = (sin h / h) 3 / (2 + cos h)
    # (coefficients c = f / ((4 + 2 cos h) / 6), s'(x_j) = (c_{j+1} - c_{j-1}) / 2h).
    nt, a, s2 = 4, 0.7, 0.01
    c = 2 * np.pi / N * nt
    hh = 2 * np.pi / N
    mu = np.sin(hh) / hh * 3 / (2 + np.cos(hh))
    prob = _translation_problem(variant, a, nt)
    vt = np.zeros((3, K, K, K), complex)
    h = K // 2
    vt[0, h, h, h] = c
    E, Er, Ed, g = prob.gradient(vt)
    assert Ed == pytest.approx((1 - np.cos(a - c)) / s2, rel=1e-12)
    g_data = {Vn.IMAGE: 1.0, Vn.STATE: 1.0, Vn.DEFSTATE: mu}[variant]   # G in rho(1) only
    assert g[0, h, h, h].real == pytest.approx(c - g_data * np.sin(a - c) / s2, rel=1e-12)
    assert abs(g[0, h, h, h].imag) < 1e-12
    assert np.abs(g[1:]).max() < 1e-11
    dv = np.zeros_like(vt)
    dv[0, h, h, h] = 0.3
    Hd = prob.hessian_matvec(vt, dv)
    # dm(1) carries G in STATE and DEFSTATE, drho(1) carries it once more in DEFSTATE
    h_data = {Vn.IMAGE: 1.0, Vn.STATE: mu, Vn.DEFSTATE: mu * mu}[variant]
    assert Hd[0, h, h, h].real == pytest.approx(0.3 * (1 + h_data / s2), rel=1e-12)
    assert np.abs(Hd[1:]).max() < 1e-11


@pytest.mark.parametrize("variant", [Vn.IMAGE, Vn.STATE, Vn.DEFSTATE])
def test_zero_velocity_gradient_of_a_single_cosine(variant):
    # v = 0, I0 = cos x, I1 = 0: lambda(t) = -(2/sigma^2) cos x, grad m = -sin x e_x, so
    # g = pi((1/sigma^2) sin 2x) e_x: -i/(2 sigma^2) at kx = +2, +i/(2 sigma^2) at kx = -2,
    # zero elsewhere. DEFSTATE's rho(1) carries the spline derivative of I0, mu (-sin x).
    x = _xgrid()
    I0 = np.broadcast_to(np.cos(x), (N, N, N)).copy()
    prob = Vn.Problem(I0, np.zeros_like(I0),
                      Vn.Params(K=K, nt=5, order=3, variant=variant, sigma2=0.01))
    g = prob.gradient(np.zeros((3, K, K, K), complex))[3]
    hh = 2 * np.pi / N
    mu = np.sin(hh) / hh * 3 / (2 + np.cos(hh)) if variant == Vn.DEFSTATE else 1.0
    ref = np.zeros_like(g)
    h = K // 2
    ref[0, h, h, h + 2] = -0.5j / 0.01 * mu
    ref[0, h, h, h - 2] = 0.5j / 0.01 * mu
    np.testing.assert_allclose(g, ref, atol=1e-10)


def test_state_and_deformation_state_share_the_energy():
    ps, vt = _problem(1)
    pd, _ = _problem(1, variant=Vn.DEFSTATE)
    vt = vt * 0.3
    assert ps.objective(vt)[0] == pd.objective(vt)[0]


def test_jacobian_equation_step_is_the_adjoint_step_of_one_minus_U():
    # J = 1 - U obeys -D_t J = J div v, the equation of lambda (Table 1 row 2), step for step
    rng = np.random.default_rng(3)
    shape = (N, N, N)
    U = 0.2 * rng.standard_normal(shape)
    d = 0.5 * rng.standard_normal(shape)
    Dp = 0.7 * rng.standard_normal((3,) + shape)
    for order in (1, 3):
        a = SL.heun_jacobian_step(U, Dp, d, 0.1, order)
        b = 1.0 - SL.heun_divergence_step(1.0 - U, Dp, d, 0.1, order)
        np.testing.assert_allclose(a, b, atol=1e-13)


def _smooth_field():
    x = _xgrid()
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    return np.cos(xx) * np.cos(y) + 0.5 * np.sin(2 * z + y) + 0.3 * np.cos(xx - 2 * z)


@pytest.mark.parametrize("order,tol", [(1, 4e-2), (3, 3e-3)])
def test_pulled_back_adjoint_matches_the_transported_adjoint(order, tol):
    # lambda(t) = J(t) lambda(1) o psi(t) solves Eq. 18: compare with the SL transport of a
    # smooth lambda(1) backward (IMAGE's adjoint) at every node; they differ by discretisation
    # only (measured 2.5e-2 trilinear, 8e-4 cubic; without J, or with nu or U of the wrong
    # sign, the difference is 0.1 to 0.4).
    prob, vt = _problem(order, K_=12)
    vt = vt * 0.5
    lam1 = _smooth_field()
    nus, Us = prob.inverse_maps(vt)
    pulled = prob._pull_back(lam1, nus, Us)
    _, V, d = prob.velocity(vt)
    Dp = SL.departure_offsets(V, prob.dt, -1, order)
    lam = lam1
    for j in range(prob.p.nt, -1, -1):
        if j < prob.p.nt:
            lam = SL.heun_divergence_step(lam, Dp, d, prob.dt, order)
        err = np.linalg.norm(pulled[j] - lam) / np.linalg.norm(lam1)
        assert err < tol, (j, err)


def test_psi0_inverts_phi1_and_J0_is_its_jacobian_determinant():
    # measured 3.5e-3 and 5.6e-3 (band truncation of the displacements dominates)
    prob, vt = _problem(3, K_=12)
    vt = vt * 0.5
    us = prob.state_defstate(vt)
    nus, Us = prob.inverse_maps(vt)
    tv = prob.to_vox[:, None, None, None]
    nu0 = S.include(nus[0], prob.shape)
    u1 = S.include(us[-1], prob.shape)
    # phi1(psi0(x)) - x = -nu0(x) - u1(x - nu0(x))
    u1_at = I.interpolate(u1 * tv, -nu0 * tv, 3) / tv
    resid = np.abs(-nu0 - u1_at).max()
    assert resid < 1e-2 * np.abs(u1).max(), resid
    J0 = 1.0 - S.include(Us[0], prob.shape)
    detpsi = Vn.Problem.jacobian_determinant_of(nus[0], prob.shape)
    assert np.abs(J0 - detpsi).max() < 1e-2 * np.abs(detpsi - 1).max()
    assert abs(J0.mean() - 1.0) < 1e-3     # psi0 is a diffeomorphism of the torus


def test_zero_velocity_maps_are_the_identity():
    prob, _ = _problem(1)
    nus, Us = prob.inverse_maps(np.zeros((3, K, K, K), complex))
    assert all(np.abs(n).max() == 0 for n in nus) and all(np.abs(u).max() == 0 for u in Us)


@pytest.mark.parametrize("order,tol", [(1, 1e-2), (3, 3e-3)])
def test_state_gradient_matches_central_differences(order, tol):
    # |fd - <g, dv>| against the Cauchy-Schwarz scale |g| |dv| (measured 4.5e-3 trilinear,
    # 1.5e-3 cubic): the directional derivatives themselves can nearly cancel
    prob, vt = _problem(order)
    vt = vt * 0.3
    g = prob.gradient(vt)[3]
    h = 1e-3
    for seed in (5, 6, 7):
        dvt = synth.random_coeffs(K, seed) * 0.05
        fd = (prob.objective(vt + h * dvt)[0] - prob.objective(vt - h * dvt)[0]) / (2 * h)
        scale = np.sqrt(S.inner(g, g) * S.inner(dvt, dvt))
        assert abs(fd - S.inner(g, dvt)) <= tol * scale, (fd, S.inner(g, dvt), scale)


def test_state_hessian_matches_gradient_differences_at_zero_residual():
    # at a zero residual the residual terms Gauss-Newton drops vanish
    prob, _ = _problem(3, zero_residual=True)
    vt = np.zeros((3, K, K, K), complex)
    d = synth.random_coeffs(K, 9) * 0.05
    h = 1e-3
    fd = (prob.gradient(vt + h * d)[3] - prob.gradient(vt - h * d)[3]) / (2 * h)
    Hd = prob.hessian_matvec(vt, d)
    assert np.linalg.norm(fd - Hd) <= 1e-3 * np.linalg.norm(Hd)


@pytest.mark.parametrize("order,tol", [(1, 2e-2), (3, 1.2e-2)])
def test_state_gauss_newton_hessian_is_symmetric_positive(order, tol):
    # |<y, Hx> - <x, Hy>| against sqrt(<x, Hx> <y, Hy>) (measured 1.0e-2 trilinear, 6.6e-3
    # cubic: the optimise-then-discretise operator is symmetric up to discretisation)
    prob, vt = _problem(order)
    vt = vt * 0.3
    for sx, sy in ((7, 8), (9, 10), (11, 12)):
        x = synth.random_coeffs(K, sx) * 0.05
        y = synth.random_coeffs(K, sy) * 0.05
        Hx, Hy = prob.hessian_matvec(vt, x), prob.hessian_matvec(vt, y)
        xHx, yHy = S.inner(x, Hx), S.inner(y, Hy)
        assert abs(S.inner(y, Hx) - S.inner(x, Hy)) <= tol * np.sqrt(xHx * yHy)
        assert xHx > S.inner(x, S.apply_L(x, 0.0025, 2))
        assert yHy > S.inner(y, S.apply_L(y, 0.0025, 2))
