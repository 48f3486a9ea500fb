"""Pins of the oracle's two-level preconditioner and flexible PCG (``oracle/multilevel.py``;
the multi-level preconditioner the paper names in Secs. 6-7 as the way to a faster PCG of
Sec. 2.2, Eqs. 13-14)."""
import numpy as np
import pytest

from oracle import gnk
from oracle import multilevel as ML
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth

from _problems import blob_pair, rel_l2


def _trig_field(shape, kmax, seed):
    """A real trigonometric polynomial on [0, 2 pi)^3 with |k_a| <= kmax, evaluated on the grid
    by direct summation, and its evaluator at arbitrary grids."""
    rng = np.random.default_rng(seed)
    modes = [(int(kz), int(ky), int(kx), complex(*rng.normal(size=2)))
             for kz in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
             for kx in range(-kmax, kmax + 1) if rng.random() < 0.3]

    def at(sh):
        z, y, x = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in sh], indexing="ij")
        f = np.zeros(sh)
        for kz, ky, kx, a in modes:
            f += (a * np.exp(1j * (kz * z + ky * y + kx * x))).real
        return f

    return at(shape), at


def test_coarse_band():
    assert [ML.coarse_band(K) for K in (8, 10, 12, 16, 32, 64)] == [4, 4, 6, 8, 16, 32]


def test_restrict_image_samples_a_trigonometric_polynomial_of_the_coarse_band():
    shape = (16, 20, 12)                    # half grid 8 x 10 x 6: |k| <= 2 is inside every axis
    f, at = _trig_field(shape, 2, seed=3)
    got = ML.restrict_image(f)
    np.testing.assert_allclose(got, f[::2, ::2, ::2], atol=1e-12)
    np.testing.assert_allclose(got, at(tuple(n // 2 for n in shape)), atol=1e-12)


def test_restrict_image_drops_modes_outside_the_half_grid_band():
    shape = (16, 16, 16)
    z, y, x = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in shape], indexing="ij")
    # the half-grid Nyquist mode and modes above it vanish (no aliasing onto lower modes)
    for f in (np.cos(4 * x), np.sin(5 * y + 2 * z), np.cos(6 * z) * np.cos(x)):
        np.testing.assert_allclose(ML.restrict_image(f), 0.0, atol=1e-12)
    np.testing.assert_allclose(ML.restrict_image(np.full(shape, 0.7)), 0.7, atol=1e-14)


def test_restrict_and_prolong_follow_the_slot_convention_of_pi_and_iota():
    K, Kc, shape = 12, 6, (16, 16, 16)
    cc = S.hermitian_part(synth.random_coeffs(Kc, seed=4, ncomp=1)[0])   # a cube of band S_c
    f = S.include(cc, shape)                             # the function it describes
    # pi of that function at band K holds the same coefficients, zero-padded
    np.testing.assert_allclose(S.project(f, K), ML.prolong_cube(cc, K), atol=1e-12)
    np.testing.assert_allclose(ML.restrict_cube(S.project(f, K), Kc), cc, atol=1e-12)
    # and the same function synthesised on the half grid is the restricted image
    np.testing.assert_allclose(S.include(cc, (8, 8, 8)), ML.restrict_image(f), atol=1e-12)


def test_restrict_is_the_adjoint_of_prolong_and_a_left_inverse():
    K, Kc = 10, 4
    a = synth.random_coeffs(K, seed=5)
    b = synth.random_coeffs(Kc, seed=6)
    b[..., 0, :, :] = b[..., :, 0, :] = b[..., :, :, 0] = 0
    assert abs(S.inner(ML.restrict_cube(a, Kc), b) - S.inner(a, ML.prolong_cube(b, K))) < 1e-12
    np.testing.assert_allclose(ML.restrict_cube(ML.prolong_cube(b, K), Kc), b, atol=0)
    # slot 0 of the coarse cube (k = -K_c/2) is never filled
    r = ML.restrict_cube(a, Kc)
    assert not r[..., 0, :, :].any() and not r[..., :, 0, :].any() and not r[..., :, :, 0].any()


class _Diag:
    """A diagonal SPD 'problem' on cubes of band K: H c = (w_k + shift_k) c on S."""

    def __init__(self, K, shift):
        self.p = Vn.Params(K=K, alpha=0.0025, s=2)
        w = S.l_symbol(K, self.p.alpha, self.p.s)
        self.d = np.where(w > 0, w + shift, 0.0)

    def hessian_matvec(self, vt, c):
        return self.d * c


def test_two_level_inverts_a_multiple_of_L_exactly():
    """H = c L~ on both levels: with an exact inner solve P^{-1} = H^{-1} (the coarse part solves
    exactly, and the scale theta carries 1/c over to the modes above the coarse band)."""
    K, Kc, c = 12, 6, 37.5
    coarse, fine = _Diag(Kc, 0.0), _Diag(K, 0.0)
    coarse.d *= c
    fine.d *= c
    tl = ML.TwoLevel(fine, coarse, inner_maxit=400, inner_tol=1e-15)
    tl.set_velocity(np.zeros((3, K, K, K), complex))
    r = synth.random_coeffs(K, seed=7)
    exact = np.where(fine.d > 0, r / np.where(fine.d > 0, fine.d, 1), 0)
    assert rel_l2(tl(r), exact) < 1e-12
    x, its, _ = ML.fpcg(lambda v: fine.d * v, r, tl, 1e-10, 20)
    assert its == 1 and rel_l2(x, exact) < 1e-12
    # no low-band content: theta = 1, P^{-1} = L~^{-1}
    rh = r - ML.prolong_cube(ML.restrict_cube(r, Kc), K)
    assert rel_l2(tl(rh), S.apply_Linv(rh, 0.0025, 2)) < 1e-14


def test_two_level_coarse_correction_beats_L_on_a_low_band_perturbation():
    """H = L~ + E D R (a large SPD perturbation on the coarse band, the regime the coarse level
    is for): with the coarse operator R H E, flexible PCG with the two-level preconditioner
    converges in far fewer iterations than PCG with L~^{-1}."""
    K, Kc = 12, 6
    rng = np.random.default_rng(15)
    fine = _Diag(K, 0.0)
    pert = ML.prolong_cube(np.where(ML.restrict_cube(fine.d, Kc) > 0,
                                    200.0 * rng.random((Kc, Kc, Kc)), 0.0), K)
    fine.d = fine.d + pert
    coarse = _Diag(Kc, 0.0)
    coarse.d = ML.restrict_cube(fine.d, Kc)
    tl = ML.TwoLevel(fine, coarse, inner_maxit=400, inner_tol=1e-13)
    tl.set_velocity(np.zeros((3, K, K, K), complex))
    b = synth.random_coeffs(K, seed=16)
    exact = np.where(fine.d > 0, b / np.where(fine.d > 0, fine.d, 1), 0)
    x, its, _ = ML.fpcg(lambda v: fine.d * v, b, tl, 1e-9, 100)
    _, its_spec, _ = gnk.pcg(lambda v: fine.d * v, b, lambda v: S.apply_Linv(v, 0.0025, 2),
                             1e-9, 100)
    assert rel_l2(x, exact) < 1e-8
    assert its <= its_spec // 2, (its, its_spec)


def test_fpcg_keeps_successive_directions_conjugate_under_a_nonlinear_preconditioner():
    """The defining property of flexible CG: <p_{k+1}, H p_k> = 0 for any preconditioner; a few
    inner CG steps (a nonlinear map of r) break it for the Fletcher-Reeves beta of plain PCG."""
    K = 8
    w = S.l_symbol(K, 0.0025, 2)
    rng = np.random.default_rng(8)
    d = np.where(w > 0, w * (1 + 20 * rng.random(w.shape)), 0.0)
    d_inner = np.where(w > 0, w * (1 + 20 * rng.random(w.shape)), 0.0)  # another operator
    hv_inner = lambda c: d_inner * c
    # exactly two inner steps (one step would only rescale L~^{-1} r, which is still linear)
    prec = lambda r: gnk.pcg(hv_inner, r, lambda c: S.apply_Linv(c, 0.0025, 2), 1e-14, 2)[0]
    b = synth.random_coeffs(K, seed=9)

    def directions(solver):
        ps = []

        def hv(p):
            ps.append(p.copy())
            return d * p

        solver(hv, b, prec, 1e-12, 6)
        return ps

    def worst(ps):
        return max(abs(S.inner(ps[i + 1], d * ps[i])) /
                   np.sqrt(S.inner(ps[i + 1], d * ps[i + 1]) * S.inner(ps[i], d * ps[i]))
                   for i in range(len(ps) - 1))

    assert worst(directions(ML.fpcg)) < 1e-12
    assert worst(directions(gnk.pcg)) > 1e-2


def test_fpcg_with_a_fixed_preconditioner_is_pcg():
    K, alpha, s = 8, 0.0025, 2
    w = S.l_symbol(K, alpha, s)
    hv = lambda c: (w + 0.9 * (w > 0)) * c
    prec = lambda c: S.apply_Linv(c, alpha, s)
    b = synth.random_coeffs(K, seed=10)
    for eta in (0.5, 1e-3, 1e-10):
        x1, i1, _ = gnk.pcg(hv, b, prec, eta, 50)
        x2, i2, _ = ML.fpcg(hv, b, prec, eta, 50)
        assert i1 == i2
        assert rel_l2(x2, x1) < 1e-10


def test_fpcg_negative_curvature_at_first_iteration_returns_the_preconditioned_rhs():
    K = 6
    b = synth.random_coeffs(K, seed=11)
    prec = lambda c: S.apply_Linv(c, 0.0025, 2)
    x, its, neg = ML.fpcg(lambda c: -c, b, prec, 1e-6, 10)
    assert neg and its == 1
    np.testing.assert_allclose(x, prec(b))


def test_two_level_on_a_registration_problem_solves_the_coarse_system_and_scales_L_on_the_rest():
    """On a real problem: R P^{-1} a solves H_c y = R a (H_c the half-grid Gauss-Newton Hessian at
    R v~), the other modes of P^{-1} a are L~^{-1} a times one positive scale, and P^{-1} is
    positive."""
    shape, K = (16, 16, 16), 8
    I0, I1 = blob_pair(shape, K, seed=0)
    prob = Vn.Problem(I0, I1, Vn.Params(K=K, nt=4, order=1, variant=Vn.DEFSTATE))
    tl = ML.TwoLevel(prob, ML.coarse_problem(prob), inner_maxit=200, inner_tol=1e-10)
    assert tl.coarse.shape == (8, 8, 8) and tl.Kc == 4
    v = 0.3 * S.hermitian_part(synth.random_velocity_coeffs(K, 4, seed=12))
    tl.set_velocity(v)
    a = S.hermitian_part(synth.random_coeffs(K, seed=13))
    b = S.hermitian_part(synth.random_coeffs(K, seed=14))
    Pa, Pb = tl(a), tl(b)
    ra = ML.restrict_cube(a, tl.Kc)
    res = tl.coarse.hessian_matvec(ML.restrict_cube(v, tl.Kc), ML.restrict_cube(Pa, tl.Kc)) - ra
    assert np.sqrt(S.inner(res, res) / S.inner(ra, ra)) < 1e-9
    low = ML.prolong_cube(np.ones((3, tl.Kc, tl.Kc, tl.Kc)), K) > 0
    hi_P = np.where(low, 0, Pa)
    hi_L = np.where(low, 0, S.apply_Linv(a, 0.0025, 2))
    t = S.inner(hi_L, hi_P) / S.inner(hi_L, hi_L)       # one positive scale for all those modes
    assert t > 0 and rel_l2(hi_P, t * hi_L) < 1e-13
    assert S.inner(a, Pa) > 0 and S.inner(b, Pb) > 0


@pytest.mark.slow
def test_two_level_registration_descends_like_the_spectral_one():
    """Same problem, both preconditioners: the energy falls monotonically and ends within 1% of
    the spectral run (the data term dominates H at every retained mode here, so the coarse
    correction does not cut the outer iterations: measured 26 vs 27)."""
    shape, K = (16, 16, 16), 8
    I0, I1 = blob_pair(shape, K, seed=0, max_vox=2.0)
    prob = Vn.Problem(I0, I1, Vn.Params(K=K, nt=5, order=1, variant=Vn.DEFSTATE))
    _, rs = gnk.register(prob, max_gn=5, max_pcg=10)
    _, rt = gnk.register(prob, max_gn=5, max_pcg=10, two_level=5)
    assert rt.pcg_inner_total > 0 and rs.pcg_inner_total == 0
    Es = [h[0] for h in rt.history] + [rt.E]
    assert all(b <= a for a, b in zip(Es, Es[1:])), Es
    assert rt.E <= rs.E * (1 + 1e-2)
