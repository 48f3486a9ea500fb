"""Pins of the oracle's PCG and Gauss-Newton driver (Sec. 2.1-2.2, Eqs. 7-8, 13-14)."""
import numpy as np
import pytest

from oracle import gnk
from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import rel_l2


def test_pcg_matches_closed_form_on_a_diagonal_operator():
    K, alpha, s, shift = 8, 0.0025, 2, 0.7
    w = S.l_symbol(K, alpha, s)
    b = synth.random_coeffs(K, seed=1)
    hv = lambda c: (w + shift * (w > 0)) * c
    prec = lambda c: S.apply_Linv(c, alpha, s)
    x, its, neg = gnk.pcg(hv, b, prec, 1e-13, 200)
    exact = np.where(w > 0, b / np.where(w > 0, w + shift, 1), 0)
    np.testing.assert_allclose(x, exact, atol=1e-12)
    assert not neg
    # exact preconditioner: one iteration
    x1, its1, _ = gnk.pcg(lambda c: w * c, b, prec, 1e-12, 10)
    assert its1 == 1
    np.testing.assert_allclose(x1, np.where(w > 0, b / np.where(w > 0, w, 1), 0), atol=1e-14)


def test_pcg_negative_curvature_at_first_iteration_returns_preconditioned_gradient():
    K = 6
    b = synth.random_coeffs(K, seed=2)
    prec = lambda c: S.apply_Linv(c, 0.0025, 2)
    x, its, neg = gnk.pcg(lambda c: -c, b, prec, 1e-6, 10)
    assert neg and its == 1
    np.testing.assert_allclose(x, prec(b))


@pytest.mark.slow
def test_gauss_newton_decreases_energy_monotonically():
    N, K = 16, 8
    shape = (N, N, N)
    I1 = synth.gaussian_blobs(shape, seed=0)
    p = Vn.Params(K=K, nt=5, order=1, variant=Vn.DEFSTATE, sigma2=0.01)
    vgen = synth.random_velocity_coeffs(K, 8, seed=1)
    base = Vn.Problem(I1, I1, p)
    _, V, _ = base.velocity(vgen)
    I0 = SL.sl_transport(I1, V * (2.0 / np.abs(V).max()), 10, +1, 1)
    prob = Vn.Problem(I0, I1, p)
    v, rep = gnk.register(prob, max_gn=4, max_pcg=5)
    Es = [h[0] for h in rep.history] + [rep.E]
    assert all(b <= a for a, b in zip(Es, Es[1:])), Es
    assert rep.E < 0.5 * rep.E0
    assert rep.grad_rel_l2 < 0.3
    assert rep.mse_rel < 0.5


class _Quadratic:
    """E(v) = 1/2 <v - v*, A (v - v*)> with A = diag(w_k + shift_k) on the retained set: the
    Gauss-Newton driver's model problem (gradient A (v - v*), Hessian A, exact everywhere)."""

    def __init__(self, K, seed, shift=3.0, fail_line_search=False):
        self.p = Vn.Params(K=K)
        w = S.l_symbol(K, self.p.alpha, self.p.s)
        rng = np.random.default_rng(seed)
        self.a = np.where(w > 0, w + shift * rng.random(w.shape), 0.0)
        self.vstar = synth.random_coeffs(K, seed) * 0.3
        self.fail = fail_line_search

    def _E(self, v):
        d = v - self.vstar
        return 0.5 * S.inner(d, self.a * d)

    def objective(self, v):
        E = self._E(v) + (1.0 if self.fail and np.any(v) else 0.0)
        return E, 0.0, E, None

    def gradient(self, v):
        E = self._E(v)
        return E, 0.0, E, self.a * (v - self.vstar)

    def hessian_matvec(self, v, c):
        return self.a * c

    def mse_rel(self, m1):
        return 0.0


def test_gauss_newton_on_a_quadratic_meets_each_forcing_term_and_converges():
    """For a quadratic, a full step leaves the PCG residual as the next gradient, so
    ||g_{n+1}|| <= eta_n ||g_n|| with eta_n = min(0.5, sqrt(||g_n|| / ||g_0||)) and the Armijo
    test accepts eps = 1 (CG's iterate satisfies <dv, A dv> = -<g, dv>): the driver's forcing,
    line search and stopping rule in one closed-form check."""
    prob = _Quadratic(8, seed=21)
    v, rep = gnk.register(prob, max_gn=20, max_pcg=50, gtol=1e-9)
    assert rep.stop_reason == gnk.STOP_GTOL
    assert rel_l2(v, prob.vstar) < 1e-8
    ratios = [h[1] for h in rep.history]        # ||g_n|| / ||g_0||, the last one at the stop
    assert ratios[-1] == rep.grad_rel_l2 <= 1e-9
    for n in range(len(ratios) - 1):
        eta = min(0.5, np.sqrt(ratios[n]))
        # (away from rounding: the FP64 residual floor is ~1e-13 of ||g_0||)
        assert ratios[n + 1] <= eta * ratios[n] * (1 + 1e-9) + 1e-12, (n, ratios)
    Es = [h[0] for h in rep.history] + [rep.E]
    assert all(b <= a for a, b in zip(Es, Es[1:]))
    assert rep.gn_iters == len(rep.history) - 1


def test_gauss_newton_stops_at_the_iteration_cap_and_on_a_failed_line_search():
    prob = _Quadratic(6, seed=22)
    v, rep = gnk.register(prob, max_gn=1, max_pcg=2, gtol=1e-12)
    assert rep.stop_reason == gnk.STOP_MAXIT and rep.gn_iters == 1 and 1 <= rep.pcg_iters_total <= 2
    stuck = _Quadratic(6, seed=22, fail_line_search=True)
    v, rep = gnk.register(stuck, max_gn=5, max_pcg=5, gtol=1e-12)
    assert rep.stop_reason == gnk.STOP_LINESEARCH and rep.gn_iters == 0
    assert not np.any(v)


class _ScaledQuadratic(_Quadratic):
    """A = 2 L~ (so one preconditioned CG step solves exactly) and a Hessian model that
    underestimates A tenfold: the Newton step comes out 10x too long and the line search must
    backtrack."""

    def __init__(self, K, seed):
        super().__init__(K, seed)
        self.a = 2.0 * S.l_symbol(K, self.p.alpha, self.p.s)

    def hessian_matvec(self, v, c):
        return 0.1 * self.a * c


def test_line_search_halves_to_the_first_armijo_step():
    """From v = 0 the step is dv = 10 v*; E(eps dv) = (1 - 10 eps)^2 E(0) and Armijo with
    constant 1e-4 admits eps <= 0.19998, so halving from 1 accepts eps = 1/8: E(v_1) = E(0)/16
    exactly (a quarter-step halving would stop at 1/16 with E = (3/8)^2 E(0))."""
    prob = _ScaledQuadratic(8, seed=23)
    v, rep = gnk.register(prob, max_gn=1, max_pcg=5, gtol=1e-12)
    assert rep.pcg_iters_total == 1 and rep.gn_iters == 1
    assert rep.E == pytest.approx(rep.E0 / 16, rel=1e-12)
    assert rel_l2(v, 1.25 * prob.vstar) < 1e-12
