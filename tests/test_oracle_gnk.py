"""Pins of the oracle's PCG and Gauss-Newton driver (Sec. 2.1-2.2, Eqs. 7-8, 13-14)."""
import numpy as np
import pytest

from oracle import gnk
from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth


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
