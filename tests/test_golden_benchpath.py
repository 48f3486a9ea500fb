"""The stored oracle results of the bench-path parity workload (``tests/golden/``, written by
``tests/golden/make_benchpath.py`` from oracle calls only) against the live FP64 oracle where
that is cheap on the host: the energy of the noise-free trilinear case (one state sweep at
96 x 112 x 96), the curvature <p, Hp> of every case from its stored gradient and product
(p = L~^{-1}(-g), the first PCG direction), and the whole trilinear registration of the 32^3
pair. A change of the oracle's arithmetic that leaves these files stale fails
here; the expensive gradients and products themselves are regenerated by the script."""
import json
import os

import numpy as np
import pytest

from _problems import BENCH_K, bench_phantom_problem, bench_velocity, first_direction, \
    small_phantom_problem
from oracle import gnk, spectral as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = [(1, 3, False), (1, 3, True), (3, 2, True)]


def _stored(order, nt, noisy):
    kind = "noisy" if noisy else "clean"
    return np.load(os.path.join(GOLDEN, f"benchpath_o{order}_nt{nt}_{kind}.npz"))


@pytest.mark.parametrize("order,nt,noisy", CASES)
def test_stored_direction_and_curvature_follow_from_the_stored_gradient_and_product(order, nt, noisy):
    ref = _stored(order, nt, noisy)
    g, Hp = ref["g"], ref["Hp"]
    for a in (g, Hp):
        assert a.dtype == np.complex64 and a.shape == (3, BENCH_K, BENCH_K, BENCH_K)
        assert np.isfinite(a).all()
    # L~ with the paper's alpha = 0.0025 and s = 2: the direction is the preconditioned -g
    p = first_direction(g, 0.0025, 2)
    pHp = S.inner(p, Hp.astype(np.complex128))
    assert pHp == pytest.approx(float(ref["pHp"]), rel=1e-6)
    assert float(ref["pHp"]) > 0
    # a Gauss-Newton product is L~ p plus a positive semidefinite data term
    assert pHp >= S.inner(p, S.apply_L(p, 0.0025, 2)) * (1 - 1e-6)


@pytest.mark.slow
def test_stored_energy_of_the_clean_trilinear_case_is_the_live_oracles():
    prob = bench_phantom_problem(1, 3, noisy=False)
    assert prob.p.alpha == 0.0025 and prob.p.s == 2
    E = prob.objective(bench_velocity())[0]
    assert float(_stored(1, 3, False)["E"]) == pytest.approx(E, rel=1e-12)


@pytest.mark.slow
def test_stored_trilinear_registration_is_the_live_oracles():
    with open(os.path.join(GOLDEN, "benchpath_registration_o1.json")) as f:
        ref = json.load(f)
    cfg = ref["config"]
    prob = small_phantom_problem(1, nt=cfg["nt"])
    _, rep = gnk.register(prob, max_gn=cfg["max_gn"], max_pcg=cfg["max_pcg"])
    assert (rep.gn_iters, rep.pcg_iters_total, rep.stop_reason) == \
        (ref["gn_iters"], ref["pcg_iters_total"], ref["stop_reason"])
    assert rep.E == pytest.approx(ref["E"], rel=1e-12)
    assert rep.grad_rel_l2 == pytest.approx(ref["grad_rel_l2"], rel=1e-10)
    assert len(rep.history) == len(ref["history"])
    for (E, r), (E_ref, r_ref) in zip(rep.history, ref["history"]):
        assert E == pytest.approx(E_ref, rel=1e-12) and r == pytest.approx(r_ref, rel=1e-10)
