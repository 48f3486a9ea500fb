"""Pins of the non-stationary oracle (ProblemNS) for the three variants: reduction to the
stationary problem, exact two-field characteristics, central differences of the energy,
symmetry and positivity of the Gauss-Newton Hessian, and a descending registration."""
import numpy as np
import pytest

from oracle import gnk
from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth
from _problems import blob_pair, voxel_velocity


VARIANTS = [Vn.DEFSTATE, Vn.IMAGE, Vn.STATE]


def problems(shape=(16, 16, 16), K=8, nt=4, order=1, variant=Vn.DEFSTATE):
    I0, I1 = blob_pair(shape, K, seed=0, order=order)
    p = Vn.Params(K=K, nt=nt, order=order, variant=variant)
    return Vn.Problem(I0, I1, p), Vn.ProblemNS(I0, I1, p)


def stack(K, nt, seed, scale):
    return np.stack([synth.random_velocity_coeffs(K, K, seed=seed + j) * scale for j in range(nt + 1)])


def test_two_field_offsets_reduce_to_the_stationary_ones():
    shape = (12, 10, 8)
    V = synth.random_displacement(shape, seed=1, max_vox=1.5)
    for direction in (+1, -1):
        a = SL.departure_offsets_ns(V, V, 0.1, direction, 1)
        b = SL.departure_offsets(V, 0.1, direction, 1)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("order", [1, 3])
def test_equal_nodes_reduce_to_the_stationary_problem(order, variant):
    st, ns = problems(order=order, variant=variant)
    K, nt = st.p.K, st.p.nt
    vt = synth.random_velocity_coeffs(K, K, seed=3) * 0.5
    vts = np.stack([vt] * (nt + 1))
    E, Er, Ed, g = st.gradient(vt)
    En, Ern, Edn, gn = ns.gradient(vts)
    assert En == pytest.approx(E, rel=1e-12) and Ern == pytest.approx(Er, rel=1e-12)
    gsum = sum(w * gj for w, gj in zip(ns.tw, gn))
    np.testing.assert_allclose(gsum, g, atol=1e-12 * np.abs(g).max())
    dv = synth.random_coeffs(K, seed=4) * 0.1
    H = st.hessian_matvec(vt, dv)
    Hn = ns.hessian_matvec(vts, np.stack([dv] * (nt + 1)))
    Hsum = sum(w * hj for w, hj in zip(ns.tw, Hn))
    np.testing.assert_allclose(Hsum, H, atol=1e-12 * np.abs(H).max())


# |fd - <g, e>_w| against |g|_w |e|_w, cubic interpolation: measured 5.7e-4 (deformation
# state), 2.2e-3 (image), 1.4e-3 (state equation); Hessian asymmetry 3.9e-4, 4.6e-4, 2.9e-3
FD_TOL = {Vn.DEFSTATE: 2e-3, Vn.IMAGE: 4e-3, Vn.STATE: 3e-3}


@pytest.mark.parametrize("variant", VARIANTS)
def test_gradient_matches_central_differences(variant):
    _, ns = problems(order=3, variant=variant)
    K, nt = ns.p.K, ns.p.nt
    vts = stack(K, nt, 10, 0.4)
    g = ns.gradient(vts)[3]
    h = 1e-3
    for seed in (30, 40):
        e = stack(K, nt, seed, 0.05)
        fd = (ns.objective(vts + h * e)[0] - ns.objective(vts - h * e)[0]) / (2 * h)
        an = ns.inner(g, e)
        scale = np.sqrt(ns.inner(g, g) * ns.inner(e, e))
        assert abs(fd - an) <= FD_TOL[variant] * scale, (fd, an, scale)


@pytest.mark.parametrize("variant", VARIANTS)
def test_hessian_is_nearly_symmetric_and_positive(variant):
    _, ns = problems(order=3, variant=variant)
    K, nt = ns.p.K, ns.p.nt
    vts = stack(K, nt, 50, 0.3)
    a = stack(K, nt, 70, 0.1)
    b = stack(K, nt, 90, 0.1)
    Ha, Hb = ns.hessian_matvec(vts, a), ns.hessian_matvec(vts, b)
    x, y = ns.inner(b, Ha), ns.inner(Hb, a)
    aHa, bHb = ns.inner(a, Ha), ns.inner(b, Hb)
    assert aHa > 0 and bHb > 0
    assert abs(x - y) <= 2e-2 * np.sqrt(aHa * bHb), (x, y)


@pytest.mark.parametrize("variant", VARIANTS)
def test_registration_descends(variant):
    _, ns = problems(variant=variant)
    v, rep = gnk.register(ns, max_gn=3, max_pcg=5)
    Es = [h[0] for h in rep.history]
    assert all(b < a for a, b in zip(Es, Es[1:]))
    assert rep.E < 0.7 * rep.E0
    assert v.shape == (ns.p.nt + 1, 3, ns.p.K, ns.p.K, ns.p.K)
