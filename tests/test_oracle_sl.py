"""Pins of the oracle's SL-RK steps (Sec. 3, Table 1) against exact solutions and invariants."""
import numpy as np
import pytest

from oracle import sl as SL
from oracle import spectral as S
from paper_2006_06823_b300 import synth


@pytest.mark.parametrize("order", [1, 3])
def test_zero_velocity_is_the_identity(order):
    shape = (6, 8, 10)
    f = synth.random_field(shape, seed=1)[0]
    V = np.zeros((3,) + shape)
    D = SL.departure_offsets(V, 0.1, +1, order)
    assert np.array_equal(D, np.zeros_like(D))
    out = SL.sl_transport(f, V, 10, +1, order)
    if order == 1:
        assert np.array_equal(out, f)
    else:
        np.testing.assert_allclose(out, f, atol=1e-12)


@pytest.mark.parametrize("order", [1, 3])
def test_constant_integer_velocity_is_an_exact_roll(order):
    shape = (8, 6, 10)
    f = synth.random_field(shape, seed=2)[0]
    nt = 4
    V = np.zeros((3,) + shape)
    V[0] += 2 * nt      # 2 voxels per step along x
    V[2] -= 1 * nt      # -1 voxel per step along z
    out = SL.sl_transport(f, V, nt, +1, order)
    np.testing.assert_allclose(out, np.roll(f, (-nt, 2 * nt), axis=(0, 2)), atol=1e-12)
    back = SL.sl_transport(f, V, nt, -1, order)
    np.testing.assert_allclose(back, np.roll(f, (nt, -2 * nt), axis=(0, 2)), atol=1e-12)


def test_shear_flow_departure_points_are_exact():
    shape = (4, 16, 8)
    ny = shape[1]
    y = np.arange(ny)
    V = np.zeros((3,) + shape)
    V[0] = (3.0 * np.sin(2 * np.pi * y / ny))[None, :, None]
    for order in (1, 3):
        D = SL.departure_offsets(V, 0.25, +1, order)
        np.testing.assert_allclose(D[0], -0.25 * V[0], atol=1e-13)
        np.testing.assert_allclose(D[1:], 0.0, atol=1e-15)


@pytest.mark.parametrize("order", [1, 3])
def test_constant_fields_are_invariant(order):
    shape = (8, 8, 8)
    V = synth.random_displacement(shape, seed=3, max_vox=5.0)
    c = np.full(shape, 0.7)
    out = SL.sl_transport(c, V, 5, +1, order)
    assert np.abs(out - 0.7).max() <= 1e-15 * 8


def test_deformation_state_with_constant_velocity_reaches_v_exactly():
    shape = (8, 10, 6)
    K = 6
    vt = np.zeros((3, K, K, K), complex)
    h = K // 2
    vt[:, h, h, h] = [0.3, -0.2, 0.5]           # the k = 0 mode: a constant field
    v = S.include(vt, shape)
    V = v * (np.array([6, 10, 8.0]) / (2 * np.pi))[:, None, None, None]
    nt = 7
    dt = 1.0 / nt
    D = SL.departure_offsets(V, dt, +1, 1)
    u = np.zeros_like(vt)
    for _ in range(nt):
        u = SL.bl_heun_source_step(u, D, v, v, dt, 1, shape, K)
    np.testing.assert_allclose(u, vt, atol=1e-14)


def _mass_drift(d_sign, order, nt=8):
    shape = (16, 16, 16)
    K = 8
    vt = synth.random_velocity_coeffs(K, 6, seed=4)
    v = S.include(vt, shape)
    vt = vt * (3.0 / np.abs(v * 16 / (2 * np.pi)).max())
    V = S.include(vt, shape) * (16 / (2 * np.pi))
    d = d_sign * S.include(S.div(vt), shape)
    rho = synth.random_field(shape, seed=5, smooth=2.0)[0] + 1.0
    dt = 1.0 / nt
    Dp = SL.departure_offsets(V, dt, -1, order)
    r = rho.copy()
    for _ in range(nt):
        r = SL.heun_divergence_step(r, Dp, d, dt, order)
    return abs(r.sum() - rho.sum()) / rho.sum()


@pytest.mark.parametrize("order,tol", [(1, 2e-3), (3, 1e-4)])
def test_continuity_adjoint_conserves_mass(order, tol):
    """-d_t rho - div(rho v) = 0 keeps sum(rho); SL conserves it up to interpolation error."""
    assert _mass_drift(+1.0, order) < tol
    # the same step with the divergence term's sign flipped must drift far more
    assert _mass_drift(-1.0, order) > 10 * tol


def test_forward_then_reverse_transport_returns_the_image():
    shape = (16, 16, 16)
    f = synth.gaussian_blobs(shape, seed=6)
    V = synth.random_displacement(shape, seed=7, max_vox=2.0, smooth=4.0)
    fwd = SL.sl_transport(f, V, 8, +1, 3)
    back = SL.sl_transport(fwd, -V, 8, +1, 3)
    assert np.abs(back - f).max() < 0.05 * np.abs(f).max()
    assert np.abs(fwd - f).max() > 0.1 * np.abs(f).max()


def test_divergence_free_constant_adjoint_step_is_pure_transport():
    shape = (6, 8, 10)
    f = synth.random_field(shape, seed=8)[0]
    V = synth.random_displacement(shape, seed=9, max_vox=2.0)
    D = SL.departure_offsets(V, 0.2, -1, 1)
    out = SL.heun_divergence_step(f, D, np.zeros(shape), 0.2, 1)
    np.testing.assert_allclose(out, SL.transport_step(f, D, 1), atol=1e-15)
