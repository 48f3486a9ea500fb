"""Pins of the oracle's band-limited operators (Sec. 2.2) against brute force and closed forms."""
import numpy as np
import pytest

from oracle import spectral as S
from paper_2006_06823_b300 import synth


SHAPES = [(8, 8, 8), (6, 10, 12), (9, 7, 11)]


@pytest.mark.parametrize("shape", SHAPES)
def test_project_matches_brute_force_dft(shape):
    f = synth.random_field(shape, seed=3)[0]
    c = S.project(f, 6)
    np.testing.assert_allclose(c, S.project_direct(f, 6), atol=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
def test_include_matches_brute_force_sum(shape):
    c = synth.random_coeffs(6, seed=4, ncomp=1)[0]
    np.testing.assert_allclose(S.include(c, shape), S.include_direct(c, shape), atol=1e-12)


def test_hermitian_cube_gives_real_field():
    c = synth.random_coeffs(8, seed=5, ncomp=1)[0]
    full = S.include_direct(c, (10, 12, 14))
    # include_direct returns the real part; the imaginary part must vanish for Hermitian c
    nz, ny, nx = 10, 12, 14
    k = S.mode_numbers(8)
    zz, yy, xx = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                             2 * np.pi * np.arange(nx) / nx, indexing="ij")
    im = np.zeros((nz, ny, nx))
    for jz in range(1, 8):
        for jy in range(1, 8):
            for jx in range(1, 8):
                im += np.imag(c[jz, jy, jx] * np.exp(1j * (k[jx] * xx + k[jy] * yy + k[jz] * zz)))
    assert np.abs(im).max() < 1e-12
    assert np.isfinite(full).all()


@pytest.mark.parametrize("shape", SHAPES)
def test_projection_is_idempotent_and_left_inverse(shape):
    f = synth.random_field(shape, seed=6)[0]
    c = S.project(f, 6)
    np.testing.assert_allclose(S.project(S.include(c, shape), 6), c, atol=1e-14)
    g = synth.random_coeffs(6, seed=7, ncomp=1)[0]
    np.testing.assert_allclose(S.project(S.include(g, shape), 6), g, atol=1e-14)


def test_parseval_and_adjointness():
    shape = (10, 12, 8)
    c = synth.random_coeffs(8, seed=8, ncomp=1)[0]
    f = S.include(c, shape)
    assert np.mean(f * f) == pytest.approx(np.sum(np.abs(c) ** 2), rel=1e-12)
    h = synth.random_field(shape, seed=9)[0]
    assert S.inner(S.project(h, 8), c) == pytest.approx(np.mean(h * f), rel=1e-12)


def test_single_cosine_mode_maps_to_one_half_at_plus_minus_k():
    shape = (12, 10, 8)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    f = np.cos(2 * x - 1 * y + 3 * z)
    K = 8
    c = S.project(f, K)
    h = K // 2
    expect = np.zeros((K, K, K), complex)
    expect[3 + h, -1 + h, 2 + h] = 0.5
    expect[-3 + h, 1 + h, -2 + h] = 0.5
    np.testing.assert_allclose(c, expect, atol=1e-14)


def test_spectral_derivatives_are_exact_on_band_limited_functions():
    shape = (12, 14, 10)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    f = np.sin(2 * x + 3 * y) + 0.5 * np.cos(x - 2 * z)
    c = S.project(f, 8)
    np.testing.assert_allclose(S.include(S.deriv(c, 0), shape),
                               2 * np.cos(2 * x + 3 * y) - 0.5 * np.sin(x - 2 * z), atol=1e-12)
    np.testing.assert_allclose(S.include(S.deriv(c, 1), shape), 3 * np.cos(2 * x + 3 * y),
                               atol=1e-12)
    np.testing.assert_allclose(S.include(S.deriv(c, 2), shape), 1.0 * np.sin(x - 2 * z),
                               atol=1e-12)
    vec = np.stack([S.project(np.sin(x), 8), S.project(np.cos(y), 8), S.project(np.sin(2 * z), 8)])
    np.testing.assert_allclose(S.include(S.div(vec), shape),
                               np.cos(x) - np.sin(y) + 2 * np.cos(2 * z), atol=1e-12)
    J = S.include(S.jacobian(vec), shape)
    np.testing.assert_allclose(J[1, 1], -np.sin(y), atol=1e-12)
    np.testing.assert_allclose(J[0, 1], 0.0, atol=1e-12)


def test_regulariser_symbol_closed_form():
    K, alpha, s = 8, 0.0025, 2
    w = S.l_symbol(K, alpha, s)
    h = K // 2
    assert w[h, h, h] == 1.0
    assert w[h + 1, h - 2, h + 3] == pytest.approx((1 + alpha * (9 + 4 + 1)) ** 2)
    assert w[0].max() == 0.0 and w[:, 0].max() == 0.0 and w[:, :, 0].max() == 0.0
    c = synth.random_coeffs(K, seed=10, ncomp=1)[0]
    np.testing.assert_allclose(S.apply_Linv(S.apply_L(c, alpha, s), alpha, s), c, atol=1e-15)


def test_hermitian_part_fixes_hermitian_cubes():
    c = synth.random_coeffs(8, seed=11, ncomp=3)
    np.testing.assert_allclose(S.hermitian_part(c), c, atol=1e-15)


def test_bspline_symbol_matches_prefilter_on_band_limited_fields():
    from oracle import interp as I
    shape = (10, 12, 14)
    c = synth.random_coeffs(8, seed=12, ncomp=1)[0]
    lhs = I.bspline_prefilter(S.include(c, shape))
    rhs = S.include(c / S.bspline_symbol(8, shape), shape)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
