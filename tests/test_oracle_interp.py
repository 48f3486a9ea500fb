"""Pins of the oracle's interpolators (Sec. 3.1, Sec. 4.2) against scipy and closed forms."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import interp as I
from paper_2006_06823_b300 import synth


def _coords(shape, D):
    nz, ny, nx = shape
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([jz + D[2], jy + D[1], jx + D[0]])


@pytest.mark.parametrize("order", [1, 3])
def test_matches_scipy_periodic_spline_interpolation(order):
    shape = (9, 10, 12)
    f = synth.random_field(shape, seed=1)[0]
    D = synth.random_displacement(shape, seed=2, max_vox=6.0, smooth=1.5)
    ref = ndimage.map_coordinates(f, _coords(shape, D), order=order, mode="grid-wrap")
    np.testing.assert_allclose(I.interpolate(f, D, order), ref, atol=1e-12)


def test_prefilter_matches_scipy_spline_filter():
    f = synth.random_field((8, 11, 9), seed=3)[0]
    ref = ndimage.spline_filter(f, order=3, mode="grid-wrap")
    np.testing.assert_allclose(I.bspline_prefilter(f), ref, atol=1e-12)


@pytest.mark.parametrize("order", [1, 3])
def test_integer_offsets_reproduce_grid_values(order):
    shape = (6, 7, 8)
    f = synth.random_field(shape, seed=4)[0]
    D = np.zeros((3,) + shape)
    D[0] += 3
    D[1] -= 2
    D[2] += 9
    out = I.interpolate(f, D, order)
    np.testing.assert_allclose(out, np.roll(f, (-9, 2, -3), axis=(0, 1, 2)), atol=1e-12)
    if order == 1:
        assert np.array_equal(out, np.roll(f, (-9, 2, -3), axis=(0, 1, 2)))


def test_trilinear_exact_on_affine_data_inside_cells():
    shape = (8, 8, 8)
    nz, ny, nx = shape
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 0.3 + 0.1 * jx - 0.2 * jy + 0.05 * jz
    rng = synth.rng(5)
    D = rng.uniform(0.0, 1.0, size=(3,) + shape)
    inside = (jx < nx - 1) & (jy < ny - 1) & (jz < nz - 1)
    out = I.trilinear(f, D)
    exact = 0.3 + 0.1 * (jx + D[0]) - 0.2 * (jy + D[1]) + 0.05 * (jz + D[2])
    np.testing.assert_allclose(out[inside], exact[inside], atol=1e-13)
    g = I.trilinear_grad(f, D)
    np.testing.assert_allclose(g[0][inside], 0.1, atol=1e-13)
    np.testing.assert_allclose(g[1][inside], -0.2, atol=1e-13)
    np.testing.assert_allclose(g[2][inside], 0.05, atol=1e-13)


def test_cubic_interpolation_is_fourth_order():
    errs = []
    for n in (16, 32, 64):
        shape = (4, 4, n)
        x = 2 * np.pi * np.arange(n) / n
        f = np.broadcast_to(np.sin(x), shape).copy()
        D = np.zeros((3,) + shape)
        D[0] += 0.37
        exact = np.broadcast_to(np.sin(2 * np.pi * (np.arange(n) + 0.37) / n), shape)
        errs.append(np.abs(I.interpolate(f, D, 3) - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > 3.7).all(), rates


@pytest.mark.parametrize("order", [1, 3])
def test_interpolant_gradient_matches_finite_differences(order):
    shape = (7, 8, 9)
    f = synth.random_field(shape, seed=6, smooth=1.0)[0]
    rng = synth.rng(7)
    D = rng.uniform(0.2, 0.8, size=(3,) + shape)  # away from cell faces (trilinear kinks)
    g = I.interpolate_grad(f, D, order)
    h = 1e-6
    for a in range(3):
        Dp, Dm = D.copy(), D.copy()
        Dp[a] += h
        Dm[a] -= h
        fd = (I.interpolate(f, Dp, order) - I.interpolate(f, Dm, order)) / (2 * h)
        np.testing.assert_allclose(g[a], fd, atol=1e-7)


def test_prefilter_then_sample_is_identity():
    f = synth.random_field((6, 9, 7), seed=8)[0]
    c = I.bspline_prefilter(f)
    np.testing.assert_allclose(I.cubic_coeffs_eval(c, np.zeros((3,) + f.shape)), f, atol=1e-12)
