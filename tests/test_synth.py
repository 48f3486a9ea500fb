"""The seeded input generators (shared by the oracle tests, the GPU tests and the benchmark):
deterministic per seed, independent across seeds, and with the documented shapes and value
distributions of the workload recipes."""
import numpy as np
import pytest

from paper_2006_06823_b300 import synth


def test_every_generator_is_a_function_of_its_seed():
    for make in (lambda s: synth.gaussian_blobs((16, 20, 24), seed=s),
                 lambda s: synth.random_velocity_coeffs(8, 6, seed=s),
                 lambda s: synth.random_field((8, 10, 12), seed=s, ncomp=2, smooth=1.0),
                 lambda s: synth.random_displacement((8, 10, 12), seed=s, max_vox=3.0),
                 lambda s: synth.add_noise(np.zeros((6, 6, 6)), seed=s)):
        a, b, c = make(3), make(3), make(4)
        assert np.array_equal(a, b)
        assert not np.array_equal(a, c)


def test_velocity_coefficients_are_hermitian_band_limited_and_decaying():
    K, K_gen = 12, 6
    c = synth.random_velocity_coeffs(K, K_gen, seed=5)
    assert c.shape == (3, K, K, K) and c.dtype == np.complex128
    # slot 0 (k = -K/2) empty; nothing outside |k| <= K_gen/2 - 1
    assert not c[:, 0].any() and not c[:, :, 0].any() and not c[:, :, :, 0].any()
    k = np.arange(K) - K // 2
    outside = np.abs(k) > K_gen // 2 - 1
    assert not c[:, outside].any() and not c[:, :, outside].any() and not c[:, :, :, outside].any()
    # c_{-k} = conj(c_k): slot j pairs with slot K - j
    j = np.arange(1, K)
    np.testing.assert_array_equal(c[:, 1:, 1:, 1:], np.conj(c[:, K - j][:, :, K - j][:, :, :, K - j]))
    # the mean of the field is real and the amplitude falls with |k|
    assert c[:, K // 2, K // 2, K // 2].imag.max() == 0
    many = np.stack([synth.random_velocity_coeffs(K, K, seed=s) for s in range(40)])
    low = np.abs(many[..., K // 2, K // 2, K // 2 + 1]).mean()
    high = np.abs(many[..., K // 2, K // 2, K // 2 + 4]).mean()
    assert high < low / 20


def test_blobs_and_phantom_follow_their_recipes():
    img = synth.gaussian_blobs((32, 32, 32), seed=0)
    assert img.min() >= 0 and img.max() <= 1 and img.max() > 0.3
    ph = synth.ellipsoid_phantom((48, 56, 48), smooth_sigma=0.0)
    assert set(np.unique(ph)) == {0.0, 0.1, 0.3, 0.5, 0.7, 0.9, 0.6}
    assert ph[24, 28, 24] == 0.6 and ph[0, 0, 0] == 0.0          # inner shell at the centre
    blurred = synth.ellipsoid_phantom((48, 56, 48))
    assert 0 <= blurred.min() and blurred.max() <= 0.9 and abs(blurred.mean() - ph.mean()) < 1e-12


def test_noise_has_variance_0_01_without_clipping():
    n = synth.add_noise(np.zeros((64, 64, 64)), seed=9)
    assert n.var() == pytest.approx(0.01, rel=0.02)
    assert abs(n.mean()) < 1e-3 and n.min() < -0.3 and n.max() > 0.3


def test_displacement_is_scaled_to_its_maximum():
    d = synth.random_displacement((10, 12, 14), seed=2, max_vox=4.5)
    assert d.shape == (3, 10, 12, 14)
    assert np.abs(d).max() == pytest.approx(4.5, rel=1e-12)
