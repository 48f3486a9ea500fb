"""Pins of the FP64 reference of the warm-start network (brute force, adjoint identities,
finite differences)."""
import numpy as np
import pytest

from oracle import cnn
from paper_2006_06823_b300 import synth


def test_conv3d_matches_explicit_loops():
    g = synth.rng(1)
    x = g.standard_normal((2, 4, 5, 3))
    w = g.standard_normal((3, 2, 27))
    b = g.standard_normal(3)
    np.testing.assert_allclose(cnn.conv3d(x, w, b), cnn.conv3d_loops(x, w, b), atol=1e-12)


def test_conv3d_input_gradient_is_the_adjoint():
    g = synth.rng(2)
    x = g.standard_normal((3, 6, 6, 6))
    y = g.standard_normal((4, 6, 6, 6))
    w = g.standard_normal((4, 3, 27))
    lhs = np.sum(cnn.conv3d(x, w) * y)
    rhs = np.sum(x * cnn.conv3d_dgrad(y, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_conv3d_weight_gradient_is_exact():
    g = synth.rng(3)
    x = g.standard_normal((2, 5, 4, 6))
    y = g.standard_normal((3, 5, 4, 6))
    dw = g.standard_normal((3, 2, 27))
    db = g.standard_normal(3)
    gw, gb = cnn.conv3d_wgrad(y, x)
    lhs = np.sum(cnn.conv3d(x, dw, db) * y)
    assert lhs == pytest.approx(np.sum(gw * dw) + np.sum(gb * db), rel=1e-12)


def test_pool_and_upsample_adjoint_pairs():
    g = synth.rng(4)
    x = g.standard_normal((2, 4, 6, 8))
    y = g.standard_normal((2, 2, 3, 4))
    assert np.sum(cnn.avgpool2(x) * y) == pytest.approx(np.sum(x * cnn.avgpool2_grad(y)), rel=1e-12)
    assert np.sum(cnn.upsample2(y) * x) == pytest.approx(np.sum(y * cnn.upsample2_grad(x)), rel=1e-12)
    np.testing.assert_allclose(cnn.avgpool2(cnn.upsample2(y)), y, atol=1e-15)


def test_network_backward_matches_central_differences():
    g = synth.rng(5)
    P = cnn.init_params(g, base_channels=2)
    x = g.standard_normal((2, 8, 8, 8))
    y, cache = cnn.forward(P, x)
    assert y.shape == (3, 4, 4, 4)
    dy = g.standard_normal(y.shape)
    grads = cnn.backward(P, cache, dy)
    h = 1e-6
    for name in ("e0a.w", "e2b.w", "d2a.w", "d1b.b", "out.w", "e3a.b"):
        d = g.standard_normal(P[name].shape)
        Pp = dict(P); Pp[name] = P[name] + h * d
        Pm = dict(P); Pm[name] = P[name] - h * d
        fd = (np.sum(cnn.forward(Pp, x)[0] * dy) - np.sum(cnn.forward(Pm, x)[0] * dy)) / (2 * h)
        an = np.sum(grads[name] * d)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)
