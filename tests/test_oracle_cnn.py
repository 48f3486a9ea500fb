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


def test_round_bf16_exact_values():
    """bfloat16 keeps 8 significant bits: 1 + 2^-7 is representable, 1 + 2^-8 is the tie
    between 1 and 1 + 2^-7 and rounds to the even one (1), 1 + 3 * 2^-9 rounds up."""
    x = np.array([1.0, 1 + 2.0 ** -7, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, 1 + 3 * 2.0 ** -8,
                  -2.5, 0.0, 3.0e38, 1e-40])
    want = np.array([1.0, 1 + 2.0 ** -7, 1.0, 1 + 2.0 ** -7, 1 + 2.0 ** -6, -2.5, 0.0,
                     2.99e38, 1e-40])
    got = cnn.round_bf16(x)
    np.testing.assert_array_equal(got[:7], want[:7])
    assert abs(got[7] - 3.0e38) <= 3.0e38 * 2.0 ** -8          # nearest, not truncated
    assert abs(got[8] - 1e-40) <= 2.0 ** -133                  # subnormal spacing
    # rounding error bound u = 2^-8 on random normal values
    r = np.random.default_rng(0).standard_normal(10000) * 100
    assert np.max(np.abs(cnn.round_bf16(r) - r) / np.abs(r)) <= 2.0 ** -8


def test_bf16_storage_network_is_close_to_exact():
    """The bf16-storage model differs from the FP64 network by roundings alone; with no
    roundings possible (every activation already a bfloat16 number) the two agree."""
    g = np.random.default_rng(6)
    P = cnn.init_params(g, 2)
    x = g.random((2, 8, 8, 8))
    y, _ = cnn.forward(P, x)
    yb, _ = cnn.forward(P, x, storage="bf16")
    assert 0 < np.linalg.norm(yb - y) / np.linalg.norm(y) < 0.05
    # zero weights except biases that are bfloat16 numbers: every activation is exact
    Z = {k: np.zeros_like(v) for k, v in P.items()}
    for k in Z:
        if k.endswith(".b"):
            Z[k] = cnn.round_bf16(g.random(Z[k].shape))
    y0, _ = cnn.forward(Z, x)
    y0b, _ = cnn.forward(Z, x, storage="bf16")
    np.testing.assert_array_equal(y0, y0b)
