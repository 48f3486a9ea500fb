"""Host-side pieces of the warm-start pipeline (no GPU): the reflection augmentation and the
parameter layout shared with the C network."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ON  # noqa: E402
from paper_2006_06823_b300 import warmstart as WS  # noqa: E402


def test_reflection_is_the_periodic_mirror_and_flips_the_velocity_component():
    g = np.random.default_rng(0)
    X = torch.as_tensor(g.standard_normal((2, 2, 8, 6, 4)), dtype=torch.float32)
    T = torch.as_tensor(g.standard_normal((2, 3, 4, 3, 2)), dtype=torch.float32)
    for axes in ([0], [1], [2], [0, 2], [0, 1, 2]):
        Xr, Tr = WS.reflect(X.clone(), T.clone(), axes)
        x, t = X.numpy(), T.numpy()
        xr, tr = x.copy(), t.copy()
        for a in axes:                       # axis a of a [.., z, y, x] array is dim -1 - a
            d = x.ndim - 1 - a
            n = x.shape[d]
            xr = np.take(xr, (-np.arange(n)) % n, axis=d)
            m = t.shape[d]
            tr = np.take(tr, (-np.arange(m)) % m, axis=d)
            tr[:, a] = -tr[:, a]
        np.testing.assert_array_equal(Xr.numpy(), xr)
        np.testing.assert_array_equal(Tr.numpy(), tr)
        # applying the same reflection twice is the identity
        X2, T2 = WS.reflect(Xr, Tr, axes)
        np.testing.assert_array_equal(X2.numpy(), x)
        np.testing.assert_array_equal(T2.numpy(), t)


class _FakeNet:
    def __init__(self, c):
        self.c = c
        self.num_params = sum(co * ci * 27 + co for _, ci, co in ON.layer_specs(c))


@pytest.mark.parametrize("c", [2, 16])
def test_bias_mask_matches_the_layer_list(c):
    m = WS._bias_mask(_FakeNet(c))
    off = 0
    for _, cin, cout in ON.layer_specs(c):
        assert not m[off:off + cout * cin * 27].any()
        off += cout * cin * 27
        assert m[off:off + cout].all()
        off += cout
    assert off == m.size
