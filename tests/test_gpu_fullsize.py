"""Parity at the paper-scale grid (192 x 224 x 192, K = 32) in the benchmark's launch
configuration, on outputs the oracle computes one by one (sampled modes and voxels) or on
a single full-grid step."""
import numpy as np
import pytest

from oracle import sl as SL
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

SHAPE = (192, 224, 192)   # nz, ny, nx
K = 32


def _coords():
    nz, ny, nx = SHAPE
    return (2 * np.pi * np.arange(nx) / nx, 2 * np.pi * np.arange(ny) / ny,
            2 * np.pi * np.arange(nz) / nz)


def test_projection_sampled_modes():
    f = synth.random_field(SHAPE, seed=31)[0]
    c = L.bl_project(torch.as_tensor(f, dtype=torch.float32, device="cuda"), K)[0].cpu().numpy()
    xs, ys, zs = _coords()
    rng = synth.rng(32)
    h = K // 2
    modes = [(h, h, h), (1, 1, 1), (K - 1, K - 1, K - 1), (h, 1, K - 1)]
    modes += [tuple(rng.integers(1, K, 3)) for _ in range(8)]
    for jz, jy, jx in modes:
        kx, ky, kz = jx - h, jy - h, jz - h
        # the definition: mean over voxels of f e^{-i k.x}, summed one mode at a time
        ex = np.exp(-1j * kx * xs)[None, None, :]
        ey = np.exp(-1j * ky * ys)[None, :, None]
        ez = np.exp(-1j * kz * zs)[:, None, None]
        ref = np.mean(f * ex * ey * ez)
        assert abs(c[jz, jy, jx] - ref) < 2e-6 * max(abs(ref), np.abs(f).mean() * 1e-2), (jz, jy, jx)


def test_inclusion_sampled_voxels():
    c = synth.random_coeffs(K, seed=33, ncomp=1, decay_power=0.5)[0]
    f = L.bl_include(torch.as_tensor(c.astype(np.complex64), device="cuda"), SHAPE)[0].cpu().numpy()
    rng = synth.rng(34)
    nz, ny, nx = SHAPE
    idx = np.stack([rng.integers(0, n, 300) for n in (nz, ny, nx)], 1)
    h = K // 2
    k = np.arange(K) - h
    sel = np.argwhere(np.ones((K, K, K), bool)[1:, 1:, 1:]) + 1
    coef = c[sel[:, 0], sel[:, 1], sel[:, 2]]
    kz, ky, kx = k[sel[:, 0]], k[sel[:, 1]], k[sel[:, 2]]
    for z, y, x in idx:
        phase = kx * 2 * np.pi * x / nx + ky * 2 * np.pi * y / ny + kz * 2 * np.pi * z / nz
        ref = np.real(np.sum(coef * np.exp(1j * phase)))
        assert abs(f[z, y, x] - ref) < 2e-6 * np.abs(c).sum() ** 0.5 + 1e-6 * abs(ref)


def test_transport_one_full_grid_step():
    V = synth.random_displacement(SHAPE, seed=35, max_vox=8.0, smooth=6.0)
    f = synth.ellipsoid_phantom(SHAPE)
    Vt = torch.as_tensor(V, dtype=torch.float32, device="cuda")
    ft = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    out = L.sl_transport(Vt, ft, 1, L.FORWARD, L.INTERP_LINEAR).cpu().numpy()
    ref = SL.sl_transport(f, V, 1, +1, 1)
    assert rel_l2(out, ref) < 1e-5
