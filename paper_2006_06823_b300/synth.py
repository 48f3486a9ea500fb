"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and builds phantom images. It holds none of the
registration method's arithmetic: no band-limited projection or inclusion, no transport,
no interpolation. Warping a phantom by a velocity (which *is* the method) is left to the
caller: the FP64 oracle in the parity tests, the library's own transport in the benchmark.

Array layout everywhere: images ``[nz][ny][nx]`` (x fastest), vector fields
``[3][nz][ny][nx]`` with component 0 = x, 1 = y, 2 = z, band-limited coefficient cubes
``[3][K][K][K]`` indexed ``[comp][jz][jy][jx]`` with wavenumber ``k = j - K/2``.

The phantoms stand in for the paper's brain MRI volumes (Sec. 4.2: 180x210x180 voxels,
intensities scaled to [0, 1]); no public dataset is reproduced.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def rng(seed: int) -> np.random.Generator:
    """PCG64 stream for one seed; every input in this project is drawn from one."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _grid(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def blob_params(shape=(32, 32, 32), seed=0, n_blobs=8):
    """Random draws of ``gaussian_blobs``: a list of (centre (x, y, z), width, amplitude).

    Centres ~ U[8, 24] voxels per axis, widths ~ U[3, 6] voxels, amplitudes ~ U[0.3, 1],
    scaled by N/32 on grids other than 32^3."""
    g = rng(seed)
    nz, ny, nx = shape
    scale = np.array([nx, ny, nz], dtype=np.float64) / 32.0
    out = []
    for _ in range(n_blobs):
        c = g.uniform(8.0, 24.0, size=3) * scale
        s = g.uniform(3.0, 6.0) * scale.mean()
        a = g.uniform(0.3, 1.0)
        out.append((c, s, a))
    return out


def gaussian_blobs(shape=(32, 32, 32), seed=0, n_blobs=8):
    """Fixed image of the small workload: the sum of the ``blob_params`` Gaussians, clipped
    to [0, 1]. float64."""
    x, y, z = _grid(shape)
    img = np.zeros(shape)
    for c, s, a in blob_params(shape, seed, n_blobs):
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        img += a * np.exp(-r2 / (2.0 * s * s))
    return np.clip(img, 0.0, 1.0)


def gaussian_blobs_device(shape, seed, device, n_blobs=8):
    """``gaussian_blobs`` evaluated on a torch device in float32 (same random draws), for
    generating many large phantoms without host work."""
    import torch
    nz, ny, nx = shape
    z = torch.arange(nz, dtype=torch.float32, device=device).view(nz, 1, 1)
    y = torch.arange(ny, dtype=torch.float32, device=device).view(1, ny, 1)
    x = torch.arange(nx, dtype=torch.float32, device=device).view(1, 1, nx)
    img = torch.zeros(shape, dtype=torch.float32, device=device)
    for c, s, a in blob_params(shape, seed, n_blobs):
        r2 = (x - float(c[0])) ** 2 + (y - float(c[1])) ** 2 + (z - float(c[2])) ** 2
        img += float(a) * torch.exp(r2 * float(-1.0 / (2.0 * s * s)))
    return img.clamp_(0.0, 1.0)


ELLIPSOID_SEMI_AXES = (0.42, 0.45, 0.40)          # fractions of (nx, ny, nz)
ELLIPSOID_SHELLS = (1.0, 0.85, 0.7, 0.55, 0.4, 0.25)
ELLIPSOID_LEVELS = (0.1, 0.3, 0.5, 0.7, 0.9, 0.6)  # outer -> inner


def ellipsoid_phantom(shape=(192, 224, 192), smooth_sigma=1.0):
    """Brain-like phantom of the paper-scale workload (no noise; see ``add_noise``).

    Six nested ellipsoidal shells centred in the volume, semi-axes
    (0.42, 0.45, 0.40) * N * {1, 0.85, 0.7, 0.55, 0.4, 0.25}, intensities
    {0.1, 0.3, 0.5, 0.7, 0.9, 0.6} from the outside in, then a periodic Gaussian blur of
    ``smooth_sigma`` voxels. float64.
    """
    nz, ny, nx = shape
    x, y, z = _grid(shape)
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    ax, ay, az = (ELLIPSOID_SEMI_AXES[0] * nx, ELLIPSOID_SEMI_AXES[1] * ny,
                  ELLIPSOID_SEMI_AXES[2] * nz)
    r = np.sqrt(((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2)
    img = np.zeros(shape)
    for frac, level in zip(ELLIPSOID_SHELLS, ELLIPSOID_LEVELS):
        img[r <= frac] = level
    if smooth_sigma > 0:
        img = ndimage.gaussian_filter(img, smooth_sigma, mode="wrap")
    return img


def add_noise(img, seed, var=0.01):
    """Adds N(0, var) noise (variance ``var``, so std 0.1 by default); no clipping."""
    return img + rng(seed).normal(0.0, np.sqrt(var), size=img.shape)


def random_velocity_coeffs(K, K_gen, seed, decay_power=2.0):
    """Unscaled random band-limited velocity coefficients, complex128 ``[3][K][K][K]``.

    Modes with |k_i| <= K_gen/2 - 1 get complex normal coefficients times
    (1 + |k|^2)^-decay_power; the rest are zero. The cube is made Hermitian
    (c_{-k} = conj c_k) so that it describes a real field, and the k = -K/2 planes are
    zero. The caller scales it to the wanted maximum displacement.
    """
    g = rng(seed)
    k = np.arange(K) - K // 2
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    h = K_gen // 2 - 1
    win = (np.abs(kx) <= h) & (np.abs(ky) <= h) & (np.abs(kz) <= h)
    amp = (1.0 + kx ** 2 + ky ** 2 + kz ** 2) ** (-decay_power)
    c = (g.standard_normal((3, K, K, K)) + 1j * g.standard_normal((3, K, K, K))) / np.sqrt(2.0)
    c = c * amp * win
    c[:, 0, :, :] = 0
    c[:, :, 0, :] = 0
    c[:, :, :, 0] = 0
    # Hermitian completion: index j maps to -k at index (K - j) for j >= 1.
    flip = c[:, ::-1, ::-1, ::-1]
    mirrored = np.zeros_like(c)
    mirrored[:, 1:, 1:, 1:] = np.conj(flip[:, :-1, :-1, :-1])
    return 0.5 * (c + mirrored)


def random_coeffs(K, seed, ncomp=3, decay_power=1.0):
    """Hermitian random coefficient cube ``[ncomp][K][K][K]``, ncomp <= 3 (test directions)."""
    assert 1 <= ncomp <= 3
    return random_velocity_coeffs(K, K, seed, decay_power=decay_power)[:ncomp].copy()


def random_field(shape, seed, ncomp=1, smooth=0.0):
    """Random real field(s) ``[ncomp][nz][ny][nx]`` (uniform [0,1)), optionally blurred."""
    f = rng(seed).random((ncomp,) + tuple(shape))
    if smooth > 0:
        f = np.stack([ndimage.gaussian_filter(fc, smooth, mode="wrap") for fc in f])
    return f


def random_displacement(shape, seed, max_vox=2.5, smooth=3.0):
    """Smooth random voxel-unit displacement ``[3][nz][ny][nx]`` with max |component| = max_vox."""
    d = random_field(shape, seed, 3, smooth) - 0.5
    d *= max_vox / max(np.abs(d).max(), 1e-30)
    return d
