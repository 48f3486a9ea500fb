"""Band-limited spaces: projection pi, inclusion iota, spectral operators. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 2.2 ("Parameterization in the space of band-limited vector fields"): the
truncated Fourier domain with bounds K_1..K_d, the inclusion iota: V~ -> V, the projection
pi: V -> V~, the scalar product <L~ v~, w~>_{l2} (Eq. 9) with L~ the projection of
L = (Id - alpha Delta)^s (Sec. 2.1, Eq. 1), and tilde operators (D~, grad~, div~) as the
projection of the differential operators.

Readings where the paper is silent (stated once here, used everywhere):
  * domain Omega = [0, 2 pi)^3, periodic; voxel j_a sits at x_a = 2 pi j_a / N_a;
  * pi(f)_k = (1/N_tot) sum_x f(x) exp(-i k.x)  (mean-normalised DFT restricted to S);
  * iota(c)(x) = sum_{k in S} c_k exp(+i k.x)   (plain synthesis), real part of it;
  * S = {k : |k_a| <= K/2 - 1}; a cube of K^3 slots indexed j = k + K/2, slot j = 0 is
    always zero (so the cube is symmetric under k -> -k);
  * symbol of L~: w_k = (1 + alpha |k|^2)^s with integer k;
  * <a, b> = Re sum_k conj(a_k) b_k over the whole cube; then <iota c, f>_mean = <c, pi f>.
"""
from __future__ import annotations

import numpy as np


def mode_numbers(K: int) -> np.ndarray:
    """Wavenumber held by cube slot j: k = j - K/2 (slot 0, k = -K/2, never retained)."""
    assert K % 2 == 0 and K >= 2
    return np.arange(K) - K // 2


def retained_mask(K: int) -> np.ndarray:
    """Boolean [K][K][K] mask of the retained set S (all three slot indices >= 1)."""
    m = np.ones((K, K, K), dtype=bool)
    m[0, :, :] = False
    m[:, 0, :] = False
    m[:, :, 0] = False
    return m


def _index_maps(K, shape):
    nz, ny, nx = shape
    assert K // 2 - 1 < min(nx, ny, nz) / 2.0, "band must lie below the grid's Nyquist"
    k = mode_numbers(K)
    return np.mod(k, nz), np.mod(k, ny), np.mod(k, nx)


def project(f: np.ndarray, K: int) -> np.ndarray:
    """pi: real field(s) [..., nz, ny, nx] -> complex cube [..., K, K, K] (Sec. 2.2).

    pi(f)_k = (1/N_tot) sum_x f(x) e^{-i k.x}. The DFT over the grid is taken with
    numpy's FFT (a library DFT) and then restricted to S.
    """
    f = np.asarray(f, dtype=np.float64)
    shape = f.shape[-3:]
    iz, iy, ix = _index_maps(K, shape)
    F = np.fft.fftn(f, axes=(-3, -2, -1)) / float(np.prod(shape))
    c = F[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return c * retained_mask(K)


def include(c: np.ndarray, shape) -> np.ndarray:
    """iota: complex cube(s) [..., K, K, K] -> real field(s) [..., nz, ny, nx] (Sec. 2.2).

    iota(c)(x) = Re sum_{k in S} c_k e^{i k.x}; with a Hermitian cube the sum is real.
    """
    c = np.asarray(c, dtype=np.complex128)
    K = c.shape[-1]
    iz, iy, ix = _index_maps(K, shape)
    lead = c.shape[:-3]
    F = np.zeros(lead + tuple(shape), dtype=np.complex128)
    cm = c * retained_mask(K)
    F[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]] = cm
    f = np.fft.ifftn(F, axes=(-3, -2, -1)) * float(np.prod(shape))
    return f.real.copy()


def project_direct(f: np.ndarray, K: int) -> np.ndarray:
    """pi by the literal triple sum over all voxels (brute force, tiny grids only)."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    k = mode_numbers(K)
    out = np.zeros((K, K, K), dtype=np.complex128)
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    for jz in range(1, K):
        for jy in range(1, K):
            for jx in range(1, K):
                phase = k[jx] * x + k[jy] * y + k[jz] * z
                out[jz, jy, jx] = np.sum(f * np.exp(-1j * phase)) / f.size
    return out


def include_direct(c: np.ndarray, shape) -> np.ndarray:
    """iota by the literal sum over retained modes at every voxel (tiny grids only)."""
    nz, ny, nx = shape
    K = c.shape[-1]
    k = mode_numbers(K)
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    out = np.zeros(shape, dtype=np.complex128)
    for jz in range(1, K):
        for jy in range(1, K):
            for jx in range(1, K):
                out += c[jz, jy, jx] * np.exp(1j * (k[jx] * x + k[jy] * y + k[jz] * z))
    return out.real


def wavevectors(K: int):
    """(kx, ky, kz) integer wavenumber grids of shape [K][K][K] (slot order [jz][jy][jx])."""
    k = mode_numbers(K).astype(np.float64)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    return kx, ky, kz


def deriv(c: np.ndarray, axis: int) -> np.ndarray:
    """Spectral partial derivative d/dx_axis (axis 0 = x, 1 = y, 2 = z): c_k -> i k_axis c_k."""
    kv = wavevectors(c.shape[-1])[axis]
    return 1j * kv * c


def grad(c: np.ndarray) -> np.ndarray:
    """grad~ of a scalar cube [K,K,K] -> [3][K,K,K] (Sec. 2.2, tilde of nabla)."""
    return np.stack([deriv(c, a) for a in range(3)])


def div(c: np.ndarray) -> np.ndarray:
    """div~ of a vector cube [3][K,K,K] -> [K,K,K] (Sec. 2.2, tilde of nabla.)."""
    return deriv(c[0], 0) + deriv(c[1], 1) + deriv(c[2], 2)


def jacobian(c: np.ndarray) -> np.ndarray:
    """D~ of a vector cube: J[a][b] = i k_b c_a, i.e. the cube of d u_a / d x_b."""
    return np.stack([np.stack([deriv(c[a], b) for b in range(3)]) for a in range(3)])


def l_symbol(K: int, alpha: float, s: int) -> np.ndarray:
    """Symbol of L~ = projection of (Id - alpha Delta)^s: w_k = (1 + alpha |k|^2)^s (Eq. 1, 9)."""
    kx, ky, kz = wavevectors(K)
    return (1.0 + alpha * (kx * kx + ky * ky + kz * kz)) ** s * retained_mask(K)


def apply_L(c: np.ndarray, alpha: float, s: int) -> np.ndarray:
    return l_symbol(c.shape[-1], alpha, s) * c


def apply_Linv(c: np.ndarray, alpha: float, s: int) -> np.ndarray:
    """Preconditioner L~^{-1} (Sec. 2.2: GNK in V~ with preconditioner L~^{-1})."""
    w = l_symbol(c.shape[-1], alpha, s)
    return np.where(w > 0, c / np.where(w > 0, w, 1.0), 0.0)


def inner(a: np.ndarray, b: np.ndarray) -> float:
    """<a, b> = Re sum conj(a) b over the whole cube(s) (the l2 product of Eq. 9)."""
    return float(np.real(np.vdot(a.ravel(), b.ravel())))


def star(a: np.ndarray, b: np.ndarray, shape) -> np.ndarray:
    """Truncated convolution a * b := pi(iota(a) iota(b)) (Sec. 2.2, Lie bracket product)."""
    return project(include(a, shape) * include(b, shape), a.shape[-1])


def hermitian_part(c: np.ndarray) -> np.ndarray:
    """(c_k + conj c_{-k}) / 2 over the cube (slot j pairs with slot K - j)."""
    flip = np.zeros_like(c)
    flip[..., 1:, 1:, 1:] = np.conj(c[..., :0:-1, :0:-1, :0:-1])
    return 0.5 * (c + flip)


def bspline_symbol(K: int, shape) -> np.ndarray:
    """Fourier symbol of the periodic cubic B-spline sampling operator on the grid.

    Sampling sum_i c_i beta3(x - i) at the knots is the circulant (1, 4, 1)/6 along each
    axis, whose eigenvalue at wavenumber k is (2 + cos(2 pi k / N)) / 3.
    """
    nz, ny, nx = shape
    kx, ky, kz = wavevectors(K)
    return ((2 + np.cos(2 * np.pi * kx / nx)) / 3 * (2 + np.cos(2 * np.pi * ky / ny)) / 3
            * (2 + np.cos(2 * np.pi * kz / nz)) / 3)
