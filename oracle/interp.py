"""Periodic trilinear and cubic B-spline interpolation at departure points. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 3.1 (the transported field and the velocity are needed off the Eulerian grid,
so an interpolator is needed; cubic is the usual choice for SL schemes) and Sec. 4.2 (the
cubic interpolator with prefiltering of Ruijters et al.: a uniform cubic B-spline whose
coefficients are obtained by a prefilter, so that the spline interpolates the samples).

Readings: the domain is periodic (the Fourier basis of Sec. 2.2 is periodic), so indices
wrap. A query point is given as the grid point j plus an offset D (voxel units); the cell
is j + floor(D) and the fraction D - floor(D), so the fraction keeps the offset's precision.

Fields are [nz][ny][nx] (one component) or [C][nz][ny][nx]; offsets are [3][nz][ny][nx]
with component 0 = x, 1 = y, 2 = z.
"""
from __future__ import annotations

import numpy as np


def _cells(D, shape):
    """Base cell indices (wrapped) and fractions per axis for offsets D from the grid."""
    nz, ny, nx = shape
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for a, (j, n) in enumerate(((jx, nx), (jy, ny), (jz, nz))):
        fl = np.floor(D[a])
        out.append(((j + fl.astype(np.int64)) % n, D[a] - fl))
    return out  # [(ix, tx), (iy, ty), (iz, tz)]


def _lin_w(t):
    return [1.0 - t, t]


def _lin_dw(t):
    return [-np.ones_like(t), np.ones_like(t)]


def trilinear(f, D):
    """Value of the trilinear interpolant of periodic f at x + D (Sec. 3.1)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 4:
        return np.stack([trilinear(fc, D) for fc in f])
    nz, ny, nx = f.shape
    (ix, tx), (iy, ty), (iz, tz) = _cells(D, f.shape)
    wx, wy, wz = _lin_w(tx), _lin_w(ty), _lin_w(tz)
    out = np.zeros(f.shape)
    for c in range(2):
        zz = (iz + c) % nz
        for b in range(2):
            yy = (iy + b) % ny
            for a in range(2):
                xx = (ix + a) % nx
                out += wz[c] * wy[b] * wx[a] * f[zz, yy, xx]
    return out


def trilinear_grad(f, D):
    """Gradient (d/dx, d/dy, d/dz in voxel units) of the trilinear interpolant at x + D."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    (ix, tx), (iy, ty), (iz, tz) = _cells(D, f.shape)
    w = (_lin_w(tx), _lin_w(ty), _lin_w(tz))
    dw = (_lin_dw(tx), _lin_dw(ty), _lin_dw(tz))
    g = np.zeros((3,) + f.shape)
    for c in range(2):
        zz = (iz + c) % nz
        for b in range(2):
            yy = (iy + b) % ny
            for a in range(2):
                xx = (ix + a) % nx
                v = f[zz, yy, xx]
                g[0] += dw[0][a] * w[1][b] * w[2][c] * v
                g[1] += w[0][a] * dw[1][b] * w[2][c] * v
                g[2] += w[0][a] * w[1][b] * dw[2][c] * v
    return g


def bspline_prefilter(f):
    """Periodic cubic B-spline coefficients c with sum_i c_i beta3(j - i) = f_j exactly.

    Per axis this is the cyclic system (c_{j-1} + 4 c_j + c_{j+1}) / 6 = f_j. A circulant
    system is diagonal in the DFT basis, so it is solved exactly by dividing the line's DFT
    by the circulant's eigenvalues (4 + 2 cos(2 pi k / N)) / 6.
    """
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 4:
        return np.stack([bspline_prefilter(fc) for fc in f])
    c = f
    for axis in range(3):
        n = f.shape[axis]
        lam = (4.0 + 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)) / 6.0
        shp = [1, 1, 1]
        shp[axis] = n
        c = np.fft.ifft(np.fft.fft(c, axis=axis) / lam.reshape(shp), axis=axis).real
    return c


def _cub_w(t):
    """Uniform cubic B-spline weights for taps -1, 0, 1, 2 at fraction t in [0, 1)."""
    s = 1.0 - t
    return [s ** 3 / 6.0,
            (3.0 * t ** 3 - 6.0 * t ** 2 + 4.0) / 6.0,
            (-3.0 * t ** 3 + 3.0 * t ** 2 + 3.0 * t + 1.0) / 6.0,
            t ** 3 / 6.0]


def _cub_dw(t):
    s = 1.0 - t
    return [-0.5 * s ** 2,
            (9.0 * t ** 2 - 12.0 * t) / 6.0,
            (-9.0 * t ** 2 + 6.0 * t + 3.0) / 6.0,
            0.5 * t ** 2]


def cubic_coeffs_eval(c, D):
    """Evaluate the periodic cubic B-spline with coefficients c at x + D (64 taps)."""
    c = np.asarray(c, dtype=np.float64)
    if c.ndim == 4:
        return np.stack([cubic_coeffs_eval(cc, D) for cc in c])
    nz, ny, nx = c.shape
    (ix, tx), (iy, ty), (iz, tz) = _cells(D, c.shape)
    wx, wy, wz = _cub_w(tx), _cub_w(ty), _cub_w(tz)
    out = np.zeros(c.shape)
    for r in range(4):
        zz = (iz + r - 1) % nz
        for q in range(4):
            yy = (iy + q - 1) % ny
            wzy = wz[r] * wy[q]
            for p in range(4):
                xx = (ix + p - 1) % nx
                out += wzy * wx[p] * c[zz, yy, xx]
    return out


def cubic_coeffs_grad(c, D):
    """Gradient (voxel units) of the cubic B-spline with coefficients c at x + D."""
    c = np.asarray(c, dtype=np.float64)
    nz, ny, nx = c.shape
    (ix, tx), (iy, ty), (iz, tz) = _cells(D, c.shape)
    w = (_cub_w(tx), _cub_w(ty), _cub_w(tz))
    dw = (_cub_dw(tx), _cub_dw(ty), _cub_dw(tz))
    g = np.zeros((3,) + c.shape)
    for r in range(4):
        zz = (iz + r - 1) % nz
        for q in range(4):
            yy = (iy + q - 1) % ny
            for p in range(4):
                xx = (ix + p - 1) % nx
                v = c[zz, yy, xx]
                g[0] += dw[0][p] * w[1][q] * w[2][r] * v
                g[1] += w[0][p] * dw[1][q] * w[2][r] * v
                g[2] += w[0][p] * w[1][q] * dw[2][r] * v
    return g


def interpolate(f, D, order):
    """Interpolate samples f at x + D: order 1 = trilinear, 3 = prefiltered cubic B-spline."""
    if order == 1:
        return trilinear(f, D)
    if order == 3:
        return cubic_coeffs_eval(bspline_prefilter(f), D)
    raise ValueError("order must be 1 or 3")


def interpolate_grad(f, D, order):
    """Gradient (voxel units) of the order-1 or order-3 interpolant of samples f at x + D."""
    if order == 1:
        return trilinear_grad(f, D)
    if order == 3:
        return cubic_coeffs_grad(bspline_prefilter(f), D)
    raise ValueError("order must be 1 or 3")
