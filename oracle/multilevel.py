"""Two-level preconditioner for the Gauss-Newton system, and flexible PCG. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 2.2 (Eqs. 13-14) solves H dv~ = -g~ by PCG with the spectral preconditioner
L~^{-1}; the discussion (Sec. 6) and the conclusions (Sec. 7) name the multi-level
preconditioner of the CLAIRE solver as the route to a faster PCG, without writing it out.
Reading used here:

  * coarse level: the same problem (variant, interpolation, nt, alpha, s, sigma^2) on the
    half grid N_a / 2 with band K_c = 2 floor(K / 4); its images are the spectral restriction
    of the fine ones (``restrict_image``) and its Gauss-Newton Hessian H_c is taken at the
    restricted velocity R v~;
  * R keeps the coefficients of the coarse band S_c = {|k|_inf <= K_c/2 - 1}; E = R^T pads
    with zeros. Under the normalisation of pi and iota a coefficient c_k describes the same
    function on every grid, so neither carries a scale factor;
  * P^{-1} r = E y + theta L~^{-1}(r - E R r), y from at most m_c PCG iterations on
    H_c y = R r (preconditioner L~_c^{-1}, zero start, relative tolerance 0.1): the coarse
    Hessian acts on the low modes, the spectral preconditioner on the rest;
  * theta = <R r, y> / <R r, L~_c^{-1} R r> (1 when R r = 0) puts the two parts on one scale.
    The cited two-level scheme applies L~^{-1} unscaled, which presumes that the regulariser
    dominates H at the modes above the coarse band; with the paper's alpha = 0.0025 the symbol
    w_k stays below 8 inside a band of 32 while the data term is tens to hundreds of times
    larger, and the unscaled split then preconditions worse than L~^{-1} alone. With theta,
    H = c L~ (any c > 0) is inverted exactly;
  * the inner PCG makes P^{-1} a nonlinear function of r, so the outer Krylov method is
    flexible PCG, beta_k = <z_{k+1}, r_{k+1} - r_k> / <z_k, r_k>; with a fixed linear
    preconditioner the subtracted term vanishes and it is PCG.
"""
from __future__ import annotations

import numpy as np

from . import spectral as S
from .gnk import pcg

INNER_TOL = 0.1


def coarse_band(K: int) -> int:
    """Band of the coarse level: K_c = 2 floor(K / 4) (even, and S_c inside S)."""
    return 2 * (K // 4)


def restrict_cube(c: np.ndarray, Kc: int) -> np.ndarray:
    """R: the coefficients of the band S_c. c is [..., K, K, K] (slot j holds k = j - K/2)."""
    K = c.shape[-1]
    assert Kc % 2 == 0 and 2 <= Kc <= K
    out = np.zeros(c.shape[:-3] + (Kc, Kc, Kc), dtype=c.dtype)
    ks = np.arange(-(Kc // 2) + 1, Kc // 2)          # the retained wavenumbers of S_c
    jf = ks + K // 2
    jc = ks + Kc // 2
    out[..., jc[:, None, None], jc[None, :, None], jc[None, None, :]] = \
        c[..., jf[:, None, None], jf[None, :, None], jf[None, None, :]]
    return out


def prolong_cube(cc: np.ndarray, K: int) -> np.ndarray:
    """E = R^T: a coarse cube [..., K_c, K_c, K_c] placed in a zero cube of edge K."""
    Kc = cc.shape[-1]
    out = np.zeros(cc.shape[:-3] + (K, K, K), dtype=cc.dtype)
    ks = np.arange(-(Kc // 2) + 1, Kc // 2)
    jf = ks + K // 2
    jc = ks + Kc // 2
    out[..., jf[:, None, None], jf[None, :, None], jf[None, None, :]] = \
        cc[..., jc[:, None, None], jc[None, :, None], jc[None, None, :]]
    return out


def restrict_image(f: np.ndarray) -> np.ndarray:
    """Spectral restriction of a periodic image [nz][ny][nx] (all even) to the half grid.

    The mean-normalised Fourier coefficients with |k_a| < n_a/2 on every axis (n = the half
    grid) are kept and synthesised on the half grid, so that a trigonometric polynomial of
    that band is simply sampled at the even voxels.
    """
    f = np.asarray(f, dtype=np.float64)
    assert all(n % 2 == 0 for n in f.shape)
    coarse = tuple(n // 2 for n in f.shape)
    F = np.fft.fftn(f) / f.size
    out = np.zeros(coarse, dtype=np.complex128)
    sel = []
    for nf, nc in zip(f.shape, coarse):
        k = np.fft.fftfreq(nc, 1.0 / nc).astype(int)       # wavenumbers of the half grid
        keep = np.abs(k) < nc / 2.0
        sel.append((np.nonzero(keep)[0], np.mod(k[keep], nf)))
    (iz, fz), (iy, fy), (ix, fx) = sel
    out[np.ix_(iz, iy, ix)] = F[np.ix_(fz, fy, fx)]
    return np.real(np.fft.ifftn(out) * out.size)


def fpcg(hv, b, prec, eta, maxit, inner=S.inner):
    """Flexible PCG for H x = b from x = 0 (Polak-Ribiere form of beta).

    Same stopping rules as ``gnk.pcg``; returns (x, iterations, negative_curvature).
    """
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = inner(r, z)
    bnorm = np.sqrt(inner(b, b))
    its = 0
    for i in range(maxit):
        Hp = hv(p)
        pHp = inner(p, Hp)
        its = i + 1
        if pHp <= 0.0:
            if i == 0:
                return z, its, True
            return x, its, True
        a = rz / pHp
        x = x + a * p
        r_old = r
        r = r - a * Hp
        if np.sqrt(inner(r, r)) <= eta * bnorm:
            break
        z = prec(r)
        rz_new = inner(r, z)
        beta = (rz_new - inner(r_old, z)) / rz
        p = z + beta * p
        rz = rz_new
    return x, its, False


class TwoLevel:
    """P^{-1} of a band-limited stationary problem: a coarse Gauss-Newton solve on the low
    modes, L~^{-1} on the rest. ``coarse`` is the half-grid problem (``coarse_problem``)."""

    def __init__(self, problem, coarse, inner_maxit, inner_tol=INNER_TOL):
        self.problem = problem
        self.coarse = coarse
        self.K = problem.p.K
        self.Kc = coarse.p.K
        self.maxit = inner_maxit
        self.tol = inner_tol
        self.vc = None
        self.inner_its = 0

    def set_velocity(self, vt):
        """The coarse Hessian is taken at R v~ (once per Gauss-Newton iterate)."""
        self.vc = restrict_cube(vt, self.Kc)

    def coarse_solve(self, rc):
        pc = self.coarse.p
        y, its, _ = pcg(lambda c: self.coarse.hessian_matvec(self.vc, c), rc,
                        lambda c: S.apply_Linv(c, pc.alpha, pc.s), self.tol, self.maxit)
        self.inner_its += its
        return y

    def __call__(self, r):
        p = self.problem.p
        rc = restrict_cube(r, self.Kc)
        y = self.coarse_solve(rc)
        q = S.inner(rc, S.apply_Linv(rc, p.alpha, p.s))
        theta = S.inner(rc, y) / q if q > 0 else 1.0
        high = r - prolong_cube(rc, self.K)
        return prolong_cube(y, self.K) + theta * S.apply_Linv(high, p.alpha, p.s)


def coarse_problem(problem):
    """The half-grid problem of a band-limited stationary ``variants.Problem``."""
    from .variants import Params, Problem

    p = problem.p
    cp = Params(K=coarse_band(p.K), nt=p.nt, alpha=p.alpha, s=p.s, sigma2=p.sigma2,
                order=p.order, variant=p.variant)
    return Problem(restrict_image(problem.I0), restrict_image(problem.I1), cp)
