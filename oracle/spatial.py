"""Spatial-domain PDE-LDDMM with SL-RK integration (the paper's "PDE-LDDMM ... SL" methods). FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1 poses the spatial problem: E(v) = 1/2 <L v, v>_{L2} + (1/sigma^2) ||m(1) - I1||^2,
L = (Id - alpha Laplacian)^s, the velocity v a field on the image grid, with the state
constraint imposed in one of three manners (IMAGE: transported m; STATE: m = I0 o phi;
DEFSTATE: the deformation state equation), Gauss-Newton-Krylov with preconditioner L^{-1}
(Eqs. 13-14); Sec. 3 solves every equation with SL-RK in Omega and states that the spatial
derivation is the band-limited one carried over.

Readings fixed here:
  * The spatial forms are the band-limited ones of Sec. 2.3 / Table 1 with pi and iota the
    identity: the truncated convolution becomes the pointwise product, D~ and grad~ the
    spectral derivatives on the full grid (i k_a over the grid wavenumbers
    k_a = -N_a/2 .. N_a/2 - 1, the Nyquist mode of a first derivative set to zero), L~ the
    symbol (1 + alpha |k|^2)^s over every grid wavenumber.
  * The L2 product is the voxel mean <a, b> = mean_x sum_c a_c b_c, so E_reg = 1/2 <L v, v>
    and the gradient below is the Riesz representative of dE under this product.
  * Every other reading (Heun step, trapezoid integrals, G = grad(I0 interpolant) o phi(1),
    dm(1) = -G . du(1), the Gauss-Newton terms of each variant, the nu and U equations of the
    state variant) is the band-limited one (``oracle/variants.py``).
  * SpatialProblem: stationary velocity; SpatialProblemNS: one field per time node.
"""
from __future__ import annotations

import numpy as np

from . import interp as I
from . import sl as SL
from .variants import DEFSTATE, IMAGE, STATE, Params, trapezoid_weights


# ------------------------------------------------------------------ grid spectral operators
def wavenumbers(shape):
    """Integer wavenumber grids (kx, ky, kz), each [nz][ny][nx], in numpy FFT order."""
    nz, ny, nx = shape
    kz, ky, kx = np.meshgrid(np.fft.fftfreq(nz, 1.0 / nz), np.fft.fftfreq(ny, 1.0 / ny),
                             np.fft.fftfreq(nx, 1.0 / nx), indexing="ij")
    return kx, ky, kz


def deriv(f, axis):
    """d f / d x_axis (axis 0 = x, 1 = y, 2 = z) of a real field on [0, 2 pi)^3, spectral;
    the Nyquist wavenumber of that axis (k = -N/2 for even N) contributes zero."""
    k = wavenumbers(f.shape)[axis].copy()
    n = f.shape[2 - axis]
    if n % 2 == 0:
        k[k == -n // 2] = 0.0
    return np.real(np.fft.ifftn(1j * k * np.fft.fftn(f)))


def grad(f):
    return np.stack([deriv(f, a) for a in range(3)])


def div(V):
    return deriv(V[0], 0) + deriv(V[1], 1) + deriv(V[2], 2)


def jacobian(U):
    """[a][b] = d U_a / d x_b."""
    return np.stack([np.stack([deriv(U[a], b) for b in range(3)]) for a in range(3)])


def l_symbol(shape, alpha, s):
    kx, ky, kz = wavenumbers(shape)
    return (1.0 + alpha * (kx * kx + ky * ky + kz * kz)) ** s


def apply_L(V, alpha, s, inverse=False):
    """L V = (Id - alpha Laplacian)^s V per component (L^{-1} with inverse=True)."""
    w = l_symbol(V.shape[1:], alpha, s)
    if inverse:
        w = 1.0 / w
    return np.stack([np.real(np.fft.ifftn(w * np.fft.fftn(c))) for c in V])


def inner(a, b):
    """<a, b> = mean over voxels of sum_c a_c b_c."""
    return float(np.sum(a * b) / a[0].size)


# ------------------------------------------------------------------ the problem
class SpatialProblem:
    """One spatial-domain registration problem: source I0, target I1, parameters (p.K unused)."""

    def __init__(self, I0, I1, params: Params):
        self.I0 = np.asarray(I0, dtype=np.float64)
        self.I1 = np.asarray(I1, dtype=np.float64)
        assert self.I0.shape == self.I1.shape and self.I0.ndim == 3
        self.p = params
        self.shape = self.I0.shape
        nz, ny, nx = self.shape
        self.tv = (np.array([nx, ny, nz], dtype=np.float64) / (2.0 * np.pi))[:, None, None, None]
        self.dt = 1.0 / params.nt
        self.tw = trapezoid_weights(params.nt)

    # hooks read by gnk.register
    def zeros(self):
        return np.zeros((3,) + self.shape)

    def inner(self, a, b):
        return inner(a, b)

    def precond(self, r):
        return apply_L(r, self.p.alpha, self.p.s, inverse=True)

    def energy_reg(self, v):
        return 0.5 * inner(apply_L(v, self.p.alpha, self.p.s), v)

    def energy_data(self, m1):
        r = m1 - self.I1
        return float(np.mean(r * r)) / self.p.sigma2

    def mse_rel(self, m1):
        return float(np.sum((m1 - self.I1) ** 2) / np.sum((self.I0 - self.I1) ** 2))

    def _offsets(self, v):
        V = v * self.tv
        return (SL.departure_offsets(V, self.dt, +1, self.p.order),
                SL.departure_offsets(V, self.dt, -1, self.p.order))

    def _warp_I0(self, u1):
        """m(1) = I0 o (id - u(1)) and G = (grad I0) o (id - u(1)) (physical)."""
        offs = -u1 * self.tv
        return (I.interpolate(self.I0, offs, self.p.order),
                I.interpolate_grad(self.I0, offs, self.p.order) * self.tv)

    # ---------------------------------------------------------------- state equations
    def state_defstate(self, v):
        """u from D_t u = v, u(0) = 0 (Sec. 2.1 deformation state as displacement; Table 1
        row 3 without projection), every node."""
        D, _ = self._offsets(v)
        us = [np.zeros_like(v)]
        for _ in range(self.p.nt):
            us.append(SL.heun_source_step(us[-1], D, v, v, self.dt, self.p.order))
        return us

    def state_image(self, v):
        """m from D_t m = 0, m(0) = I0 (Eq. 3 in SL form), every node."""
        D, _ = self._offsets(v)
        ms = [self.I0.copy()]
        for _ in range(self.p.nt):
            ms.append(SL.transport_step(ms[-1], D, self.p.order))
        return ms

    def inverse_maps(self, v):
        """nu and U backward from nu(1) = 0, U(1) = 0: -D_t nu = -v, -D_t U = -div v + U div v
        (the state variant's backward maps, psi = id - nu, J = 1 - U)."""
        _, Dp = self._offsets(v)
        d = div(v)
        nus, Us = [None] * (self.p.nt + 1), [None] * (self.p.nt + 1)
        nus[-1], Us[-1] = np.zeros_like(v), np.zeros(self.shape)
        for j in range(self.p.nt - 1, -1, -1):
            nus[j] = SL.heun_source_step(nus[j + 1], Dp, -v, -v, self.dt, self.p.order)
            Us[j] = SL.heun_jacobian_step(Us[j + 1], Dp, d, self.dt, self.p.order)
        return nus, Us

    def _pull_back(self, f, nus, Us):
        """J_j (f o psi_j) at every node."""
        return [(1.0 - U) * I.interpolate(f, -nu * self.tv, self.p.order) for nu, U in zip(nus, Us)]

    def _backward(self, f_end, v):
        """-D_t f = f div v backward from f(1) (Table 1 rows 2, 4, 6, 8 without projection)."""
        _, Dp = self._offsets(v)
        d = div(v)
        fs = [None] * (self.p.nt + 1)
        fs[-1] = f_end
        for j in range(self.p.nt - 1, -1, -1):
            fs[j] = SL.heun_divergence_step(fs[j + 1], Dp, d, self.dt, self.p.order)
        return fs

    # ---------------------------------------------------------------- assembly
    def _assemble_image(self, base, lams, gms):
        """L base + sum_j w_j lambda_j grad m_j (Eqs. 15-16 with the identity for pi, iota)."""
        out = apply_L(base, self.p.alpha, self.p.s)
        for w, lam, gm in zip(self.tw, lams, gms):
            out = out + w * lam[None] * gm
        return out

    def _assemble_defstate(self, base, rhos, us):
        """L base + sum_j w_j (rho_j - (D u_j)^T rho_j) (Eqs. 32-33 with the identity)."""
        out = apply_L(base, self.p.alpha, self.p.s)
        for w, rho, u in zip(self.tw, rhos, us):
            out = out + w * (rho - np.einsum("abzyx,azyx->bzyx", jacobian(u), rho))
        return out

    # ---------------------------------------------------------------- public API
    def objective(self, v):
        if self.p.variant == IMAGE:
            m1 = self.state_image(v)[-1]
        else:
            m1, _ = self._warp_I0(self.state_defstate(v)[-1])
        er, ed = self.energy_reg(v), self.energy_data(m1)
        return er + ed, er, ed, m1

    def gradient(self, v):
        p = self.p
        if p.variant == IMAGE:
            ms = self.state_image(v)
            m1 = ms[-1]
            lams = self._backward(-(2.0 / p.sigma2) * (m1 - self.I1), v)
            g = self._assemble_image(v, lams, [grad(m) for m in ms])
        elif p.variant == STATE:
            us = self.state_defstate(v)
            m1, _ = self._warp_I0(us[-1])
            ms = [I.interpolate(self.I0, -u * self.tv, p.order) for u in us]
            nus, Us = self.inverse_maps(v)
            lams = self._pull_back(-(2.0 / p.sigma2) * (m1 - self.I1), nus, Us)
            g = self._assemble_image(v, lams, [grad(m) for m in ms])
        else:
            us = self.state_defstate(v)
            m1, G = self._warp_I0(us[-1])
            rhos = self._backward(-(2.0 / p.sigma2) * (m1 - self.I1)[None] * G, v)
            g = self._assemble_defstate(v, rhos, us)
        er, ed = self.energy_reg(v), self.energy_data(m1)
        return er + ed, er, ed, g

    def _inc_defstate(self, v, dv, us):
        """du(1) from D_t du = dv - (D u) dv, du(0) = 0 (Eq. 36 without projection)."""
        D, _ = self._offsets(v)
        F = [dv - np.einsum("abzyx,bzyx->azyx", jacobian(u), dv) for u in us]
        du = np.zeros_like(v)
        for j in range(self.p.nt):
            du = SL.heun_source_step(du, D, F[j], F[j + 1], self.dt, self.p.order)
        return du

    def hessian_matvec(self, v, dv):
        p = self.p
        if p.variant == IMAGE:
            ms = self.state_image(v)
            gms = [grad(m) for m in ms]
            D, _ = self._offsets(v)
            F = [-np.sum(gm * dv, axis=0) for gm in gms]          # Eq. 19 without projection
            dm = np.zeros(self.shape)
            for j in range(p.nt):
                dm = SL.heun_source_step(dm, D, F[j], F[j + 1], self.dt, p.order)
            dlams = self._backward(-(2.0 / p.sigma2) * dm, v)    # Eq. 20
            return self._assemble_image(dv, dlams, gms)
        us = self.state_defstate(v)
        _, G = self._warp_I0(us[-1])
        dm1 = -np.sum(G * self._inc_defstate(v, dv, us), axis=0)
        if p.variant == STATE:
            ms = [I.interpolate(self.I0, -u * self.tv, p.order) for u in us]
            nus, Us = self.inverse_maps(v)
            dlams = self._pull_back(-(2.0 / p.sigma2) * dm1, nus, Us)
            return self._assemble_image(dv, dlams, [grad(m) for m in ms])
        drhos = self._backward(-(2.0 / p.sigma2) * dm1[None] * G, v)
        return self._assemble_defstate(dv, drhos, us)


class SpatialProblemNS(SpatialProblem):
    """Non-stationary spatial forms (the paper's "NSt. PDE-LDDMM ... SL" rows): the unknown is
    [v_0 .. v_nt], one field per node t_j = j / nt ([nt+1][3][nz][ny][nx]); every step uses the
    two-field characteristics of its end nodes (SL.departure_offsets_ns), the divergence of
    the node it reads, the gradient and Hessian at node j are the integrands at t_j, and the
    product is the trapezoid-weighted sum of the voxel-mean products of the nodes. With all
    nodes equal it reduces to SpatialProblem (the weighted sum of the g_j is its gradient)."""

    def zeros(self):
        return np.zeros((self.p.nt + 1, 3) + self.shape)

    def inner(self, a, b):
        return float(sum(w * inner(x, y) for w, x, y in zip(self.tw, a, b)))

    def precond(self, r):
        return np.stack([apply_L(x, self.p.alpha, self.p.s, inverse=True) for x in r])

    def energy_reg(self, vs):
        return float(sum(w * 0.5 * inner(apply_L(v, self.p.alpha, self.p.s), v)
                         for w, v in zip(self.tw, vs)))

    def _offsets_ns(self, vs):
        p = self.p
        Vs = [v * self.tv for v in vs]
        Df = [SL.departure_offsets_ns(Vs[j + 1], Vs[j], self.dt, +1, p.order) for j in range(p.nt)]
        Db = [SL.departure_offsets_ns(Vs[j], Vs[j + 1], self.dt, -1, p.order) for j in range(p.nt)]
        return Df, Db

    def state_defstate(self, vs):
        Df, _ = self._offsets_ns(vs)
        us = [np.zeros_like(vs[0])]
        for j in range(self.p.nt):
            us.append(SL.heun_source_step(us[-1], Df[j], vs[j], vs[j + 1], self.dt, self.p.order))
        return us

    def state_image(self, vs):
        Df, _ = self._offsets_ns(vs)
        ms = [self.I0.copy()]
        for j in range(self.p.nt):
            ms.append(SL.transport_step(ms[-1], Df[j], self.p.order))
        return ms

    def inverse_maps(self, vs):
        _, Db = self._offsets_ns(vs)
        ds = [div(v) for v in vs]
        nus, Us = [None] * (self.p.nt + 1), [None] * (self.p.nt + 1)
        nus[-1], Us[-1] = np.zeros_like(vs[0]), np.zeros(self.shape)
        for j in range(self.p.nt - 1, -1, -1):
            nus[j] = SL.heun_source_step(nus[j + 1], Db[j], -vs[j + 1], -vs[j], self.dt, self.p.order)
            Us[j] = SL.heun_jacobian_step_ns(Us[j + 1], Db[j], ds[j + 1], ds[j], self.dt, self.p.order)
        return nus, Us

    def _backward_ns(self, f_end, vs):
        _, Db = self._offsets_ns(vs)
        ds = [div(v) for v in vs]
        fs = [None] * (self.p.nt + 1)
        fs[-1] = f_end
        for j in range(self.p.nt - 1, -1, -1):
            fs[j] = SL.heun_divergence_step_ns(fs[j + 1], Db[j], ds[j + 1], ds[j], self.dt, self.p.order)
        return fs

    def _node_image(self, base, lams, gms):
        return np.stack([apply_L(b, self.p.alpha, self.p.s) + lam[None] * gm
                         for b, lam, gm in zip(base, lams, gms)])

    def _node_defstate(self, base, rhos, us):
        return np.stack([apply_L(b, self.p.alpha, self.p.s) + rho
                         - np.einsum("abzyx,azyx->bzyx", jacobian(u), rho)
                         for b, rho, u in zip(base, rhos, us)])

    def gradient(self, vs):
        p = self.p
        if p.variant == IMAGE:
            ms = self.state_image(vs)
            m1 = ms[-1]
            lams = self._backward_ns(-(2.0 / p.sigma2) * (m1 - self.I1), vs)
            g = self._node_image(vs, lams, [grad(m) for m in ms])
        elif p.variant == STATE:
            us = self.state_defstate(vs)
            m1, _ = self._warp_I0(us[-1])
            ms = [I.interpolate(self.I0, -u * self.tv, p.order) for u in us]
            nus, Us = self.inverse_maps(vs)
            lams = self._pull_back(-(2.0 / p.sigma2) * (m1 - self.I1), nus, Us)
            g = self._node_image(vs, lams, [grad(m) for m in ms])
        else:
            us = self.state_defstate(vs)
            m1, G = self._warp_I0(us[-1])
            rhos = self._backward_ns(-(2.0 / p.sigma2) * (m1 - self.I1)[None] * G, vs)
            g = self._node_defstate(vs, rhos, us)
        er, ed = self.energy_reg(vs), self.energy_data(m1)
        return er + ed, er, ed, g

    def hessian_matvec(self, vs, dvs):
        p = self.p
        Df, _ = self._offsets_ns(vs)
        if p.variant == IMAGE:
            ms = self.state_image(vs)
            gms = [grad(m) for m in ms]
            F = [-np.sum(gm * dv, axis=0) for gm, dv in zip(gms, dvs)]
            dm = np.zeros(self.shape)
            for j in range(p.nt):
                dm = SL.heun_source_step(dm, Df[j], F[j], F[j + 1], self.dt, p.order)
            return self._node_image(dvs, self._backward_ns(-(2.0 / p.sigma2) * dm, vs), gms)
        us = self.state_defstate(vs)
        _, G = self._warp_I0(us[-1])
        F = [dv - np.einsum("abzyx,bzyx->azyx", jacobian(u), dv) for u, dv in zip(us, dvs)]
        du = np.zeros_like(vs[0])
        for j in range(p.nt):
            du = SL.heun_source_step(du, Df[j], F[j], F[j + 1], self.dt, p.order)
        dm1 = -np.sum(G * du, axis=0)
        if p.variant == STATE:
            ms = [I.interpolate(self.I0, -u * self.tv, p.order) for u in us]
            nus, Us = self.inverse_maps(vs)
            dlams = self._pull_back(-(2.0 / p.sigma2) * dm1, nus, Us)
            return self._node_image(dvs, dlams, [grad(m) for m in ms])
        drhos = self._backward_ns(-(2.0 / p.sigma2) * dm1[None] * G, vs)
        return self._node_defstate(dvs, drhos, us)
