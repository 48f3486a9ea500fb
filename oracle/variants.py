"""Energy, gradient and Gauss-Newton Hessian-vector product of BL PDE-LDDMM. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The three variants of Sec. 2.3, each with a stationary band-limited velocity v~ (one cube
for all t) and SL-RK integration of every equation (Sec. 3.3, Table 1):

  * IMAGE  -- original BL PDE-LDDMM (Sec. 2.3.1, Eqs. 15-20): spatial state m and adjoint
    lambda, band-limited incremental state dm~ and incremental adjoint dlambda~;
    g = L~v~ + int lambda~ * grad~ m~ dt, H dv~ = L~dv~ + int dlambda~ * grad~ m~ dt.
  * STATE -- BL PDE-LDDMM based on the state equation (Sec. 2.3.2): m(t) = I0 o phi(t),
    lambda(t) = J(t) lambda(1) o psi(t), with phi = id - iota(u~) from the deformation state
    equation, psi = id - iota(nu~) and J = 1 - iota(U~) from two backward equations; the
    gradient and Hessian are those of IMAGE (Eqs. 15-16) with these m and lambda.
  * DEFSTATE -- BL PDE-LDDMM based on the deformation state equation (Sec. 2.3.3,
    Eqs. 31-37): displacement u~ with phi = id - iota(u~), m(1) = I0 o phi(1); adjoint rho~;
    g = L~v~ + int (rho~ - D~u~ * rho~) dt, H dv~ = L~dv~ + int (drho~ - D~u~ * drho~) dt.

Energy (Eq. 10): E = 1/2 <L~v~, v~> + (1/sigma^2) ||m(1) - I1||^2 with the L2 norm read as
the mean over voxels (the same normalisation as pi, so that <iota c, f> = <c, pi f>).

Readings fixed here (the paper is ambiguous, silent or has typos at these places):
  * D~u~ * rho~ in the DEFSTATE gradient is (D iota(u~))^T iota(rho~) projected, i.e.
    component b = sum_a d_b u_a rho_a (the adjoint of v -> (Du) v).
  * The DEFSTATE Hessian of Eq. 33 prints D~ du~ * rho~; the Gauss-Newton operator
    (J^T W J, which is symmetric) has D~u~ * drho~ there, and that is what is used.
  * Table 1 row 6 prints lambda~ on the right-hand side of the dlambda~ equation; Eq. 20
    has dlambda~, which is used.
  * rho~(1) = pi(-(2/sigma^2) r G), drho~(1) = pi(-(2/sigma^2) dm(1) G) with r = m(1) - I1,
    dm(1) = -G . iota(du~(1)) and G = (grad I0) o phi(1), the exact derivative of
    m(1) = I0 o (id - iota(u~(1))) with respect to u~(1) (the paper writes grad m(1)).
  * Time integrals: trapezoid rule over the nt + 1 nodes t_j = j / nt.
  * STATE: the nu~ equation of Sec. 2.3.2 prints -nu~_t as its right-hand side; psi(t) maps
    the point at time t to its position at time 1, psi = id - iota(nu~), which makes the
    right-hand side -v~ (psi(t) = id + int_t^1 v), and that is used.
  * STATE, Gauss-Newton Hessian: lambda(t) = J(t) lambda(1) o psi(t) varies with dv through
    lambda(1), psi and J; the Sec. 2.3.2 formula for dlambda keeps the psi term, which is
    proportional to grad lambda(1), i.e. to the residual. Gauss-Newton drops every term
    proportional to the residual (as IMAGE drops lambda grad dm), which leaves
    dlambda(t) = J(t) dlambda(1) o psi(t) with dlambda(1) = -(2/sigma^2) dm(1) and
    dm(1) = -G . iota(du~(1)) (the sign of the exact derivative of I0 o (id - iota(u~)));
    du~ solves the incremental deformation state equation (Eq. 36), and that is what is
    used. dnu~ is then not needed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import interp as I
from . import sl as SL
from . import spectral as S

IMAGE = 1
STATE = 2
DEFSTATE = 3


@dataclass
class Params:
    K: int = 16
    nt: int = 10
    alpha: float = 0.0025
    s: int = 2
    sigma2: float = 0.01
    order: int = 1          # 1 trilinear, 3 cubic B-spline
    variant: int = DEFSTATE


def trapezoid_weights(nt):
    w = np.full(nt + 1, 1.0 / nt)
    w[0] = w[-1] = 0.5 / nt
    return w


class Problem:
    """One registration problem: source I0 (moving), target I1 (fixed), parameters."""

    def __init__(self, I0, I1, params: Params):
        self.I0 = np.asarray(I0, dtype=np.float64)
        self.I1 = np.asarray(I1, dtype=np.float64)
        assert self.I0.shape == self.I1.shape and self.I0.ndim == 3
        self.p = params
        self.shape = self.I0.shape
        nz, ny, nx = self.shape
        # physical [0, 2 pi) -> voxel units, per component x, y, z
        self.to_vox = np.array([nx, ny, nz], dtype=np.float64) / (2.0 * np.pi)
        self.dt = 1.0 / params.nt
        self.tw = trapezoid_weights(params.nt)

    # ---------------------------------------------------------------- velocity (Sec. 3.2)
    def velocity(self, vt):
        """v = iota(v~) (physical), V = v in voxel units, d = iota(div~ v~) (Eq. 46, Table 1)."""
        v = S.include(vt, self.shape)
        V = v * self.to_vox[:, None, None, None]
        d = S.include(S.div(vt), self.shape)
        return v, V, d

    def energy_reg(self, vt):
        """1/2 <L~ v~, v~>_{l2} (Eq. 10, first term, stationary v~)."""
        return 0.5 * S.inner(S.apply_L(vt, self.p.alpha, self.p.s), vt)

    def energy_data(self, m1):
        """(1/sigma^2) ||m(1) - I1||^2 as a voxel mean (Eq. 10, second term)."""
        r = m1 - self.I1
        return float(np.mean(r * r)) / self.p.sigma2

    # ------------------------------------------------------------------ DEFSTATE (V3)
    def _warp_I0(self, u1):
        """m(1) = I0 o phi(1), phi = id - iota(u~(1)), and G = (grad I0) o phi(1) (physical)."""
        offs = -S.include(u1, self.shape) * self.to_vox[:, None, None, None]
        m1 = I.interpolate(self.I0, offs, self.p.order)
        G = I.interpolate_grad(self.I0, offs, self.p.order) * self.to_vox[:, None, None, None]
        return m1, G

    def state_defstate(self, vt):
        """u~ from D~_t u~ = v~, u~(0) = 0 (Eq. 34; Table 1 row 3), all nodes kept."""
        p = self.p
        v, V, d = self.velocity(vt)
        D = SL.departure_offsets(V, self.dt, +1, p.order)
        u = np.zeros((3, p.K, p.K, p.K), dtype=np.complex128)
        us = [u]
        for _ in range(p.nt):
            u = SL.bl_heun_source_step(u, D, v, v, self.dt, p.order, self.shape, p.K)
            us.append(u)
        return us

    def _jacobians(self, us):
        """Spatial D iota(u~_j): [j][a][b] = d u_a / d x_b (physical)."""
        return [S.include(S.jacobian(u), self.shape) for u in us]

    def _adjoint_bl(self, rho_end, vt):
        """Backward sweep of -D~_t rho~ = rho~ * div~ v~ (Eqs. 35/37; Table 1 rows 4/8)."""
        p = self.p
        v, V, d = self.velocity(vt)
        Dp = SL.departure_offsets(V, self.dt, -1, p.order)
        rhos = [None] * (p.nt + 1)
        rhos[p.nt] = rho_end
        rho = rho_end
        for j in range(p.nt - 1, -1, -1):
            rho = SL.bl_heun_divergence_step(rho, Dp, d, self.dt, p.order, self.shape, p.K)
            rhos[j] = rho
        return rhos

    def _assemble_defstate(self, base, rhos, Jus):
        """L~ base + sum_j w_j (rho~_j - pi((D iota u~_j)^T iota(rho~_j))) (Eqs. 32-33)."""
        out = S.apply_L(base, self.p.alpha, self.p.s).astype(np.complex128)
        for j, (rho, Ju) in enumerate(zip(rhos, Jus)):
            r_sp = S.include(rho, self.shape)
            JT = np.einsum("abzyx,azyx->bzyx", Ju, r_sp)
            out = out + self.tw[j] * (rho - S.project(JT, self.p.K))
        return out

    # ------------------------------------------------------------------ IMAGE (V1)
    def state_image(self, vt):
        """m from D_t m = 0, m(0) = I0 (Eq. 17; Table 1 row 1), all nodes kept (spatial)."""
        p = self.p
        v, V, d = self.velocity(vt)
        D = SL.departure_offsets(V, self.dt, +1, p.order)
        m = self.I0.copy()
        ms = [m]
        for _ in range(p.nt):
            m = SL.transport_step(m, D, p.order)
            ms.append(m)
        return ms

    def _grad_mtilde(self, ms):
        """iota(grad~ m~_j) with m~_j = pi(m_j) (Sec. 2.3.1), [j][3] spatial, physical."""
        return [S.include(S.grad(S.project(m, self.p.K)), self.shape) for m in ms]

    def _assemble_image(self, base, lams, gms, project_lam=True):
        """L~ base + sum_j w_j pi(iota(lambda~_j) iota(grad~ m~_j)) (Eqs. 15-16); lams are
        spatial fields (projected first, lambda~ = pi(lambda)) or, project_lam=False, cubes."""
        p = self.p
        out = S.apply_L(base, p.alpha, p.s).astype(np.complex128)
        for j in range(p.nt + 1):
            lt = S.project(lams[j], p.K) if project_lam else lams[j]
            out = out + self.tw[j] * S.project(S.include(lt, self.shape)[None] * gms[j], p.K)
        return out

    # ------------------------------------------------------------------ STATE (V2)
    def _compose_I0(self, us):
        """m_j = I0 o phi_j, phi_j = id - iota(u~_j) (Sec. 2.3.2), every node."""
        return [I.interpolate(self.I0, -S.include(u, self.shape) * self.to_vox[:, None, None, None],
                              self.p.order) for u in us]

    def inverse_maps(self, vt):
        """nu~_j and U~_j at every node (Sec. 2.3.2), backward from nu~(1) = 0, U~(1) = 0:
        -D~_t nu~ = -v~ and -D~_t U~ = -div~ v~ + U~ * div~ v~ in SL form (Sec. 3.3).
        psi_j = id - iota(nu~_j) (physical), J_j = 1 - iota(U~_j)."""
        p = self.p
        v, V, d = self.velocity(vt)
        Dp = SL.departure_offsets(V, self.dt, -1, p.order)
        nu = np.zeros((3, p.K, p.K, p.K), dtype=np.complex128)
        U = np.zeros((p.K, p.K, p.K), dtype=np.complex128)
        nus, Us = [None] * (p.nt + 1), [None] * (p.nt + 1)
        nus[p.nt], Us[p.nt] = nu, U
        for j in range(p.nt - 1, -1, -1):
            # backward in time: D_tau nu = -v along X+
            nu = SL.bl_heun_source_step(nu, Dp, -v, -v, self.dt, p.order, self.shape, p.K)
            U = SL.bl_heun_jacobian_step(U, Dp, d, self.dt, p.order, self.shape, p.K)
            nus[j], Us[j] = nu, U
        return nus, Us

    def _pull_back(self, f, nus, Us):
        """f_j = J_j (f o psi_j) at every node (lambda(t) = J(t) lambda(1) o psi(t))."""
        out = []
        for nu, U in zip(nus, Us):
            offs = -S.include(nu, self.shape) * self.to_vox[:, None, None, None]
            out.append((1.0 - S.include(U, self.shape)) * I.interpolate(f, offs, self.p.order))
        return out

    def _grads_state(self, vt):
        """u~_j, m_j, iota(grad~ m~_j) and the inverse maps of the STATE variant."""
        us = self.state_defstate(vt)
        ms = self._compose_I0(us)
        nus, Us = self.inverse_maps(vt)
        return us, ms, self._grad_mtilde(ms), nus, Us

    def _inc_defstate(self, vt, dvt, us):
        """du~(1) from D~_t du~ = dv~ - D~u~ * dv~, du~(0) = 0 (Eq. 36; Table 1 row 7)."""
        p = self.p
        v, V, d = self.velocity(vt)
        D = SL.departure_offsets(V, self.dt, +1, p.order)
        dv = S.include(dvt, self.shape)
        F = [dv - np.einsum("abzyx,bzyx->azyx", Ju, dv) for Ju in self._jacobians(us)]
        du = np.zeros_like(dvt, dtype=np.complex128)
        for j in range(p.nt):
            du = SL.bl_heun_source_step(du, D, F[j], F[j + 1], self.dt, p.order, self.shape, p.K)
        return du

    # ------------------------------------------------------------------ public API
    def objective(self, vt):
        """(E, E_reg, E_data, m(1)) at v~ (Eq. 10 with the variant's state equation)."""
        if self.p.variant in (DEFSTATE, STATE):
            us = self.state_defstate(vt)
            m1, _ = self._warp_I0(us[-1])
        else:
            m1 = self.state_image(vt)[-1]
        er, ed = self.energy_reg(vt), self.energy_data(m1)
        return er + ed, er, ed, m1

    def gradient(self, vt):
        """Returns (E, E_reg, E_data, g~) (Eq. 15 for IMAGE and STATE, Eq. 32 for DEFSTATE)."""
        p = self.p
        if p.variant == STATE:
            us, ms, gms, nus, Us = self._grads_state(vt)
            m1, _ = self._warp_I0(us[-1])
            lams = self._pull_back(-(2.0 / p.sigma2) * (m1 - self.I1), nus, Us)
            g = self._assemble_image(vt, lams, gms)
        elif p.variant == DEFSTATE:
            us = self.state_defstate(vt)
            m1, G = self._warp_I0(us[-1])
            r = m1 - self.I1
            rho1 = S.project(-(2.0 / p.sigma2) * r[None] * G, p.K)
            rhos = self._adjoint_bl(rho1, vt)
            g = self._assemble_defstate(vt, rhos, self._jacobians(us))
        else:
            ms = self.state_image(vt)
            m1 = ms[-1]
            v, V, d = self.velocity(vt)
            Dp = SL.departure_offsets(V, self.dt, -1, p.order)
            lam = -(2.0 / p.sigma2) * (m1 - self.I1)          # lambda(1)
            lams = [None] * (p.nt + 1)
            lams[p.nt] = lam
            for j in range(p.nt - 1, -1, -1):                   # Eq. 18, Table 1 row 2
                lam = SL.heun_divergence_step(lam, Dp, d, self.dt, p.order)
                lams[j] = lam
            g = self._assemble_image(vt, lams, self._grad_mtilde(ms))   # lambda~ * grad~ m~
        er, ed = self.energy_reg(vt), self.energy_data(m1)
        return er + ed, er, ed, g

    def hessian_matvec(self, vt, dvt):
        """Gauss-Newton H dv~ at v~ (Eq. 16 for IMAGE and, as read, STATE; Eq. 33 as read
        for DEFSTATE)."""
        p = self.p
        v, V, d = self.velocity(vt)
        D = SL.departure_offsets(V, self.dt, +1, p.order)
        dv = S.include(dvt, self.shape)
        if p.variant == STATE:
            us, ms, gms, nus, Us = self._grads_state(vt)
            _, G = self._warp_I0(us[-1])
            dm1 = -np.sum(G * S.include(self._inc_defstate(vt, dvt, us), self.shape), axis=0)
            dlams = self._pull_back(-(2.0 / p.sigma2) * dm1, nus, Us)
            return self._assemble_image(dvt, dlams, gms)
        if p.variant == DEFSTATE:
            us = self.state_defstate(vt)
            _, G = self._warp_I0(us[-1])
            dm1 = -np.sum(G * S.include(self._inc_defstate(vt, dvt, us), self.shape), axis=0)
            drho1 = S.project(-(2.0 / p.sigma2) * dm1[None] * G, p.K)
            drhos = self._adjoint_bl(drho1, vt)
            return self._assemble_defstate(dvt, drhos, self._jacobians(us))
        ms = self.state_image(vt)
        gms = self._grad_mtilde(ms)
        # incremental state D~_t dm~ = -grad~ m~ * dv~ (Eq. 19; Table 1 row 5)
        F = [-np.sum(gm * dv, axis=0) for gm in gms]
        dm = np.zeros((p.K, p.K, p.K), dtype=np.complex128)
        for j in range(p.nt):
            dm = SL.bl_heun_source_step(dm, D, F[j], F[j + 1], self.dt, p.order, self.shape, p.K)
        dlam = -(2.0 / p.sigma2) * dm                             # dlambda~(1)
        Dp = SL.departure_offsets(V, self.dt, -1, p.order)
        out = S.apply_L(dvt, p.alpha, p.s).astype(np.complex128)
        for j in range(p.nt, -1, -1):                             # Eq. 20; Table 1 row 6
            out = out + self.tw[j] * S.project(S.include(dlam, self.shape)[None] * gms[j], p.K)
            if j > 0:
                dlam = SL.bl_heun_divergence_step(dlam, Dp, d, self.dt, p.order, self.shape, p.K)
        return out

    # ------------------------------------------------------------------ diagnostics
    def mse_rel(self, m1):
        """MSE_rel = ||m(1) - I1||^2 / ||I0 - I1||^2 (Sec. 5.1.1)."""
        return float(np.sum((m1 - self.I1) ** 2) / np.sum((self.I0 - self.I1) ** 2))

    @staticmethod
    def jacobian_determinant_of(u1, shape):
        """det D phi per voxel for phi = id - iota(u~) (physical units): det(I - D iota(u~)).
        The paper reports its minimum and maximum over the volume (Sec. 5.1.1, Table 3)."""
        Du = S.include(S.jacobian(u1), shape)   # [a][b][z][y][x] = d u_a / d x_b
        A = np.eye(3)[:, :, None, None, None] - Du
        return np.linalg.det(np.moveaxis(A, (0, 1), (-2, -1)))

    def jacobian_determinant(self, vt):
        """det D phi(1) of the deformation-state solution for vt (DEFSTATE)."""
        return self.jacobian_determinant_of(self.state_defstate(vt)[-1], self.shape)

    def max_displacement_vox(self, vt):
        """Max over voxels of |phi(1)(x) - x| in voxels (DEFSTATE: |iota(u~(1))|)."""
        us = self.state_defstate(vt)
        u = S.include(us[-1], self.shape) * self.to_vox[:, None, None, None]
        return float(np.sqrt((u * u).sum(0)).max())


class ProblemNS(Problem):
    """Non-stationary forms of the three variants (Sec. 2.3 with a time-dependent v~_t; the
    paper's NSt rows): the unknown is v~ = [v~_0 .. v~_nt], one cube per node t_j = j/nt
    ([nt+1][3][K][K][K]). Equations as in Problem with v~ replaced by v~(t_j) at node j.
    Deformation state:
      state   u~_{j+1} = pi[iota(u~_j) o X_j + dt/2 (v_j(X_j) + v_{j+1}(x))],
              X_j from departure_offsets_ns(V_{j+1}, V_j) (R10);
      adjoint rho~_j = pi[Heun step of -D_t rho = rho div v_t along X+_j],
              X+_j from departure_offsets_ns(V_j, V_{j+1}), d(X+) from d_{j+1}, d(x) from d_j;
      energy  E = 1/2 sum_j w_j <L~v~_j, v~_j> + (1/sigma^2) mean r^2 (trapezoid weights w_j);
      gradient at node j (the integrand of Eq. 32 at t_j, the Riesz representative for the
              weighted product <a, b>_w = sum_j w_j <a_j, b_j>):
              g_j = L~v~_j + rho~_j - pi((D iota u~_j)^T iota rho~_j);
      Gauss-Newton Hessian likewise with drho~ and the incremental state
              D~_t du~ = dv~_t - D~u~ * dv~_t.
    Image variant: m_{j+1} = m_j o X_j; lambda_j = Heun step of -D_t lambda = lambda div v_t
    along X+_j; g_j = L~v~_j + pi(iota(pi lambda_j) iota(grad~ m~_j)); the incremental state
    dm~ with right-hand sides -grad~ m~_j * dv~_j, dlambda~ along X+_j, H_j likewise.
    State-equation variant: u~ as above, nu~_j = pi[iota(nu~_{j+1}) o X+_j - dt/2 (v_{j+1}(X+_j)
    + v_j(x))], U~ with d_{j+1}(X+_j) and d_j(x), lambda_j = J_j lambda(1) o psi_j, g_j and H_j
    as for the image variant with these m_j and lambda_j.
    With all nodes equal each reduces to Problem (the weighted sum of g_j is the stationary
    gradient)."""

    def inner(self, a, b):
        return float(sum(w * S.inner(x, y) for w, x, y in zip(self.tw, a, b)))

    def precond(self, c):
        return np.stack([S.apply_Linv(cj, self.p.alpha, self.p.s) for cj in c])

    def zeros(self):
        K = self.p.K
        return np.zeros((self.p.nt + 1, 3, K, K, K), dtype=np.complex128)

    def velocities(self, vts):
        return [self.velocity(vt) for vt in vts]

    def _offsets(self, vel):
        p = self.p
        Df = [SL.departure_offsets_ns(vel[j + 1][1], vel[j][1], self.dt, +1, p.order)
              for j in range(p.nt)]
        Db = [SL.departure_offsets_ns(vel[j][1], vel[j + 1][1], self.dt, -1, p.order)
              for j in range(p.nt)]
        return Df, Db

    def energy_reg(self, vts):
        return float(sum(w * 0.5 * S.inner(S.apply_L(vt, self.p.alpha, self.p.s), vt)
                         for w, vt in zip(self.tw, vts)))

    def state_defstate(self, vts):
        p = self.p
        vel = self.velocities(vts)
        Df, _ = self._offsets(vel)
        u = np.zeros((3, p.K, p.K, p.K), dtype=np.complex128)
        us = [u]
        for j in range(p.nt):
            u = SL.bl_heun_source_step(u, Df[j], vel[j][0], vel[j + 1][0], self.dt, p.order,
                                       self.shape, p.K)
            us.append(u)
        return us

    def _adjoint_ns(self, rho_end, vel, Db):
        p = self.p
        rhos = [None] * (p.nt + 1)
        rhos[p.nt] = rho = rho_end
        for j in range(p.nt - 1, -1, -1):
            rho = SL.bl_heun_divergence_step_ns(rho, Db[j], vel[j + 1][2], vel[j][2], self.dt,
                                                p.order, self.shape, p.K)
            rhos[j] = rho
        return rhos

    def _assemble_ns(self, base, rhos, Jus):
        out = []
        for bj, rho, Ju in zip(base, rhos, Jus):
            JT = np.einsum("abzyx,azyx->bzyx", Ju, S.include(rho, self.shape))
            out.append(S.apply_L(bj, self.p.alpha, self.p.s) + rho - S.project(JT, self.p.K))
        return np.stack(out)

    def state_image(self, vts):
        Df, _ = self._offsets(self.velocities(vts))
        ms = [self.I0.copy()]
        for j in range(self.p.nt):
            ms.append(SL.transport_step(ms[-1], Df[j], self.p.order))
        return ms

    def inverse_maps(self, vts):
        p = self.p
        vel = self.velocities(vts)
        _, Db = self._offsets(vel)
        nu = np.zeros((3, p.K, p.K, p.K), dtype=np.complex128)
        U = np.zeros((p.K, p.K, p.K), dtype=np.complex128)
        nus, Us = [None] * (p.nt + 1), [None] * (p.nt + 1)
        nus[p.nt], Us[p.nt] = nu, U
        for j in range(p.nt - 1, -1, -1):
            nu = SL.bl_heun_source_step(nu, Db[j], -vel[j + 1][0], -vel[j][0], self.dt, p.order,
                                        self.shape, p.K)
            U = SL.bl_heun_jacobian_step_ns(U, Db[j], vel[j + 1][2], vel[j][2], self.dt, p.order,
                                            self.shape, p.K)
            nus[j], Us[j] = nu, U
        return nus, Us

    def _assemble_image_ns(self, base, lams, gms, project_lam=True):
        out = []
        for bj, lam, gm in zip(base, lams, gms):
            lt = S.project(lam, self.p.K) if project_lam else lam
            out.append(S.apply_L(bj, self.p.alpha, self.p.s)
                       + S.project(S.include(lt, self.shape)[None] * gm, self.p.K))
        return np.stack(out)

    def _inc_defstate_ns(self, vts, dvts, us, Df):
        p = self.p
        Jus = self._jacobians(us)
        dvs = [S.include(dv, self.shape) for dv in dvts]
        F = [dv - np.einsum("abzyx,bzyx->azyx", Ju, dv) for Ju, dv in zip(Jus, dvs)]
        du = np.zeros((3, p.K, p.K, p.K), dtype=np.complex128)
        for j in range(p.nt):
            du = SL.bl_heun_source_step(du, Df[j], F[j], F[j + 1], self.dt, p.order, self.shape, p.K)
        return du

    def objective(self, vts):
        if self.p.variant == IMAGE:
            m1 = self.state_image(vts)[-1]
        else:
            m1, _ = self._warp_I0(self.state_defstate(vts)[-1])
        er, ed = self.energy_reg(vts), self.energy_data(m1)
        return er + ed, er, ed, m1

    def gradient(self, vts):
        p = self.p
        vel = self.velocities(vts)
        _, Db = self._offsets(vel)
        if p.variant == IMAGE:
            ms = self.state_image(vts)
            m1 = ms[-1]
            lams = [None] * (p.nt + 1)
            lams[p.nt] = lam = -(2.0 / p.sigma2) * (m1 - self.I1)
            for j in range(p.nt - 1, -1, -1):
                lam = SL.heun_divergence_step_ns(lam, Db[j], vel[j + 1][2], vel[j][2], self.dt, p.order)
                lams[j] = lam
            g = self._assemble_image_ns(vts, lams, self._grad_mtilde(ms))
            er, ed = self.energy_reg(vts), self.energy_data(m1)
            return er + ed, er, ed, g
        if p.variant == STATE:
            us = self.state_defstate(vts)
            m1, _ = self._warp_I0(us[-1])
            nus, Us = self.inverse_maps(vts)
            lams = self._pull_back(-(2.0 / p.sigma2) * (m1 - self.I1), nus, Us)
            g = self._assemble_image_ns(vts, lams, self._grad_mtilde(self._compose_I0(us)))
            er, ed = self.energy_reg(vts), self.energy_data(m1)
            return er + ed, er, ed, g
        us = self.state_defstate(vts)
        m1, G = self._warp_I0(us[-1])
        rho1 = S.project(-(2.0 / p.sigma2) * (m1 - self.I1)[None] * G, p.K)
        rhos = self._adjoint_ns(rho1, vel, Db)
        g = self._assemble_ns(vts, rhos, self._jacobians(us))
        er, ed = self.energy_reg(vts), self.energy_data(m1)
        return er + ed, er, ed, g

    def hessian_matvec(self, vts, dvts):
        p = self.p
        vel = self.velocities(vts)
        Df, Db = self._offsets(vel)
        if p.variant == IMAGE:
            ms = self.state_image(vts)
            gms = self._grad_mtilde(ms)
            F = [-np.sum(gm * S.include(dv, self.shape), axis=0) for gm, dv in zip(gms, dvts)]
            dm = np.zeros((p.K, p.K, p.K), dtype=np.complex128)
            for j in range(p.nt):
                dm = SL.bl_heun_source_step(dm, Df[j], F[j], F[j + 1], self.dt, p.order, self.shape, p.K)
            dlams = [None] * (p.nt + 1)
            dlams[p.nt] = dlam = -(2.0 / p.sigma2) * dm
            for j in range(p.nt - 1, -1, -1):
                dlam = SL.bl_heun_divergence_step_ns(dlam, Db[j], vel[j + 1][2], vel[j][2], self.dt,
                                                     p.order, self.shape, p.K)
                dlams[j] = dlam
            return self._assemble_image_ns(dvts, dlams, gms, project_lam=False)
        us = self.state_defstate(vts)
        _, G = self._warp_I0(us[-1])
        dm1 = -np.sum(G * S.include(self._inc_defstate_ns(vts, dvts, us, Df), self.shape), axis=0)
        if p.variant == STATE:
            nus, Us = self.inverse_maps(vts)
            dlams = self._pull_back(-(2.0 / p.sigma2) * dm1, nus, Us)
            return self._assemble_image_ns(dvts, dlams, self._grad_mtilde(self._compose_I0(us)))
        Jus = self._jacobians(us)
        drho1 = S.project(-(2.0 / p.sigma2) * dm1[None] * G, p.K)
        drhos = self._adjoint_ns(drho1, vel, Db)
        return self._assemble_ns(dvts, drhos, Jus)
