"""Semi-Lagrangian Runge-Kutta (SL-RK) integration: characteristics and Table 1 steps. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 3.1 -- departure points from the characteristic equation D_t X = v(t, X) with
the two-stage scheme of Eqs. 40-42 (X* = x - dt v; v* = v(X*); X = x - dt/2 (v* + v)),
then the transport equation D_t u = f(u, v) (Eq. 38) solved on the Eulerian grid along the
characteristic (Eq. 43) with a Runge-Kutta step. Sec. 3.2 -- in the band-limited domain the
characteristics come from iota(v~) (Eq. 46) and the equation is D~_t u~ = f~ (Eq. 44).
Sec. 3.3 / Table 1 -- the SL form of each state, adjoint and incremental equation.

Readings (the cited works that define the RK step are not in the paper):
  * RK step = Heun (explicit trapezoid): with departure point X of the grid point x,
        u^{j+1}(x) = u^j(X) + dt/2 [ f_j(X) + f_{j+1}(x) ],
    where f_j(X) is the right-hand side at the old time level evaluated at X, and
    f_{j+1}(x) the right-hand side at the new level at x, using the Euler predictor
    u* = u^j(X) + dt f_j(X) wherever f depends on the unknown.
  * Equations marked "-D_t" (adjoints) run backward in time, t from 1 to 0. With tau = 1 - t
    they are forward transports along -v, so their departure points X+ come from the same
    two-stage scheme with +dt v.
  * Band-limited steps: each step is iota -> the spatial Heun step on the grid -> pi, so the
    unknown stays in V~ at every time node.
  * Stationary velocity: X and X+ are computed once and reused by every step.

Units: velocities passed here are voxel units per unit time (the physical velocity of
[0, 2 pi)^3 times N_a / (2 pi)); offsets are voxels.
"""
from __future__ import annotations

import numpy as np

from . import interp as I
from . import spectral as S


def departure_offsets(V, dt, direction, order):
    """Offsets D = X - x of the departure points for one time step (Eqs. 40-42).

    direction = +1: forward-in-time equations (X* = x - dt V; X = x - dt/2 (V(X*) + V)).
    direction = -1: backward-in-time (adjoint) equations, the same scheme along -V.
    V: voxel-unit velocity [3][nz][ny][nx]; order: 1 trilinear, 3 cubic B-spline.
    """
    sgn = -1.0 if direction > 0 else 1.0
    Dstar = sgn * dt * V                       # X* - x
    Vstar = I.interpolate(V, Dstar, order)     # v* = v o X*
    return sgn * 0.5 * dt * (Vstar + V)        # X - x


def departure_offsets_ns(V_here, V_other, dt, direction, order):
    """Offsets of one step between two nodes with different velocities (non-stationary v).

    direction = +1 (state, arrival node t_{j+1}): X* = x - dt V_{j+1}(x),
    X = x - dt/2 (V_{j+1}(x) + V_j(X*)), i.e. V_here = V_{j+1}, V_other = V_j.
    direction = -1 (adjoint, arrival node t_j of the backward sweep): X+* = x + dt V_j(x),
    X+ = x + dt/2 (V_j(x) + V_{j+1}(X+*)), i.e. V_here = V_j, V_other = V_{j+1}.
    With V_here = V_other this is departure_offsets."""
    sgn = -1.0 if direction > 0 else 1.0
    Dstar = sgn * dt * V_here
    Vstar = I.interpolate(V_other, Dstar, order)
    return sgn * 0.5 * dt * (Vstar + V_here)


def transport_step(u, D, order):
    """D_t u = 0 (Table 1 row 1, state equation in SL form): u^{j+1}(x) = u^j(X)."""
    return I.interpolate(u, D, order)


def heun_source_step(u, D, F_old, F_new, dt, order):
    """D_t u = F(t) with a right-hand side independent of u (Table 1 rows 3, 5, 7):
    u^{j+1}(x) = u^j(X) + dt/2 [ F_j(X) + F_{j+1}(x) ]."""
    return I.interpolate(u, D, order) + 0.5 * dt * (I.interpolate(F_old, D, order) + F_new)


def heun_divergence_step(u, Dplus, d, dt, order):
    """-D_t u = u div v (Table 1 rows 2, 4, 6, 8), one step backward in time.

    Along the backward characteristic the equation reads D_tau u = u d with d = div v, so
    a = u^{j+1}(X+); f_old = a d(X+); u* = a + dt f_old; u^j(x) = a + dt/2 (f_old + u* d(x)).
    """
    a = I.interpolate(u, Dplus, order)
    d_dep = I.interpolate(d, Dplus, order)
    f_old = a * d_dep
    u_star = a + dt * f_old
    return a + 0.5 * dt * (f_old + u_star * d)


def heun_jacobian_step(U, Dplus, d, dt, order):
    """-D_t U = -div v + U div v (the Jacobian equation of the state-equation variant,
    Sec. 2.3.2), one step backward in time.

    Along the backward characteristic D_tau U = d (U - 1) with d = div v, so
    a = U^{j+1}(X+); f_old = d(X+) (a - 1); U* = a + dt f_old;
    U^j(x) = a + dt/2 (f_old + d(x) (U* - 1))."""
    a = I.interpolate(U, Dplus, order)
    f_old = I.interpolate(d, Dplus, order) * (a - 1.0)
    u_star = a + dt * f_old
    return a + 0.5 * dt * (f_old + d * (u_star - 1.0))


def heun_jacobian_step_ns(U, Dplus, d_next, d_here, dt, order):
    """heun_jacobian_step between nodes t_j and t_{j+1} (non-stationary v): d(X+) from d_{j+1},
    d(x) from d_j."""
    a = I.interpolate(U, Dplus, order)
    f_old = I.interpolate(d_next, Dplus, order) * (a - 1.0)
    u_star = a + dt * f_old
    return a + 0.5 * dt * (f_old + d_here * (u_star - 1.0))


def heun_divergence_step_ns(u, Dplus, d_next, d_here, dt, order):
    """-D_t u = u div v_t between nodes t_j and t_{j+1} (non-stationary v): as
    heun_divergence_step with d(X+) taken from d_{j+1} and d(x) from d_j."""
    a = I.interpolate(u, Dplus, order)
    f_old = a * I.interpolate(d_next, Dplus, order)
    u_star = a + dt * f_old
    return a + 0.5 * dt * (f_old + u_star * d_here)


def sl_transport(field, V, nt, direction, order):
    """nt steps of D_t u = 0 (forward) or -D_t u = 0 (backward) with stationary V.

    This is the unit the SL throughput metric counts: one grid point advanced one step.
    """
    dt = 1.0 / nt
    D = departure_offsets(V, dt, direction, order)
    u = np.asarray(field, dtype=np.float64)
    for _ in range(nt):
        u = transport_step(u, D, order)
    return u


# ----- band-limited forms (Sec. 3.2: the unknown lives in V~; iota -> SL step -> pi) -----

def bl_transport_step(c, D, order, shape, K):
    """One BL step of D~_t u~ = 0: pi( iota(u~) o X )."""
    return S.project(transport_step(S.include(c, shape), D, order), K)


def bl_heun_source_step(c, D, F_old, F_new, dt, order, shape, K):
    """One BL step of D~_t u~ = F with spatial right-hand sides F_j, F_{j+1} on the grid."""
    return S.project(heun_source_step(S.include(c, shape), D, F_old, F_new, dt, order), K)


def bl_heun_jacobian_step_ns(c, Dplus, d_next, d_here, dt, order, shape, K):
    """One backward BL step of the U~ equation with node-dependent divergence."""
    return S.project(heun_jacobian_step_ns(S.include(c, shape), Dplus, d_next, d_here, dt, order), K)


def bl_heun_divergence_step_ns(c, Dplus, d_next, d_here, dt, order, shape, K):
    """One backward BL step of -D~_t u~ = u~ * div~ v~_t with node-dependent divergence."""
    return S.project(heun_divergence_step_ns(S.include(c, shape), Dplus, d_next, d_here, dt, order), K)


def bl_heun_jacobian_step(c, Dplus, d, dt, order, shape, K):
    """One backward BL step of -D~_t U~ = -div~ v~ + U~ * div~ v~ (Sec. 2.3.2)."""
    return S.project(heun_jacobian_step(S.include(c, shape), Dplus, d, dt, order), K)


def bl_heun_divergence_step(c, Dplus, d, dt, order, shape, K):
    """One backward BL step of -D~_t u~ = u~ * div~ v~ (Table 1 rows 4, 6, 8)."""
    return S.project(heun_divergence_step(S.include(c, shape), Dplus, d, dt, order), K)
