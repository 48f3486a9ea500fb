"""Gauss-Newton-Krylov optimisation in V~: PCG with L~^{-1}, update length, stopping. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 2.1 (Eqs. 7-8) and Sec. 2.2 (Eqs. 13-14): v~^{n+1} = v~^n + eps dv~^n, with
dv~^n from preconditioned conjugate gradients on H dv~ = -g~, preconditioner L~^{-1};
Sec. 4.3: at most 10 Gauss-Newton iterations and 5 PCG iterations in the paper's runs.

Readings (the stopping rules of the cited work are not written out in the paper):
  * PCG: zero initial guess; stop when ||r|| <= eta ||g|| with forcing
    eta = min(0.5, sqrt(||g_n|| / ||g_ref||)), or at max_pcg iterations, or on
    non-positive curvature (if that happens at the first iteration, the preconditioned
    steepest-descent direction L~^{-1}(-g) is returned).
  * Update length eps: Armijo backtracking from eps = 1, halving up to 10 times, accepting
    E(v + eps dv) <= E(v) + 1e-4 eps <g, dv>; no acceptable eps stops with LINESEARCH.
  * Stop when ||g_n||_2 / ||g_ref||_2 <= gtol, g_ref the gradient at v~ = 0 (the cold-start
    gradient, so warm starts are measured against the same reference), or after max_gn
    updates.
  * ``two_level = m > 0`` replaces L~^{-1} by the two-level preconditioner of
    ``oracle/multilevel.py`` (at most m coarse PCG iterations per application) and PCG by
    flexible PCG; the coarse Hessian is re-taken at every Gauss-Newton iterate.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import spectral as S

STOP_GTOL = 1
STOP_MAXIT = 2
STOP_LINESEARCH = 3


def pcg(hv, b, prec, eta, maxit, inner=S.inner):
    """Preconditioned CG for H x = b from x = 0. Returns (x, iterations, negative_curvature)."""
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
                return prec(b), its, True
            return x, its, True
        a = rz / pHp
        x = x + a * p
        r = r - a * Hp
        if np.sqrt(inner(r, r)) <= eta * bnorm:
            break
        z = prec(r)
        rz_new = inner(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, its, False


@dataclass
class Report:
    gn_iters: int = 0
    pcg_iters_total: int = 0
    stop_reason: int = 0
    E0: float = 0.0
    E: float = 0.0
    E_reg: float = 0.0
    E_data: float = 0.0
    grad_rel_l2: float = 0.0
    grad_rel_inf: float = 0.0
    mse_rel: float = 0.0
    pcg_inner_total: int = 0
    history: list = field(default_factory=list)


def register(problem, v0=None, max_gn=5, max_pcg=10, gtol=1e-3, g_ref=None, two_level=0):
    """Gauss-Newton-Krylov registration from v0 (zero by default). Returns (v~, Report)."""
    p = problem.p
    K = p.K
    # the problem may define its own unknown (a stack of cubes), product and preconditioner
    inner = getattr(problem, "inner", S.inner)
    if hasattr(problem, "zeros"):
        v = problem.zeros() if v0 is None else np.array(v0, problem.zeros().dtype)
        prec = problem.precond
    else:
        v = np.zeros((3, K, K, K), dtype=np.complex128) if v0 is None else np.array(v0, np.complex128)
        prec = lambda c: S.apply_Linv(c, p.alpha, p.s)
    solver = pcg
    tl = None
    if two_level > 0:
        from . import multilevel as ML

        tl = ML.TwoLevel(problem, ML.coarse_problem(problem), two_level)
        prec, solver = tl, ML.fpcg
    if g_ref is None:
        g_ref = problem.gradient(np.zeros_like(v))[3] if v0 is not None else None
    rep = Report()
    E, Er, Ed, g = problem.gradient(v)
    if g_ref is None:
        g_ref = g
    gref_l2 = np.sqrt(inner(g_ref, g_ref))
    gref_inf = np.abs(g_ref).max()
    rep.E0 = E
    for n in range(max_gn):
        gn = np.sqrt(inner(g, g))
        rep.history.append((E, gn / gref_l2))
        if gn / gref_l2 <= gtol:
            rep.stop_reason = STOP_GTOL
            break
        eta = min(0.5, np.sqrt(gn / gref_l2))
        if tl is not None:
            tl.set_velocity(v)
        dv, its, _ = solver(lambda c: problem.hessian_matvec(v, c), -g, prec, eta, max_pcg, inner)
        rep.pcg_iters_total += its
        slope = inner(g, dv)
        eps, accepted = 1.0, False
        for _ in range(11):
            Et = problem.objective(v + eps * dv)[0]
            if Et <= E + 1e-4 * eps * slope:
                accepted = True
                break
            eps *= 0.5
        if not accepted:
            rep.stop_reason = STOP_LINESEARCH
            break
        v = v + eps * dv
        rep.gn_iters = n + 1
        E, Er, Ed, g = problem.gradient(v)
    else:
        rep.stop_reason = STOP_MAXIT
    gn = np.sqrt(inner(g, g))
    if rep.stop_reason == STOP_MAXIT and gn / gref_l2 <= gtol:
        rep.stop_reason = STOP_GTOL
    m1 = problem.objective(v)[3]
    rep.E, rep.E_reg, rep.E_data = E, Er, Ed
    rep.grad_rel_l2 = gn / gref_l2
    rep.grad_rel_inf = np.abs(g).max() / gref_inf
    rep.mse_rel = problem.mse_rel(m1)
    if tl is not None:
        rep.pcg_inner_total = tl.inner_its
    return v, rep
