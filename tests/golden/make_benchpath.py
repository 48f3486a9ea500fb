"""Writes the stored oracle results of the bench-path parity workload.

Calls only the FP64 oracle (``oracle/``) on seeded generator inputs; nothing here touches
the GPU library. The inputs are those of ``_problems.bench_phantom_problem`` (the ellipsoid
phantom at 96 x 112 x 96 warped by a random band-limited velocity, N(0, 0.01) noise, K = 32,
deformation-state variant, Sec. 2.3.3) and ``_problems.small_phantom_problem`` (the same recipe
at 32^3, K = 16); the tests rebuild the inputs and read the oracle's outputs from here, because
the FP64 gradient and Gauss-Newton product at a million voxels take minutes of host time.

Outputs:
- ``benchpath_o{order}_nt{nt}_{noisy|clean}.npz``: the oracle's energy E, gradient g (Eqs.
  32-33 with the adjoint of Eq. 35) and Gauss-Newton product Hp (Eqs. 36-37) at
  ``bench_velocity()``, and <p, Hp>; g and Hp stored as complex64, E and <p, Hp> in FP64.
  p is the first PCG direction L~^{-1}(-g), formed from the stored g by
  ``_problems.first_direction`` and rounded to complex64 (the precision the GPU receives its
  arguments in), so that a test forms the same p bit for bit.
- ``benchpath_registration_o{order}.json``: the oracle's Gauss-Newton registration of the
  32^3 pair (nt = 4, 3 GN x <= 20 PCG): iteration counts, stop reason, energy, relative
  residual and the per-iterate history.

    python tests/golden/make_benchpath.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import gnk, spectral as S  # noqa: E402
from _problems import (bench_phantom_problem, bench_velocity, first_direction,  # noqa: E402
                       small_phantom_problem)

GRAD_CASES = [(1, 3, False), (1, 3, True), (3, 2, True)]   # (order, nt, noisy)
REG_CASES = [1, 3]                                         # interpolation order
REG_NT, REG_MAX_GN, REG_MAX_PCG = 4, 3, 20


def grad_name(order, nt, noisy):
    return f"benchpath_o{order}_nt{nt}_{'noisy' if noisy else 'clean'}.npz"


def reg_name(order):
    return f"benchpath_registration_o{order}.json"


def write_grad(order, nt, noisy):
    prob = bench_phantom_problem(order, nt, noisy)
    vt = bench_velocity()
    E, _, _, g = prob.gradient(vt)
    g32 = g.astype(np.complex64)
    p = first_direction(g32, prob.p.alpha, prob.p.s)
    Hp = prob.hessian_matvec(vt, p)
    np.savez_compressed(os.path.join(HERE, grad_name(order, nt, noisy)), E=np.float64(E),
                        g=g32, Hp=Hp.astype(np.complex64), pHp=np.float64(S.inner(p, Hp)))


def write_reg(order):
    prob = small_phantom_problem(order, nt=REG_NT)
    _, rep = gnk.register(prob, max_gn=REG_MAX_GN, max_pcg=REG_MAX_PCG)
    out = {"gn_iters": int(rep.gn_iters), "pcg_iters_total": int(rep.pcg_iters_total),
           "stop_reason": int(rep.stop_reason), "E": float(rep.E),
           "grad_rel_l2": float(rep.grad_rel_l2),
           "history": [[float(a), float(b)] for a, b in rep.history],
           "config": {"shape": [32, 32, 32], "K": 16, "nt": REG_NT, "order": order,
                      "max_gn": REG_MAX_GN, "max_pcg": REG_MAX_PCG}}
    with open(os.path.join(HERE, reg_name(order)), "w") as f:
        json.dump(out, f, indent=1)


def main():
    for case in GRAD_CASES:
        write_grad(*case)
        print("wrote", grad_name(*case))
    for order in REG_CASES:
        write_reg(order)
        print("wrote", reg_name(order))


if __name__ == "__main__":
    main()
