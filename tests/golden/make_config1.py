"""Writes the stored oracle result of the small registration workload.

Calls only the FP64 oracle (``oracle/``) on seeded generator inputs; nothing here touches
the GPU library. Output: ``config1_seed0.npz`` (the oracle's final velocity cube) and
``config1_seed0.json`` (its report). Workload: 32^3 Gaussian-blob pair warped by a random
stationary band-limited velocity (8^3 modes, 3 voxels max), deformation-state variant,
K = 16, nt = 10, trilinear SL, alpha = 0.0025, s = 2, sigma^2 = 0.01, 5 Gauss-Newton x <= 10
PCG iterations.

    python tests/golden/make_config1.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import gnk, variants as Vn  # noqa: E402
from _problems import oracle_problem  # noqa: E402

CONFIG = dict(shape=(32, 32, 32), K=16, nt=10, variant=Vn.DEFSTATE, order=1, seed=0,
              max_gn=5, max_pcg=10, gtol=1e-3)


def main():
    c = CONFIG
    prob = oracle_problem(c["shape"], c["K"], c["variant"], c["order"], nt=c["nt"], seed=c["seed"])
    v, rep = gnk.register(prob, max_gn=c["max_gn"], max_pcg=c["max_pcg"], gtol=c["gtol"])
    np.savez_compressed(os.path.join(HERE, "config1_seed0.npz"), v=v.astype(np.complex128))
    out = {k: (float(x) if isinstance(x, (float, np.floating)) else x)
           for k, x in vars(rep).items() if k != "history"}
    out["history"] = [[float(a), float(b)] for a, b in rep.history]
    out["max_disp_vox"] = prob.max_displacement_vox(v)
    out["config"] = {k: (list(x) if isinstance(x, tuple) else x) for k, x in c.items()}
    with open(os.path.join(HERE, "config1_seed0.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
