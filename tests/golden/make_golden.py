"""Writes the stored expected values under tests/golden/ by calling the oracle only.

    python tests/golden/make_golden.py            # small fixtures
    python tests/golden/make_golden.py --large    # adds the 256^3 iteration count (about a minute)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2603_23343_gb300 import inputs  # noqa: E402


def poisson32():
    """32^3 Poisson, b ~ U[-1,1) seed 0, x0 = 0, Jacobi, tol 1e-6, maxit 2000."""
    b = inputs.poisson_problem(32, 0, np.float64)
    res = oracle.pcg(b, tol=1e-6, maxit=2000, history=True)
    return dict(workload="poisson 32^3 seed 0 jacobi", n=32, seed=0, tol=1e-6, maxit=2000,
                iters=res["iters"], status=res["status"], relres=res["relres"],
                true_relres=oracle.true_relres(b, res["x"]), hist=res["hist"].tolist())


def poisson256():
    """256^3 Poisson, b ~ U[-1,1) seed 0, x0 = 0, Jacobi, tol 1e-6 (iteration count only)."""
    b = inputs.poisson_problem(256, 0, np.float64)
    res = oracle.pcg(b, tol=1e-6, maxit=2000, history=True)
    return dict(workload="poisson 256^3 seed 0 jacobi", n=256, seed=0, tol=1e-6, maxit=2000,
                iters=res["iters"], status=res["status"], relres=res["relres"],
                hist_every_50=res["hist"][::50].tolist())


if __name__ == "__main__":
    with open(os.path.join(HERE, "pcg_poisson32_seed0.json"), "w") as f:
        json.dump(poisson32(), f, indent=1)
    if "--large" in sys.argv:
        with open(os.path.join(HERE, "pcg_poisson256_seed0.json"), "w") as f:
            json.dump(poisson256(), f, indent=1)
