"""Writes the stored expected values under tests/golden/ by calling the oracle only.

    python tests/golden/make_golden.py            # small fixtures
    python tests/golden/make_golden.py --large    # adds the 256^3 iteration count (about a minute)
    python tests/golden/make_golden.py --config2  # the 512^3 lognormal solution on a lattice (minutes)
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


# lattice of the stored 512^3 solution values: every 32nd point from 16 on each axis (16^3 points)
LATTICE_START, LATTICE_STEP = 16, 32


def config2_512():
    """512^3 lognormal block coefficients (8^3 blocks, seed 1), b ~ U[-1,1) seed 1, x0 = 0,
    Jacobi-PCG to 1e-10 (two orders below the solves it is compared with): the solution on the
    lattice, with the full solution's 2-norm and the true residual."""
    n = 512
    k, b = inputs.varcoeff_problem(n, n, n, seed=1, kb=8, dtype=np.float64)
    k = k.astype(np.float64)
    res = oracle.pcg(b, tol=1e-10, maxit=40000, k=k, kb=8)
    x = res["x"]
    sl = slice(LATTICE_START, None, LATTICE_STEP)
    return dict(workload="lognormal 512^3 kb 8 seed 1 jacobi", n=n, seed=1, kb=8, tol=1e-10,
                iters=res["iters"], status=res["status"], relres=res["relres"],
                true_relres=oracle.true_relres(b, x, k, 8), x_norm2=float(np.linalg.norm(x)),
                lattice_start=LATTICE_START, lattice_step=LATTICE_STEP,
                x_lattice=x[sl, sl, sl].ravel().tolist())


if __name__ == "__main__":
    with open(os.path.join(HERE, "pcg_poisson32_seed0.json"), "w") as f:
        json.dump(poisson32(), f, indent=1)
    if "--large" in sys.argv:
        with open(os.path.join(HERE, "pcg_poisson256_seed0.json"), "w") as f:
            json.dump(poisson256(), f, indent=1)
    if "--config2" in sys.argv:
        with open(os.path.join(HERE, "pcg_lognormal512_seed1_lattice.json"), "w") as f:
            json.dump(config2_512(), f)
