"""Writes tests/golden/c4_oracle.json: the oracle's FP64 solves of the first
four right-hand sides of the many-right-hand-side workload (1024 x 1024
lattice, quenched U(1) at beta = 12, 500 Metropolis sweeps from seed 5,
m0 = m_ref + 0.01 with m_ref the critical mass of the 256 x 256 beta = 12 field
(seed 17) in tests/golden/mcrit.json, SM-AMG with tile sides 4 then 4
(coarsest 64 x 64 solved exactly), FGMRES(30) to a true relative residual of
1e-10; right-hand sides: the first four of fixtures.gaussian_rhs(64, 1024,
1024, 6)).

The 1024 x 1024 field's own critical mass is not tabulated: the oracle's
Arnoldi route (eigenvalues of smallest real part) had not converged after
1 h 51 min on this host, and shift-invert needs a sparse LU that took 233 s
already at 128 x 128.  The critical masses of the beta = 12 fields at 64^2,
128^2 and 256^2 lie within 0.008 of each other, so m_ref + 0.01 keeps the
operator's spectrum to the right of the origin with margin.

For each of the four it stores the outer iteration count, the true relative
residual and the solution at 32 sampled sites (both spins), so that the GPU's
solutions can be compared element by element at those sites.

    python tests/golden/make_c4_oracle.py [--workers N]

Only the oracle and the input fixtures are called.  The hierarchy is built
once; the four solves run in forked worker processes (no GPU is involved).
"""
import json
import multiprocessing
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import amg, krylov  # noqa: E402
from oracle import wilson as W  # noqa: E402
from paper_2608_03515_b300 import fixtures as fx  # noqa: E402

OUT = os.path.join(HERE, "c4_oracle.json")
L, BETA, FIELD_SEED, SWEEPS = 1024, 12.0, 5, 500
MASS_REF, DM, AGGS, RESTART, TOL = "L256_b12_s17", 0.01, [4, 4], 30, 1e-10
RHS_SEED, NCHECK, NSAMPLE, SAMPLE_SEED = 6, 4, 32, 7

_state = {}


def _solve(r):
    D, levels, b = _state["D"], _state["levels"], _state["psi"][r]
    t0 = time.time()
    res = krylov.fgmres(lambda v: D @ v, lambda v: amg.vcycle(levels, v), W.to_flat(b), RESTART, TOL, 5000)
    x = W.from_flat(res.x, L, L)
    sites = _state["sites"]
    sample = [[[float(x[a, t, xx].real), float(x[a, t, xx].imag)] for a in range(2)] for (t, xx) in sites]
    return {"rhs": r, "iterations": res.iterations, "true_relres": res.true_relres, "converged": res.converged,
            "x_norm": float(np.linalg.norm(res.x)), "x_at_sites": sample, "seconds": time.time() - t0}


def main(workers):
    table = json.load(open(os.path.join(HERE, "mcrit.json")))
    mc = table[MASS_REF]["m_crit"]
    m0 = mc + DM
    t0 = time.time()
    theta = fx.metropolis_u1(L, L, BETA, SWEEPS, FIELD_SEED)
    U = fx.links_from_angles(theta)
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, L, L, AGGS)
    print(f"field + hierarchy {time.time() - t0:.0f} s", flush=True)
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    sites = [(int(t), int(x)) for t, x in zip(rng.integers(0, L, NSAMPLE), rng.integers(0, L, NSAMPLE))]
    _state.update(D=D, levels=levels, psi=fx.gaussian_rhs(NCHECK, L, L, RHS_SEED), sites=sites)
    with multiprocessing.get_context("fork").Pool(workers) as pool:
        rows = pool.map(_solve, range(NCHECK))
    out = {"L": L, "beta": BETA, "seed": FIELD_SEED, "sweeps": SWEEPS, "mass_ref": MASS_REF, "m_ref": mc, "m0": m0,
           "tiles": AGGS,
           "restart": RESTART, "tol": TOL, "rhs_seed": RHS_SEED, "rhs_count": 64, "checked": NCHECK,
           "sites": sites, "solves": rows}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps([(r["rhs"], r["iterations"], r["true_relres"], round(r["seconds"])) for r in rows]))


if __name__ == "__main__":
    args = sys.argv[1:]
    main(int(args[args.index("--workers") + 1]) if "--workers" in args else NCHECK)
