"""Writes tests/golden/mcrit_dense.json: the critical mass of two 64x64 fields
from all eigenvalues of the dense Wilson-Dirac matrix (LAPACK), beside the
value of the Arnoldi route (ARPACK, eigenvalues of smallest real part) that
tabulates the larger fields in tests/golden/mcrit.json, at both of its
tolerances (1e-6, and 1e-4 for the weak-coupling fields of 256^2 and more).

    python tests/golden/make_mcrit_dense.py

Fields: the fixtures' quenched Metropolis fields, 500 sweeps from a cold start,
at the benchmark coupling (beta = 6, seed 2) and at the weak coupling of the
1024^2 workload (beta = 12, seed 5).  Entries already in the file are kept,
missing values are added.  Only the oracle and the input fixtures are called.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import spectrum  # noqa: E402
from paper_2608_03515_b300 import fixtures as fx  # noqa: E402

OUT = os.path.join(HERE, "mcrit_dense.json")
FIELDS = [(64, 6.0, 2), (64, 12.0, 5)]
SWEEPS = 500
ARPACK_TOLS = (1e-6, 1e-4)


def main():
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for (L, beta, seed) in FIELDS:
        key = f"L{L}_b{beta:g}_s{seed}"
        e = out.setdefault(key, {"L": L, "beta": beta, "seed": seed, "sweeps": SWEEPS})
        U = fx.links_from_angles(fx.metropolis_u1(L, L, beta, SWEEPS, seed))
        if "m_crit" not in e:
            t0 = time.time()
            e["m_crit"] = spectrum.critical_mass(U, dense=True)
            print(key, "dense", e["m_crit"], f"{time.time() - t0:.0f} s", flush=True)
        arp = e.setdefault("arpack", {})
        for tol in ARPACK_TOLS:
            if f"{tol:g}" not in arp:
                t0 = time.time()
                arp[f"{tol:g}"] = spectrum.critical_mass(U, dense=False, tol=tol)
                print(key, "arpack", tol, arp[f"{tol:g}"], f"{time.time() - t0:.0f} s", flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
