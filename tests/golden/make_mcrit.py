"""Writes tests/golden/mcrit.json: the critical mass of each synthetic gauge
field used by the tests and the benchmark, computed by the oracle's spectrum
routine (m_crit = -min Re lambda(D at m0 = 0)) on the quenched Metropolis
fields of the fixtures module (500 sweeps from a cold start).

    python tests/golden/make_mcrit.py [--serving] [--tol T] [L ...]
        L ...      only these lattice sizes (default: all)
        --serving  also the eight serving fields per size
        --tol T    ARPACK's relative tolerance (default 1e-6; the entries
                   computed with another one record it)

Only the oracle and the input fixtures are called.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import spectrum  # noqa: E402
from paper_2608_03515_b300 import fixtures as fx  # noqa: E402

OUT = os.path.join(HERE, "mcrit.json")
SWEEPS = 500

# (L, beta, seed): the 32^2 field at beta = 3 (seed 0), the 256^2 field at
# beta = 6 (seed 2), the 512^2 field at beta = 10 (seed 4), the 1024^2 field at
# beta = 12 (seed 5), and the serving fields k = 0..7 (beta = 2 + 10 k / 7,
# seed 10 + k) at every serving lattice size.
FIELDS = [(32, 3.0, 0), (256, 6.0, 2), (512, 10.0, 4), (1024, 12.0, 5)]
SERVING = [(L, round(2.0 + 10.0 * k / 7.0, 12), 10 + k) for L in (64, 128, 256, 512, 1024) for k in range(8)]


def key(L, beta, seed):
    return f"L{L}_b{beta:g}_s{seed}"


def main(sizes=None, serving=False, tol=1e-6):
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for (L, beta, seed) in FIELDS + (SERVING if serving else []):
        if sizes and L not in sizes:
            continue
        k = key(L, beta, seed)
        if k in table:
            continue
        t0 = time.time()
        theta = fx.metropolis_u1(L, L, beta, SWEEPS, seed)
        mc = spectrum.critical_mass(fx.links_from_angles(theta), tol=tol)
        entry = {"L": L, "beta": beta, "seed": seed, "sweeps": SWEEPS, "m_crit": mc}
        if tol != 1e-6:
            entry["arpack_tol"] = tol
        print(k, mc, f"{time.time() - t0:.1f}s", flush=True)
        # merge with what other runs wrote meanwhile
        table = json.load(open(OUT)) if os.path.exists(OUT) else {}
        table[k] = entry
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    tol = float(args[args.index("--tol") + 1]) if "--tol" in args else 1e-6
    main([int(a) for a in args if a.isdigit()] or None, serving="--serving" in args, tol=tol)
