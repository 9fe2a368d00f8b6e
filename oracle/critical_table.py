"""Writes tests/golden/critical_rayleigh.json: the critical Rayleigh number
Ra_c(E) at Pr = 1, radius ratio 0.35, no Ekman pumping, from the onset
eigenproblem of ``oracle.onset`` (Section 6.1, Eq. lin).  The workloads give Ra as
a multiple of Ra_c.  Calls only the oracle.

    python -m oracle.critical_table
"""
import json
import os
import sys

import numpy as np

from .onset import marginal_rayleigh

CASES = [  # E, radial resolution n_c, initial Ra guess, m scan range, drift-frequency guess
    (1e-3, 48, 5e4, range(1, 10), None),
    (1e-5, 96, 5e6, range(6, 26), None),
    (1e-6, 160, 1.7e8, range(32, 46), None),
    (1e-4, 64, 5e5, range(2, 16), None),
    # at E = 1e-8 the QZ estimate without a guess lands on spurious branches of the
    # tau pencil; the scan follows the thermal Rossby wave from omega_d ~ -1e5
    (1e-8, 320, 6.0e10, range(132, 157, 6), -1.0e5j),
]


def critical(E, n_c, ra0, ms, guess=None, log=lambda *a: print(*a, flush=True)):
    best = None
    ra_guess = ra0
    prev = None
    for m in ms:
        ra, lam = marginal_rayleigh(E, 1.0, 0.35, m, n_c, ra_guess, guess=guess)
        log("E=%g m=%d Ra=%.8e omega=%.6e" % (E, m, ra, lam.imag))
        # with a branch guess every mode starts from the same Ra below onset (a
        # start above the marginal Ra lets the continuation lose the branch)
        ra_guess = ra if guess is None else ra0
        if best is None or ra < best[0]:
            best = (ra, m, lam.imag)
        if prev is not None and ra > prev and m > best[1] + 2:
            break
        prev = ra
    return best


def main(out=None):
    out = out or os.path.join(os.path.dirname(__file__), "..", "tests", "golden", "critical_rayleigh.json")
    which = [float(a) for a in sys.argv[1:]] or None
    table = {}
    if os.path.exists(out):
        table = json.load(open(out))
    for E, nc, ra0, ms, guess in CASES:
        if which and E not in which:
            continue
        ra, m, om = critical(E, nc, ra0, ms, guess)
        table["%g" % E] = {"Ra_c": ra, "m_c": m, "omega_d": om, "Pr": 1.0, "eta": 0.35, "n_c": nc,
                           "source": "oracle.onset, integration/tau operators, no Ekman pumping"}
        json.dump(table, open(out, "w"), indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    main()
