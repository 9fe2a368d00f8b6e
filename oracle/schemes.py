"""IMEX time schemes (Section 4, Eqs. multistep, multistep1 and dirks; Table 1).

Test infrastructure only (see the package docstring).

Multistep, constant dt, in the form of Eq. multistep1:
  (I - b0 dt Imp) y_{n+1} = sum_j a_j y_{n+1-j} + dt sum_j (bE_j Exp_{n+1-j} + bI_j Imp_{n+1-j})
  CNAB2: a = (1), b0 = 1/2, bI = (1/2), bE = (3/2, -1/2)            (Section 4)
  SBDF2: a = (4/3, -1/3), b0 = 2/3, bE = (4/3, -2/3)
  SBDF3: a = (18/11, -9/11, 2/11), b0 = 6/11, bE = (18/11, -18/11, 6/11)
  (the classical backward-differentiation / extrapolation pairs, divided by the
  coefficient of y_{n+1}).
  Start-up (the paper only says a lower-order starter is needed): CNAB2 takes
  bE = (1) on its first step; SBDF3 takes one SBDF1 (IMEX Euler) step and one
  SBDF2 step; SBDF2 takes one SBDF1 step.

Diagonally implicit (Eq. dirks), stiffly accurate, stage 0 = y_n:
  (I - a_ii dt Imp) y_i = y_n + dt sum_{j<i} (aE_ij Exp_j + aI_ij Imp_j),  y_{n+1} = y_nu
  ARS443 (Ascher, Ruuth & Spiteri 1997, Section 2.8), rows i = 0..4:
    aI: [0], [0,1/2], [0,1/6,1/2], [0,-1/2,1/2,1/2], [0,3/2,-3/2,1/2,1/2]
    aE: [0], [1/2], [11/18,1/18], [5/6,-5/6,1/2], [1/4,7/4,3/4,-7/4]
  BPR353 (Boscarino, Pareschi & Russo 2013, Section 8.3; Table 1: third order,
  five implicit and three explicit terms per step), rows i = 0..4:
    aI: [0], [1/2,1/2], [5/18,-1/9,1/2], [1/2,0,0,1/2], [1/4,0,3/4,-1/2,1/2]
    aE: [0], [1], [4/9,2/9], [1/4,0,3/4], [1/4,0,3/4,0]
  Its first implicit column is not zero: the stages use the implicit term of
  y_n itself.  The tableau is recalled from the cited paper (not printed in this
  one) and pinned by the order conditions and by Table 1's term counts.
"""
from fractions import Fraction as Fr

import numpy as np

MULTISTEP = ("CNAB2", "SBDF2", "SBDF3")
DIRK = ("ARS443", "BPR353")

# enum values of the C interface
SCHEME_ID = {"CNAB2": 0, "SBDF2": 1, "SBDF3": 2, "ARS443": 3, "BPR353": 4}


def multistep_coeffs(name, n_done):
    """(a, b0, bI, bE) for the step taken after ``n_done`` completed steps."""
    if name == "CNAB2":
        bE = [1.0] if n_done == 0 else [1.5, -0.5]
        return [1.0], 0.5, [0.5], bE
    order = {"SBDF2": 2, "SBDF3": 3}[name]
    k = min(order, n_done + 1)
    if k == 1:
        return [1.0], 1.0, [0.0], [1.0]
    if k == 2:
        return [4 / 3, -1 / 3], 2 / 3, [0.0, 0.0], [4 / 3, -2 / 3]
    return [18 / 11, -9 / 11, 2 / 11], 6 / 11, [0.0, 0.0, 0.0], [18 / 11, -18 / 11, 6 / 11]


def implicit_weights(name):
    """All values of b0 / a_ii the scheme uses (start-up included)."""
    if name == "CNAB2":
        return [0.5]
    if name == "SBDF2":
        return [1.0, 2 / 3]
    if name == "SBDF3":
        return [1.0, 2 / 3, 6 / 11]
    if name in DIRK:
        return [0.5]
    raise ValueError(name)


def ars443_exact():
    h = Fr(1, 2)
    aI = [[0] * 5 for _ in range(5)]
    aE = [[0] * 5 for _ in range(5)]
    aI[1][1] = h
    aI[2][1], aI[2][2] = Fr(1, 6), h
    aI[3][1], aI[3][2], aI[3][3] = Fr(-1, 2), h, h
    aI[4][1], aI[4][2], aI[4][3], aI[4][4] = Fr(3, 2), Fr(-3, 2), h, h
    aE[1][0] = h
    aE[2][0], aE[2][1] = Fr(11, 18), Fr(1, 18)
    aE[3][0], aE[3][1], aE[3][2] = Fr(5, 6), Fr(-5, 6), h
    aE[4][0], aE[4][1], aE[4][2], aE[4][3] = Fr(1, 4), Fr(7, 4), Fr(3, 4), Fr(-7, 4)
    return aI, aE


def bpr353_exact():
    h = Fr(1, 2)
    aI = [[0] * 5 for _ in range(5)]
    aE = [[0] * 5 for _ in range(5)]
    aI[1][0], aI[1][1] = h, h
    aI[2][0], aI[2][1], aI[2][2] = Fr(5, 18), Fr(-1, 9), h
    aI[3][0], aI[3][3] = h, h
    aI[4][0], aI[4][2], aI[4][3], aI[4][4] = Fr(1, 4), Fr(3, 4), -h, h
    aE[1][0] = Fr(1)
    aE[2][0], aE[2][1] = Fr(4, 9), Fr(2, 9)
    aE[3][0], aE[3][2] = Fr(1, 4), Fr(3, 4)
    aE[4][0], aE[4][2] = Fr(1, 4), Fr(3, 4)
    return aI, aE


def dirk_tableau(name):
    exact = {"ARS443": ars443_exact, "BPR353": bpr353_exact}
    if name not in exact:
        raise ValueError(name)
    aI, aE = exact[name]()
    return (np.array([[float(v) for v in r] for r in aI]),
            np.array([[float(v) for v in r] for r in aE]))
