"""Pins of the onset solver's root finders (Section 6.1, Eq. lin) against the
critical values the paper prints, and of the committed Ra_c table against an
independent discretisation.

* Section 6.1 (caption of the eigenfunction figure): with Ekman pumping, E = 3e-6,
  Pr = 0.025, radius ratio 0.35, the first unstable mode is m = 12 at
  Ra_c = 9.55263e6 with omega_d = -9.42690e3.  The collocation operators carry the
  exact pumping term implicitly, so the root finders run on that pencil here.
* The Ra_c table of the workloads (Pr = 1, radius ratio 0.35, no pumping) is
  written by ``oracle.critical_table`` on the integration/tau pencil; the
  collocation pencil, built from grid differentiation matrices with no shared
  operator code, must find the same Ra_c, m_c and omega_d.
* Arnoldi iteration (``leading_eigenvalue_arnoldi``) and the QZ path agree.

Table 2 (Gillet et al. 2007's set-up, radius ratio 4/11, E = 1e-6, Pr = 0.025) is
not used as a pin: with the printed Eq. lin and the fixed-temperature T_c the
marginal m = 13 mode lies near Ra = 3.35e7 with omega_d ~ -1.95e4, not at the
tabulated 1.3851e7 / -1.3028e4; the paper does not print the heating profile and
scales that table was computed with.
"""
import json
import os

import numpy as np

from oracle.collocation import leading_eigenvalue_collocation
from oracle.onset import (critical_rayleigh, leading_eigenvalue, leading_eigenvalue_arnoldi,
                          leading_of_pencil, marginal_rayleigh, pencil)
from tests.parity_util import GOLDEN

E3, PR3, ETA = 3e-6, 0.025, 0.35


def _coll(E, Pr, n_r, pumping):
    return lambda m, ra: leading_eigenvalue_collocation(E, Pr, ra, ETA, m, n_r, guess=None, pumping=pumping)


def test_critical_rayleigh_with_pumping_reproduces_section_6_1():
    """Minimum over m = 11, 12, 13 of the marginal Ra (Brent's method on the
    leading growth rate): m_c = 12, Ra_c = 9.55263e6 and omega_d = -9.42690e3 to
    the printed digits."""
    ra, m, om = critical_rayleigh(E3, PR3, ETA, (11, 12, 13), 97, 9.0e6, 1.1e7,
                                  eigenvalue=_coll(E3, PR3, 97, True))
    assert m == 12
    assert round(ra, -1) == 9.55263e6, ra
    assert round(om, 2) == -9426.90, om


def test_marginal_rayleigh_brackets_from_below_and_above():
    """The bracketing root finder reaches the same marginal Ra from a start below
    and above it (factor-2 steps, then Brent's method)."""
    lead = _coll(E3, PR3, 97, True)
    f = lambda ra, g: lead(12, ra)
    a, la = marginal_rayleigh(E3, PR3, ETA, 12, 97, 6.0e6, eigenvalue=f)
    b, lb = marginal_rayleigh(E3, PR3, ETA, 12, 97, 2.0e7, eigenvalue=f)
    assert abs(a - 9.55263e6) < 5.0 and abs(b - 9.55263e6) < 5.0
    assert abs(la.real) < 1e-6 and abs(lb.real) < 1e-6
    assert abs(la.imag - (-9426.90)) < 5e-3


def test_critical_table_entry_from_the_collocation_pencil():
    """E = 1e-3 (the tiny workload's Ra_c): m = 4, 5, 6 scanned on the collocation
    pencil without pumping give the table's m_c = 5, Ra_c and omega_d."""
    t = json.load(open(os.path.join(GOLDEN, "critical_rayleigh.json")))["0.001"]
    ra, m, om = critical_rayleigh(1e-3, 1.0, ETA, (4, 5, 6), 49, 4.0e4, 8.0e4,
                                  eigenvalue=_coll(1e-3, 1.0, 49, False))
    assert m == t["m_c"] == 5
    assert abs(ra - t["Ra_c"]) < 1e-6 * t["Ra_c"]
    assert abs(om - t["omega_d"]) < 1e-5 * abs(t["omega_d"])


def test_critical_table_entry_at_the_sparse_workload_ekman_number():
    """E = 1e-5 (the n_r = 257 workloads' Ra_c): the table's critical mode m = 17
    is marginal on the collocation pencil at the tabulated Ra_c, drifting at the
    tabulated omega_d."""
    t = json.load(open(os.path.join(GOLDEN, "critical_rayleigh.json")))["1e-05"]
    lam = _coll(1e-5, 1.0, 129, False)(17, t["Ra_c"])
    assert abs(lam.real) < 1e-4 * abs(lam.imag) * 1e-3
    assert abs(lam.imag - t["omega_d"]) < 1e-6 * abs(t["omega_d"])


def test_table_generator_root_finder_reproduces_its_entry():
    """The default path of ``marginal_rayleigh`` (integration/tau pencil, Arnoldi
    continuation of the drift-frequency branch) gives the committed E = 1e-3 entry."""
    t = json.load(open(os.path.join(GOLDEN, "critical_rayleigh.json")))["0.001"]
    ra, lam = marginal_rayleigh(1e-3, 1.0, ETA, 5, t["n_c"], 5.0e4)
    assert abs(ra - t["Ra_c"]) < 1e-8 * t["Ra_c"]
    assert abs(lam.imag - t["omega_d"]) < 1e-6 * abs(t["omega_d"])


def test_arnoldi_agrees_with_qz():
    """Table 3's case without pumping (E = 3e-6, Ra = 1e7, Pr = 0.025, m = 12):
    the Arnoldi eigenvalue nearest a rough guess equals the QZ-selected leading
    eigenvalue after shift-and-invert refinement, and it is the finite eigenvalue
    of largest real part of the pencil."""
    n_c = 96
    q = leading_eigenvalue(E3, PR3, 1e7, ETA, 12, n_c)
    a = leading_eigenvalue_arnoldi(E3, PR3, 1e7, ETA, 12, n_c, 600.0 - 9500.0j)
    assert abs(a - q) < 1e-9 * abs(q)
    import scipy.linalg as sl
    L, M = pencil(E3, PR3, 1e7, ETA, 12, n_c)
    w = sl.eig(L, M, right=False)
    w = w[np.isfinite(w) & (np.abs(w) < 1e8)]
    assert abs(w[np.argmax(w.real)] - q) < 1e-4 * abs(q)     # QZ on the unscaled pencil: an estimate
    assert abs(leading_of_pencil(L, M, q) - q) < 1e-9 * abs(q)
