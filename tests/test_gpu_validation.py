"""Section 6.1 validation on the GPU: a run of the compiled stepper started from
the onset solver's leading m = 12 eigenmode (E = 3e-6, Ra = 1e7, Pr = 0.025,
radius ratio 0.35) at (N_r, N_c, N_m) = (257, 170, 128) grows and drifts at the
eigenvalue of the same discretisation (614.99910 - 9536.95338i), within the time
error of each scheme at dt = 1e-7.  The DIRK scheme (ARS443) hits it to 1e-8 and
reproduces the eigensolver's growth rate and drift frequency of Table 3
(tests/golden/growth_rates_table3.json) to the six digits the paper underlines
for its own DIRK runs (BPR353: 6.14999e2, -9.53695e3).  The multistep schemes
carry a time error of a few 1e-3 in tau at this dt, as Table 3 shows for the
paper's own multistep runs (SBDF3 6.150048e2, CNAB2 6.150091e2 against
6.149994e2), so they are held to 1e-6 of |lambda| only."""
import json
import os

import numpy as np
import pytest

from oracle.onset import leading_mode
from tests.parity_util import GOLDEN

pytestmark = pytest.mark.gpu

N_R, N_PHI, M_MODE, DT = 257, 384, 12, 1e-7
SCHEME_TOL = {"SBDF3": 1e-6, "ARS443": 1e-8, "BPR353": 1e-8, "CNAB2": 1e-6}   # relative error of lambda


@pytest.fixture(scope="module")
def mode():
    t3 = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))
    nc = (2 * (N_R - 1)) // 3
    lam, p, th = leading_mode(t3["E"], t3["Pr"], t3["Ra"], t3["eta"], M_MODE, nc, n_r=N_R,
                              guess=complex(t3["eigensolver"]["tau"], t3["eigensolver"]["omega_d"]))
    return t3, nc, lam, p, th


@pytest.mark.parametrize("scheme", ["SBDF3", "CNAB2", "ARS443", "BPR353"])
def test_growth_rate_and_drift_of_the_m12_mode(mode, scheme):
    from paper_1902_07092_gb300.binding import Solver
    t3, nc, lam, p, th = mode
    s = Solver(N_R, N_PHI, t3["E"], t3["Ra"], t3["Pr"], t3["eta"], scheme, DT)
    assert s.n_c == nc
    P = np.zeros((s.M, nc), complex)
    T = np.zeros_like(P)
    a = 1e-8 / np.max(np.abs(th))
    P[M_MODE], T[M_MODE] = a * p, a * th
    s.set_state(T, P, np.zeros(nc))
    K1, K2 = 100, 2100                      # 2e-4 viscous times, a third of a drift period
    s.step(K1)
    z1 = np.vdot(T[M_MODE], s.get_state()[1][M_MODE]) / np.vdot(T[M_MODE], T[M_MODE])
    s.step(K2 - K1)
    th2 = s.get_state()[1][M_MODE]
    z2 = np.vdot(T[M_MODE], th2) / np.vdot(T[M_MODE], T[M_MODE])
    est = np.log(z2 / z1) / ((K2 - K1) * DT)
    print("%s: tau %.7e omega_d %.7e | eigenvalue %.7e %.7e | Table 3 %.7e %.7e" % (
        scheme, est.real, est.imag, lam.real, lam.imag, t3["eigensolver"]["tau"], t3["eigensolver"]["omega_d"]))
    assert np.linalg.norm(th2 - z2 * T[M_MODE]) < 1e-6 * np.linalg.norm(th2)
    assert abs(est - lam) < SCHEME_TOL[scheme] * abs(lam)
    if scheme in ("ARS443", "BPR353"):
        lsb = t3["eigensolver"]
        assert abs(est.real - lsb["tau"]) < 1e-3
        assert abs(est.imag - lsb["omega_d"]) < 5e-3
    s.close()
