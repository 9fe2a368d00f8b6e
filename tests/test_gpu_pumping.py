"""Ekman pumping on the GPU (option "pumping_eps"): parity with the oracle's
pumping (exact and implicit in the collocation formulation, approximate F_eps of
Eq. approx_pump and explicit in the integration formulation), and the Section 6.1
validation with pumping: runs started from the leading m = 12 eigenmode grow and
drift at the eigenvalue (Table 3).

Tolerances as for the runs without pumping (tests/test_gpu_parity.py,
tests/test_gpu_collocation.py): the pumping terms are linear in the state and
evaluated from the same grid values, so they add no new amplification of
rounding errors."""
import json
import os

import numpy as np
import pytest

from oracle.collocation import CollocationStepper, leading_mode_collocation
from oracle.explicit import explicit_terms
from oracle.onset import leading_mode
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import GOLDEN, assert_state_close, critical_rayleigh, rel_l2
from tests.test_gpu_collocation import EPS, coll_state, compare_state, rounding_growth, set_both
from tests.test_gpu_parity import random_state

pytestmark = pytest.mark.gpu

EPS_PUMP = 3e-3


def pair(n_r, n_phi, E, ra_factor, scheme, dt, radial):
    from paper_1902_07092_gb300.binding import Solver
    Ra = ra_factor * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, radial=radial, pumping_eps=EPS_PUMP)
    if radial == "collocation":
        ora = CollocationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, pumping=True)
    else:
        ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, pumping_eps=EPS_PUMP)
    return gpu, ora


@pytest.mark.parametrize("n_r,n_phi", [(65, 192), (257, 768)])
def test_pumping_explicit_terms_match_oracle(n_r, n_phi):
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4, "integration")
    psi, th, u = random_state(n_r, n_phi, 1.0, 3, psi_amp=1.0, u_amp=1.0)
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    tol = max(1e-12, 4 * n_r * n_r * EPS)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    print("pumping explicit terms n_r=%d: psi %.2e theta %.2e u %.2e (tol %.1e)" % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_pumping_steps_match_oracle_integration(scheme, amp):
    n_r, n_phi = 33, 96
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4, "integration")
    th = inputs.theta_init(n_r, n_phi, amp, 1, cfg=1)
    psi = inputs.theta_init(n_r, n_phi, amp, 2, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, amp, 3, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for _ in range(4):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    gpu.close()


def test_pumping_steps_match_oracle_n257():
    n_r, n_phi = 257, 768
    gpu, ora = pair(n_r, n_phi, 1e-5, 10.0, "ARS443", 1e-7, "integration")
    th = inputs.theta_init(n_r, n_phi, 1e-3, 2, cfg=2)
    z, zu = inputs.zero_state(n_r, n_phi)
    u = inputs.theta_init(n_r, n_phi, 1e-3, 4, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, z, u)
    ora.set_state(z, th, u)
    for _ in range(2):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 2e-12, oracle=ora)
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (129, 384)])
def test_pumping_collocation_explicit_rows_match_oracle(n_r, n_phi):
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4, "collocation")
    psi, th, u = coll_state(n_r, n_phi, 1.0, 3, psi_amp=1.0, u_amp=1.0)
    set_both(gpu, ora, psi, th, u)
    ew, et, eu = gpu.explicit_terms()
    rw, _, rt, ru = ora.explicit(ora.y)
    tol = max(1e-12, 4 * n_r * n_r * EPS)
    errs = (rel_l2(ew, rw), rel_l2(et, rt), rel_l2(eu, ru))
    print("pumping collocation rows n_r=%d: omega %.2e theta %.2e u %.2e" % ((n_r,) + errs))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF2", "SBDF3", "ARS443"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_pumping_collocation_steps_match_oracle(scheme, amp):
    n_r, n_phi = 33, 96
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4, "collocation")
    psi, th, u = coll_state(n_r, n_phi, amp, 1, psi_amp=amp, u_amp=amp)
    # the step-k bar follows the oracle's own growth of a rounding-size difference
    # (up to ~10x per step for the strongly nonlinear amp = 1 states)
    Ra = 2.0 * critical_rayleigh(1e-3)
    d = rounding_growth(lambda: CollocationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, scheme, 1e-4, pumping=True),
                        psi, th, u, 4)
    set_both(gpu, ora, psi, th, u)
    for k in range(4):
        gpu.step(1)
        ora.step()
        tol = max(1e-12, 2.0 ** 7 * d[k])
        e = compare_state(gpu, ora, tol, tol_w=max(tol, n_r ** 4 * EPS / 4))
        print("pumping collocation %s amp %g step %d: %s" % (scheme, amp, k + 1, {a: "%.2e" % b for a, b in e.items()}))
    gpu.close()


def test_pumping_mixed_precision_explicit_terms():
    """Mixed precision with pumping: the FP32 explicit stage within the bound of
    tests/test_gpu_mixed.py, 8 n_r log2(n_phi) 2^-24."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    n_r, n_phi = 65, 192
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4, "integration")
    pizza_set_option(gpu.ctx, "precision", 1)
    psi, th, u = random_state(n_r, n_phi, 1.0, 3, psi_amp=1.0, u_amp=1.0)
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    tol = 8 * n_r * np.log2(n_phi) * 2.0 ** -24
    print("pumping mixed explicit terms: psi %.2e theta %.2e u %.2e (tol %.1e)" % (errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


def test_pumping_option_limits():
    from paper_1902_07092_gb300.binding import PizzaError, Solver, pizza_set_option
    s = Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    for bad in (-1.0, float("nan"), 2.0):
        with pytest.raises(PizzaError):
            pizza_set_option(s.ctx, "pumping_eps", bad)
    pizza_set_option(s.ctx, "pumping_eps", 1e-3)
    with pytest.raises(PizzaError) as ei:
        s.tape_begin(5)
    assert ei.value.code == -8
    pizza_set_option(s.ctx, "pumping_eps", 0.0)
    s.tape_begin(5)
    s.close()


# --------------------------------------------------------- Section 6.1 --------
def growth(s, M_MODE, T, K1, K2, dt):
    s.step(K1)
    z1 = np.vdot(T[M_MODE], s.get_state()[1][M_MODE]) / np.vdot(T[M_MODE], T[M_MODE])
    s.step(K2 - K1)
    th2 = s.get_state()[1][M_MODE]
    z2 = np.vdot(T[M_MODE], th2) / np.vdot(T[M_MODE], T[M_MODE])
    return np.log(z2 / z1) / ((K2 - K1) * dt), np.linalg.norm(th2 - z2 * T[M_MODE]) / np.linalg.norm(th2)


def test_pumping_growth_rate_collocation_matches_table3():
    """Collocation with the exact pumping, (N_r, N_m) = (129, 128), ARS443,
    dt = 1e-7, started from the oracle's leading m = 12 eigenmode (E = 3e-6,
    Ra = 1e7, Pr = 0.025): growth rate and drift within 2e-3 and 5e-3 of the
    eigensolver's Table 3 values with pumping (2.122883e2, -9.436506e3)."""
    from paper_1902_07092_gb300.binding import Solver
    t3 = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))
    ref = t3["eigensolver_pumping"]
    n_r, n_phi, m, dt = 129, 384, 12, 1e-7
    lam, w, p, th = leading_mode_collocation(t3["E"], t3["Pr"], t3["Ra"], t3["eta"], m, n_r,
                                             guess=complex(ref["tau"], ref["omega_d"]), pumping=True)
    s = Solver(n_r, n_phi, t3["E"], t3["Ra"], t3["Pr"], t3["eta"], "ARS443", dt, radial="collocation",
               pumping_eps=EPS_PUMP)
    P = np.zeros((s.M, n_r), complex)
    T = np.zeros_like(P)
    a = 1e-8 / np.max(np.abs(th))
    P[m], T[m] = a * p, a * th
    s.set_state(T, P, np.zeros(n_r))
    est, resid = growth(s, m, T, 100, 2100, dt)
    print("collocation with pumping: %.7e %.7e | eigenvalue %.7e %.7e" % (est.real, est.imag, lam.real, lam.imag))
    assert resid < 1e-6
    assert abs(est - lam) < 1e-8 * abs(lam)
    assert abs(est.real - ref["tau"]) < 2e-3
    assert abs(est.imag - ref["omega_d"]) < 5e-3
    s.close()


def test_pumping_growth_rate_integration_matches_its_eigenvalue():
    """Integration with F_eps (eps = 3e-3), (N_r, N_c, N_m) = (257, 170, 128),
    ARS443, dt = 1e-7: the run grows and drifts at the eigenvalue of the oracle's
    onset pencil with the same F_eps."""
    from paper_1902_07092_gb300.binding import Solver
    t3 = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))
    n_r, n_phi, m, dt = 257, 384, 12, 1e-7
    nc = (2 * (n_r - 1)) // 3
    lam, p, th = leading_mode(t3["E"], t3["Pr"], t3["Ra"], t3["eta"], m, nc, n_r=n_r, guess=214.4 - 9436.8j,
                              pumping_eps=EPS_PUMP)
    s = Solver(n_r, n_phi, t3["E"], t3["Ra"], t3["Pr"], t3["eta"], "ARS443", dt, pumping_eps=EPS_PUMP)
    P = np.zeros((s.M, nc), complex)
    T = np.zeros_like(P)
    a = 1e-8 / np.max(np.abs(th))
    P[m], T[m] = a * p, a * th
    s.set_state(T, P, np.zeros(nc))
    est, resid = growth(s, m, T, 100, 2100, dt)
    print("integration with F_eps: %.7e %.7e | eigenvalue %.7e %.7e" % (est.real, est.imag, lam.real, lam.imag))
    assert resid < 1e-6
    assert abs(est - lam) < 1e-8 * abs(lam)
    s.close()
