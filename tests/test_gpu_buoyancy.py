"""Implicit buoyancy on the GPU (option "buoy_implicit", Section 4): the
temperature of each stage is solved first and its buoyancy joins the
streamfunction (collocation: vorticity) system.  Parity with the oracle's
steppers with buoy_implicit=True, themselves pinned against dense solves of the
coupled systems and, for the integration formulation, by the order of an
eigenmode run (tests/test_oracle_physics.py, tests/test_oracle_collocation.py).

Tolerances as for explicit buoyancy (tests/test_gpu_parity.py): 1e-12 at n_r = 33,
2e-12 at 257.  At n_r = 1025 (N_c = 682, the temperature solved by FP32 solves
with FP64-residual corrections) the streamfunction block's conditioning grows
with N_c (measured 5e-13 against the oracle): 5e-12."""
import json
import os

import numpy as np
import pytest

from oracle.onset import leading_mode
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import GOLDEN, assert_state_close, critical_rayleigh

pytestmark = pytest.mark.gpu


def pair(n_r, n_phi, E, Ra, scheme, dt):
    from paper_1902_07092_gb300.binding import Solver
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, buoy_implicit=True)
    ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, buoy_implicit=True)
    return gpu, ora


def nonzero_state(n_r, n_phi, amp, seed):
    th = inputs.theta_init(n_r, n_phi, amp, seed, cfg=1)
    psi = inputs.theta_init(n_r, n_phi, amp * 1e-2, seed + 1, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, amp, seed + 2, cfg=9, m_min=0)[0].real.copy()
    return psi, th, u


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_implicit_buoyancy_steps_match_oracle_tiny(scheme, amp):
    n_r, n_phi = 33, 96
    gpu, ora = pair(n_r, n_phi, 1e-3, 2.0 * critical_rayleigh(1e-3), scheme, 1e-4)
    psi, th, u = nonzero_state(n_r, n_phi, amp, 1)
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for _ in range(4):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    gpu.close()


def test_implicit_buoyancy_steps_match_oracle_n257():
    n_r, n_phi = 257, 768
    gpu, ora = pair(n_r, n_phi, 1e-5, 10.0 * critical_rayleigh(1e-5), "ARS443", 1e-7)
    psi, th, u = nonzero_state(n_r, n_phi, 1e-3, 2)
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for _ in range(2):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 2e-12, oracle=ora)
    gpu.close()


def test_implicit_buoyancy_steps_match_oracle_n1025():
    n_r, n_phi = 1025, 24
    gpu, ora = pair(n_r, n_phi, 1e-6, 5.0 * critical_rayleigh(1e-6), "SBDF3", 1e-9)
    psi, th, u = nonzero_state(n_r, n_phi, 1e-3, 3)
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, 5e-12, oracle=ora)
        print("implicit buoyancy n_r=1025 step %d: %s" % (k + 1, {a: "%.2e" % b for a, b in e.items() if a != "_norms"}))
    gpu.close()


def test_implicit_buoyancy_eigenmode_run_grows_at_the_eigenvalue():
    """The Section 6.1 validation run (E = 3e-6, Ra = 1e7, Pr = 0.025, m = 12,
    (257, 170, 128), ARS443, dt = 1e-7) with the buoyancy implicit."""
    from paper_1902_07092_gb300.binding import Solver
    t3 = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))
    n_r, n_phi, m, dt = 257, 384, 12, 1e-7
    nc = (2 * (n_r - 1)) // 3
    lam, p, th = leading_mode(t3["E"], t3["Pr"], t3["Ra"], t3["eta"], m, nc, n_r=n_r,
                              guess=complex(t3["eigensolver"]["tau"], t3["eigensolver"]["omega_d"]))
    s = Solver(n_r, n_phi, t3["E"], t3["Ra"], t3["Pr"], t3["eta"], "ARS443", dt, buoy_implicit=True)
    P = np.zeros((s.M, nc), complex)
    T = np.zeros_like(P)
    a = 1e-8 / np.max(np.abs(th))
    P[m], T[m] = a * p, a * th
    s.set_state(T, P, np.zeros(nc))
    s.step(100)
    z1 = np.vdot(T[m], s.get_state()[1][m]) / np.vdot(T[m], T[m])
    s.step(2000)
    z2 = np.vdot(T[m], s.get_state()[1][m]) / np.vdot(T[m], T[m])
    est = np.log(z2 / z1) / (2000 * dt)
    print("implicit buoyancy eigenmode run: %.7e %.7e | eigenvalue %.7e %.7e" % (est.real, est.imag, lam.real, lam.imag))
    assert abs(est - lam) < 1e-7 * abs(lam)
    s.close()


def test_implicit_buoyancy_option_limits():
    from paper_1902_07092_gb300.binding import PizzaError, Solver, pizza_set_option
    s = Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4, buoy_implicit=True)
    with pytest.raises(PizzaError):
        pizza_set_option(s.ctx, "buoy_implicit", 2)
    with pytest.raises(PizzaError) as ei:
        s.tape_begin(5)
    assert ei.value.code == -8
    s.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_implicit_buoyancy_collocation_steps_match_oracle(scheme, amp):
    """Collocation (Section 3.1) with the buoyancy implicit: the solve runs the
    temperature rows first, then the vorticity-streamfunction rows."""
    from oracle.collocation import CollocationStepper
    from paper_1902_07092_gb300.binding import Solver
    from tests.test_gpu_collocation import EPS, coll_state, compare_state, rounding_growth, set_both
    n_r, n_phi = 33, 96
    Ra = 2.0 * critical_rayleigh(1e-3)
    gpu = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, scheme, 1e-4, radial="collocation", buoy_implicit=True)
    ora = CollocationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, scheme, 1e-4, buoy_implicit=True)
    psi, th, u = coll_state(n_r, n_phi, amp, 1, psi_amp=amp, u_amp=amp)
    # the step-k bar follows the oracle's own growth of a rounding-size difference
    # (up to ~10x per step for the strongly nonlinear amp = 1 states)
    d = rounding_growth(lambda: CollocationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, scheme, 1e-4,
                                                   buoy_implicit=True), psi, th, u, 4)
    set_both(gpu, ora, psi, th, u)
    for k in range(4):
        gpu.step(1)
        ora.step()
        tol = max(1e-12, 2.0 ** 7 * d[k])
        compare_state(gpu, ora, tol, tol_w=max(tol, n_r ** 4 * EPS / 4))
    gpu.close()


def test_implicit_buoyancy_collocation_steps_match_oracle_n129():
    from oracle.collocation import CollocationStepper
    from paper_1902_07092_gb300.binding import Solver
    from tests.test_gpu_collocation import EPS, coll_state, compare_state, set_both
    n_r, n_phi = 129, 384
    Ra = 10.0 * critical_rayleigh(1e-5)
    gpu = Solver(n_r, n_phi, 1e-5, Ra, 1.0, 0.35, "ARS443", 1e-7, radial="collocation", buoy_implicit=True)
    ora = CollocationStepper(n_r, n_phi, 1e-5, Ra, 1.0, 0.35, "ARS443", 1e-7, buoy_implicit=True)
    psi, th, u = coll_state(n_r, n_phi, 1e-3, 2, psi_amp=1e-5, u_amp=1e-5)
    set_both(gpu, ora, psi, th, u)
    for _ in range(2):
        gpu.step(1)
        ora.step()
        compare_state(gpu, ora, 2e-12, tol_w=max(2e-12, n_r ** 4 * EPS / 4))
    gpu.close()
