"""Mixed precision (option "precision" = 1): the explicit stage in FP32, the state,
history, linear couplings, boundary rows and solves in FP64.  Errors are measured
against the FP64 oracle (n_r <= 257) and, at n_r = 2049 where the oracle cannot run
50 steps, against the FP64 GPU path, which the sampled large-workload parity test
pins to the oracle.

Bars: the time-stepped state stays within 1e-6 (relative L2) of FP64 per step and
after 50 steps.  The explicit right-hand sides themselves carry the FP32 rounding
of the transforms, amplified by the radial differentiation of the flux form (up to
n_r, as for FP64) and summed over O(log n) butterfly levels: bound
8 n_r log2(n_phi) u_32, u_32 = 2^-24."""
import math

import numpy as np
import pytest

from oracle.explicit import explicit_terms
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def mixed_solver(n_r, n_phi, E, Ra, scheme, dt):
    from paper_1902_07092_gb300.binding import Solver, pizza_set_option
    s = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt)
    pizza_set_option(s.ctx, "precision", 1)
    return s


def state_rel(a, b):
    ga = np.concatenate([np.asarray(x).ravel() for x in a])
    gb = np.concatenate([np.asarray(x).ravel() for x in b])
    return rel_l2(ga, gb)


@pytest.mark.parametrize("n_r,n_phi", [(65, 192), (257, 768)])
def test_mixed_explicit_terms_error(n_r, n_phi):
    Ra = 2.0 * critical_rayleigh(1e-3)
    gpu = mixed_solver(n_r, n_phi, 1e-3, Ra, "CNAB2", 1e-4)
    ora = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4)
    th = inputs.theta_init(n_r, n_phi, 1.0, 3, cfg=7, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1.0, 4, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    tol = 8 * n_r * math.log2(n_phi) * U32
    print("mixed explicit terms n_r=%d: psi %.2e theta %.2e u %.2e (tol %.1e)" % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi", [(129, 384), (257, 768), (513, 1536)])
def test_mixed_lean_radial_kernels_match_oracle(n_r, n_phi):
    """Option radial_lean = 1 in mixed precision: the FP32 three-array radial
    kernels (half-length DCT-I with the odd outputs' prefix sums in FP64, FP32
    transforms and field arithmetic at each radius, FP32 grid arrays, the analysed
    coefficients widened to FP64 for the banded applies) give the explicit terms
    the streamfunction and temperature explicit terms within the mixed bar,
    8 n_r log2(n_phi) u_32, of the FP64 oracle, and two steps within 1e-6 of it.
    The zonal-flow term is forced by the m = 0 mean [v omega]_0, which the FP32
    azimuthal kernel forms with the cancellation of its terms (to ~1e-4 of them)
    whatever the radial layout: there the lean layout must stay within the batched
    layout's own error plus the bar."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    Ra = 2.0 * critical_rayleigh(1e-3)
    ora = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4)
    th = inputs.theta_init(n_r, n_phi, 1.0, 3, cfg=7, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1.0, 4, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=9, m_min=0)[0].real.copy()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    errs = {}
    for lean in (0, 1):
        gpu = mixed_solver(n_r, n_phi, 1e-3, Ra, "CNAB2", 1e-4)
        pizza_set_option(gpu.ctx, "radial_lean", lean)
        gpu.set_state(th, psi, u)
        ep, et, eu = gpu.explicit_terms()
        errs[lean] = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
        gpu.close()
    tol = 8 * n_r * math.log2(n_phi) * U32
    print("mixed explicit terms n_r=%d, lean: psi %.2e theta %.2e u %.2e; batched: u %.2e (tol %.1e)"
          % ((n_r,) + errs[1] + (errs[0][2], tol)))
    assert max(errs[1][:2]) <= tol
    assert errs[1][2] <= errs[0][2] + tol
    # two steps from a small state
    E, dt = 1e-5, 1e-8
    Ra = 5.0 * critical_rayleigh(E)
    gpu = mixed_solver(n_r, 24, E, Ra, "SBDF3", dt)
    pizza_set_option(gpu.ctx, "radial_lean", 1)
    ora = IntegrationStepper(n_r, 24, E, Ra, 1.0, 0.35, "SBDF3", dt)
    th = inputs.theta_init(n_r, 24, 1e-3, 81, cfg=1, m_min=0)
    psi = inputs.theta_init(n_r, 24, 1e-5, 82, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, 24, 1e-3, 83, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = state_rel(gpu.get_state(), ora.y)
        print("mixed lean n_r=%d step %d: state rel err %.2e" % (n_r, k + 1, e))
        assert e <= 1e-6
    gpu.close()


def test_mixed_steps_sparse_workload():
    """n_r = 257, n_phi = 768, E = 1e-5, Ra = 10 Ra_c, ARS443, dt = 1e-7, seeded
    perturbation 1e-3: five steps against the FP64 oracle."""
    n_r, n_phi, E, dt = 257, 768, 1e-5, 1e-7
    Ra = 10.0 * critical_rayleigh(E)
    gpu = mixed_solver(n_r, n_phi, E, Ra, "ARS443", dt)
    ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", dt)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 2, cfg=2)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for k in range(5):
        gpu.step(1)
        ora.step()
        e = state_rel(gpu.get_state(), ora.y)
        print("mixed sparse step %d: state rel err %.2e" % (k + 1, e))
        assert e <= 1e-6
    gpu.close()


def test_mixed_large_workload_50_steps():
    """n_r = 2049, n_phi = 6144, E = 1e-8, SBDF3, dt = 1e-10, perturbation 1e-3
    (seed 3): 50 steps of the mixed path against the FP64 path, state compared
    after every step."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E, dt = 2049, 6144, 1e-8, 1e-10
    Ra = 2.0e11     # 3.2 Ra_c at E = 1e-8 (Ra_c = 6.16e10)
    ref = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt)
    mix = mixed_solver(n_r, n_phi, E, Ra, "SBDF3", dt)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 3, cfg=3)
    z, zu = inputs.zero_state(n_r, n_phi)
    ref.set_state(th, z, zu)
    mix.set_state(th, z, zu)
    worst = 0.0
    for k in range(50):
        ref.step(1)
        mix.step(1)
        if k % 7 == 0 or k == 49:
            e = state_rel(mix.get_state(), ref.get_state())
            worst = max(worst, e)
            print("mixed large step %d: state rel err vs FP64 %.2e" % (k + 1, e))
            assert e <= 1e-6
    ref.close()
    mix.close()


def test_mixed_precision_option_limits():
    from paper_1902_07092_gb300.binding import PizzaError, Solver, pizza_set_option
    s = Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4, radial="collocation")
    with pytest.raises(PizzaError) as ei:
        pizza_set_option(s.ctx, "precision", 1)
    assert ei.value.code == -8
    s.close()
    s = Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    with pytest.raises(PizzaError) as ei:
        pizza_set_option(s.ctx, "precision", 2)
    assert ei.value.code == -8
    pizza_set_option(s.ctx, "precision", 1)
    with pytest.raises(PizzaError):
        pizza_set_option(s.ctx, "radial", 0)
    s.close()
