"""The n_r = 2049, n_phi = 6144 workload (N_m = 2048, N_c = 1365, E = 1e-8,
Pr = 1, Ra = 20 Ra_c, SBDF3, dt = 1e-10, seeded temperature perturbation of
amplitude 1e-3) against the oracle's banded Appendix A stepper, full state after
every step: the FP64 path and the mixed-precision path (FP32 explicit stage) run
side by side from the same initial state.

Bars (relative L2):
* FP64 theta: 1e-12 per step.  Its row-scaled tau systems have a 2-norm
  condition number ~3e5 at n_r = 1025 and both solves are refined with an FP64
  residual; measured 6e-16.
* FP64 Psi and the whole state (which Psi dominates once the buoyancy has
  driven it): 5e-11.  The streamfunction systems at this size have an effective
  condition number ~2e5 (row-scaled 2-norm condition up to ~4e8 at n_r = 1025
  on the highest modes), so two FP64-refined solves agree to ~2e5 eps = 4.4e-11;
  measured 2.8e-12 after the first step.
* FP64 u_bar: max(20, c_u) times the state bar, c_u the cancellation factor of
  its forcing (tests/parity_util.py).
* mixed precision: 1e-6 of the whole state after every step (the mixed-precision bar of the time step).
"""
import numpy as np
import pytest

from oracle.banded import BandedIntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import assert_state_close, critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu

N_STEPS = 8   # oracle steps (~7 s each on 16 host cores)


def _whole(y):
    return np.concatenate([np.asarray(x).ravel() for x in y])


def test_large_workload_fp64_and_mixed_against_banded_oracle():
    from paper_1902_07092_gb300.binding import Solver, pizza_set_option
    wl = inputs.WORKLOADS["large_n2049_p6144"]
    n_r, n_phi, E, dt = wl["n_r"], wl["n_phi"], wl["E"], wl["dt"]
    Ra = wl["ra_factor"] * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt)
    mix = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt)
    pizza_set_option(mix.ctx, "precision", 1)
    ora = BandedIntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt)
    th = inputs.theta_init(n_r, n_phi, wl["amp"], wl["seed"], cfg=wl["cfg"])
    z, zu = inputs.zero_state(n_r, n_phi)
    for s in (gpu, mix):
        s.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for k in range(N_STEPS):
        gpu.step(1)
        mix.step(1)
        ora.step()
        g, mx = gpu.get_state(), mix.get_state()
        ref = ora.y
        e = {name: rel_l2(a, b) for name, a, b in zip(("psi", "theta", "u"), g, ref)}
        e_state = rel_l2(_whole(g), _whole(ref))
        e_mixed = rel_l2(_whole(mx), _whole(ref))
        print("n_r = 2049 step %d: FP64 state %.2e psi %.2e theta %.2e u %.2e | mixed %.2e" % (
            k + 1, e_state, e["psi"], e["theta"], e["u"], e_mixed))
        assert_state_close(g, ref, 5e-11, oracle=ora)
        assert e["theta"] <= 1e-12
        assert e_mixed <= 1e-6
    for s in (gpu, mix):
        s.close()
