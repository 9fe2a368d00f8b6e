"""Failure detection without a GPU fault: a NaN planted in the initial state (a
valid input that the kernels only propagate) is reported as PIZZA_ENONFINITE by
pizza_synchronize when option "check_finite" is on, by pizza_diagnostics always,
and in a batch only for the context that carries it; pizza_set_state clears it."""
import numpy as np
import pytest

from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh

pytestmark = pytest.mark.gpu

ENONFINITE = -4


def _solver(radial="integration", check=True):
    from paper_1902_07092_gb300.binding import Solver, pizza_set_option
    s = Solver(33, 96, 1e-3, 2.0 * critical_rayleigh(1e-3), 1.0, 0.35, "CNAB2", 1e-4, radial=radial)
    if check:
        pizza_set_option(s.ctx, "check_finite", 1)
    return s


def _states(n_r, n_phi, n_c=None, bad=False):
    th = inputs.theta_init(n_r, n_phi, 1e-3, 1, cfg=1, n_c=n_c)
    if bad:
        th[3, 2] = np.nan
    z, zu = inputs.zero_state(n_r, n_phi, n_c=n_c)
    return th, z, zu


@pytest.mark.parametrize("radial", ["integration", "collocation"])
def test_nan_state_is_reported_and_cleared(radial):
    from paper_1902_07092_gb300.binding import PizzaError, pizza_synchronize
    s = _solver(radial)
    nc = 33 if radial == "collocation" else None
    s.set_state(*_states(33, 96, nc, bad=True))
    s.step(2)
    with pytest.raises(PizzaError) as ei:
        pizza_synchronize(s.ctx)
    assert ei.value.code == ENONFINITE
    with pytest.raises(PizzaError) as ei:
        s.diagnostics()
    assert ei.value.code == ENONFINITE
    s.set_state(*_states(33, 96, nc))
    s.step(2)
    pizza_synchronize(s.ctx)
    assert np.all(np.isfinite(s.get_state()[1]))
    s.close()


def test_without_the_scan_synchronize_stays_silent_and_diagnostics_reports():
    from paper_1902_07092_gb300.binding import PizzaError, pizza_synchronize
    s = _solver(check=False)
    s.set_state(*_states(33, 96, bad=True))
    s.step(1)
    pizza_synchronize(s.ctx)
    with pytest.raises(PizzaError) as ei:
        s.diagnostics()
    assert ei.value.code == ENONFINITE
    s.close()


def test_nan_in_one_context_of_a_batch_is_reported_for_that_context_only():
    from paper_1902_07092_gb300.binding import Batch, PizzaError, pizza_synchronize
    good, bad = _solver(), _solver()
    good.set_state(*_states(33, 96))
    bad.set_state(*_states(33, 96, bad=True))
    b = Batch([good, bad])
    b.step(3)
    pizza_synchronize(good.ctx)
    with pytest.raises(PizzaError) as ei:
        pizza_synchronize(bad.ctx)
    assert ei.value.code == ENONFINITE
    b.close()
    good.close()
    bad.close()


ECFL = -5


@pytest.mark.parametrize("radial,precision", [("integration", 0), ("integration", 1), ("collocation", 0)])
def test_courant_guard_reports_the_rates_of_eq_cfl(radial, precision):
    """Option cfl_alpha (Eq. cfl): one CNAB2 step evaluates the explicit terms of
    the initial state once; the fused maxima of the azimuthal kernel must be the
    Courant rates pizza_diagnostics computes for that state, and the guard trips
    exactly when dt exceeds alpha / max(rate)."""
    import re

    from paper_1902_07092_gb300.binding import PizzaError, pizza_last_error, pizza_set_option, pizza_synchronize
    n_r, n_phi = 33, 96
    nc = 33 if radial == "collocation" else None
    th = inputs.theta_init(n_r, n_phi, 1.0, 4, cfg=7, m_min=0, n_c=nc)
    ps = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=8, n_c=nc)
    ps[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1.0, 6, cfg=9, m_min=0, n_c=nc)[0].real.copy()
    if radial == "collocation":
        # wall conditions of psi for a valid collocation state: psi = (1 - x^2)^2 p(x)
        from oracle import chebyshev as ch
        from oracle.geometry import gauss_lobatto
        x = gauss_lobatto(n_r)
        grid = ch.synthesis(ps.T, n_r) * ((1 - x * x) ** 2)[:, None]
        ps = ch.analysis(grid, n_r).T.copy()
    s = _solver(radial, check=False)
    if precision:
        pizza_set_option(s.ctx, "precision", precision)
    s.set_state(th, ps, u)
    d = s.diagnostics()
    rate = max(d["cfl_s"], d["cfl_phi"])
    assert rate > 0
    dt = 1e-4
    tol = 1e-12 if precision == 0 else 1e-5
    for alpha, trips in ((0.5 * dt * rate, True), (2.0 * dt * rate, False)):
        s.set_state(th, ps, u)
        pizza_set_option(s.ctx, "cfl_alpha", alpha)
        s.step(1)
        if trips:
            with pytest.raises(PizzaError) as ei:
                pizza_synchronize(s.ctx)
            assert ei.value.code == ECFL
            r = [float(v) for v in re.search(r"rates ([-+0-9.e]+), ([-+0-9.e]+)\)", pizza_last_error(s.ctx)).groups()]
            assert abs(r[0] - d["cfl_s"]) <= tol * d["cfl_s"], (r, d)
            assert abs(r[1] - d["cfl_phi"]) <= tol * d["cfl_phi"], (r, d)
        else:
            pizza_synchronize(s.ctx)      # no error; the maxima were cleared by the previous call
    pizza_set_option(s.ctx, "cfl_alpha", 0.0)
    s.step(1)
    pizza_synchronize(s.ctx)
    s.close()
