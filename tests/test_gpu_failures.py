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
