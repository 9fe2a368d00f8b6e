"""Pins of the oracle's discrete adjoint: the adjoint of the explicit stage against
exact directional derivatives (the explicit terms are quadratic in the state, so a
central difference is exact up to rounding), and the gradient of the time-averaged
Nusselt number against central finite differences of whole CNAB2 runs."""
import numpy as np
import pytest

from oracle.adjoint import adjoint_cnab2, explicit_adjoint, nusselt_minus_one
from oracle.explicit import explicit_terms
from oracle.stepper import IntegrationStepper


def _rand_state(rng, M, nc, amp):
    c = lambda: amp * (rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))) / (1 + np.arange(nc)) ** 2
    psi, th = c(), c()
    psi[0] = 0.0
    th[0] = th[0].real
    u = amp * rng.standard_normal(nc) / (1 + np.arange(nc)) ** 2
    return psi, th, u


def _dot(a, b):
    return sum(float(np.real(np.vdot(x, y))) for x, y in zip(a, b))


@pytest.mark.parametrize("n_r,n_phi", [(17, 24), (33, 48)])
def test_explicit_adjoint_passes_the_dot_product_test(n_r, n_phi):
    st = IntegrationStepper(n_r, n_phi, 1e-3, 3e5, 0.7, 0.35, "CNAB2", 1e-4)
    g = st.g
    rng = np.random.default_rng(11)
    y = _rand_state(rng, g.M, g.n_c, 1.0)
    d = _rand_state(rng, g.M, g.n_c, 1.0)
    ebar = _rand_state(rng, g.M, g.n_c, 1.0)
    plus = explicit_terms(g, *(a + b for a, b in zip(y, d)))
    minus = explicit_terms(g, *(a - b for a, b in zip(y, d)))
    jvp = tuple(0.5 * (p - q) for p, q in zip(plus, minus))
    adj, _ = explicit_adjoint(g, *y, ebar)
    lhs = _dot(ebar, jvp)
    rhs = _dot(adj, d)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def test_explicit_ra_derivative_is_exact():
    st = IntegrationStepper(17, 24, 1e-3, 3e5, 1.0, 0.35, "CNAB2", 1e-4)
    g = st.g
    rng = np.random.default_rng(3)
    y = _rand_state(rng, g.M, g.n_c, 1.0)
    _, dE = explicit_adjoint(g, *y, tuple(np.zeros_like(x) for x in y))
    e1 = explicit_terms(g, *y)[0]
    g.ops.Ra += 1000.0
    e2 = explicit_terms(g, *y)[0]
    g.ops.Ra -= 1000.0
    assert np.abs((e2 - e1) / 1000.0 - dE).max() <= 1e-9 * np.abs(dE).max()


def _objective(n_r, n_phi, Ra, y0, K, dt=2e-4):
    st = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", dt)
    st.set_state(*y0)
    J = 0.0
    for _ in range(K):
        st.step()
        J += nusselt_minus_one(st.g, st.y[1]) / K
    return J


def test_cnab2_adjoint_gradient_matches_finite_differences():
    """J = (1/K) sum_{n=1..K} (Nu_n - 1), K = 6 CNAB2 steps at (17, 24), E = 1e-3,
    strongly nonlinear state: dJ/dtheta_0 along a seeded direction and dJ/dRa
    against central differences (h = 1e-6 relative)."""
    n_r, n_phi, Ra, K = 17, 24, 2e5, 6
    st = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 2e-4)
    rng = np.random.default_rng(5)
    y0 = _rand_state(rng, st.g.M, st.g.n_c, 0.5)
    J, lam, dRa = adjoint_cnab2(st, y0, K)
    assert abs(J - _objective(n_r, n_phi, Ra, y0, K)) <= 1e-13 * max(abs(J), 1e-300)
    dth = _rand_state(rng, st.g.M, st.g.n_c, 1.0)[1]
    h = 1e-6
    yp = (y0[0], y0[1] + h * dth, y0[2])
    ym = (y0[0], y0[1] - h * dth, y0[2])
    fd = (_objective(n_r, n_phi, Ra, yp, K) - _objective(n_r, n_phi, Ra, ym, K)) / (2 * h)
    ad = float(np.real(np.vdot(lam[1], dth)))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    hR = 1e-6 * Ra
    fdR = (_objective(n_r, n_phi, Ra + hR, y0, K) - _objective(n_r, n_phi, Ra - hR, y0, K)) / (2 * hR)
    assert abs(fdR - dRa) <= 1e-5 * abs(dRa), (fdR, dRa)
