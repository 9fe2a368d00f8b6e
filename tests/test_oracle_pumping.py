"""Pins of the oracle's Ekman pumping (Eqs. pumping_full, uphi, uphicoll and
approx_pump) against the values the paper prints and against each other."""
import json
import os

import numpy as np

from oracle import chebyshev as ch
from oracle.collocation import CollocationOperators, leading_eigenvalue_collocation
from oracle.explicit import Grid, radial_fields
from oracle.onset import leading_eigenvalue
from oracle.operators import IntegrationOperators
from oracle.pumping import collocation_blocks, integration_grid, upsilon
from tests.parity_util import GOLDEN

E3, PR, RA, ETA, M12 = 3e-6, 0.025, 1e7, 0.35, 12


def test_collocation_onset_with_pumping_matches_table3():
    """Table 3, eigensolver row with Ekman pumping (E = 3e-6, Ra = 1e7, Pr = 0.025,
    m = 12): tau = 2.122883e2, omega_d = -9.436506e3.  The exact pumping is implicit
    in the collocation operators."""
    t3 = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))["eigensolver_pumping"]
    lam = leading_eigenvalue_collocation(E3, PR, RA, ETA, M12, 97, guess=212.0 - 9436.0j, pumping=True)
    assert abs(lam.real - t3["tau"]) < 2e-3
    assert abs(lam.imag - t3["omega_d"]) < 5e-3


def test_collocation_marginal_mode_with_pumping_matches_the_critical_eigenmode():
    """Section 6.1: with Ekman pumping the m = 12 mode at E = 3e-6, Pr = 0.025 is
    marginal at Ra_c = 9.55263e6 and drifts at omega_d = -9.42690e3."""
    lam = leading_eigenvalue_collocation(E3, PR, 9.55263e6, ETA, M12, 97, guess=-9427.0j, pumping=True)
    assert abs(lam.real) < 1e-2          # the printed Ra_c has 6 digits: d tau/d Ra ~ 6e-5
    assert abs(lam.imag - (-9426.90)) < 1e-2


def test_approximate_pumping_tends_to_the_exact_form_pointwise():
    """F_eps of Eq. approx_pump (written in the regularised streamfunction Psi) and
    the exact F of Eq. pumping_full (written in omega, psi = h^2 Psi and the
    velocities, as the collocation rows hold it) are two derivations of the same
    term: at eps -> 0 they agree at every interior point, for m >= 1 and for the
    zonal-flow term Upsilon u_bar."""
    n_r, n_phi, m = 65, 12, 3
    nc = (2 * (n_r - 1)) // 3
    ops = IntegrationOperators(n_r, nc, ETA, E3, PR, RA)
    g = Grid(ops, n_phi)
    rng = np.random.default_rng(7)
    psi_hat = np.zeros((g.M, nc), complex)
    psi_hat[m, :12] = (rng.standard_normal(12) + 1j * rng.standard_normal(12)) / (1.0 + np.arange(12)) ** 2
    u_hat = np.zeros(nc)
    u_hat[:10] = rng.standard_normal(10) / (1.0 + np.arange(10)) ** 2
    eps = 1e-10
    Fe = integration_grid(g, psi_hat, u_hat, eps)
    # exact form on the same fields through the collocation operators
    o = CollocationOperators(n_r, ETA, E3, PR, RA, pumping=True)
    v, uphi, omega, theta = radial_fields(g, psi_hat, np.zeros_like(psi_hat), u_hat)
    cp = np.zeros(n_r, complex)
    cp[:nc] = ch.hat_to_plain(psi_hat[m], n_r)
    psi_grid = g.h2 * (g.T @ cp)
    Fw, Fpsi, Fu = collocation_blocks(o, m)
    F_exact = Fw @ ch.analysis(omega[:, m], n_r) + Fpsi @ ch.analysis(psi_grid, n_r)
    inner = g.h2 > 0.2
    scale = np.max(np.abs(F_exact[inner]))
    assert np.max(np.abs(Fe[inner, m] - F_exact[inner])) < 1e-7 * scale
    # zonal flow: -Upsilon u_bar (implicit, collocation) against Upsilon_eps u_bar
    # (1 + (E/2) omega_0) (explicit, integration): the self-interaction part is
    # the (E/2) omega_0 factor
    ub = uphi[:, 0].real
    w0 = omega[:, 0].real
    lhs = Fe[inner, 0].real
    rhs = -(Fu @ ch.analysis(ub, n_r))[inner] * (1.0 + 0.5 * E3 * w0[inner])
    assert np.max(np.abs(lhs - rhs)) < 1e-7 * np.max(np.abs(rhs))
    # Upsilon itself: (s_o/E)^(1/2) (s_o^2 - s^2)^(-3/4)
    s = 1.0 / (1.0 - ETA) - 0.3
    assert abs(upsilon(ops.ann, E3, np.array([s]))[0]
               - (1.0 / (1.0 - ETA) / E3) ** 0.5 * ((1.0 / (1.0 - ETA)) ** 2 - s * s) ** -0.75) < 1e-9


def test_integration_onset_with_approximate_pumping_converges_to_the_exact_one():
    """With F_eps explicit in the integrated equations (Eq. psiint), the m = 12
    eigenvalue at Ra = 1e7 lies above the exact-pumping one by O(eps): tripling eps
    triples the gap (Section 6.1 reports the same trend for its own runs,
    Table 3: 2.148113e2 at eps = 3e-3, 2.123799e2 at 1e-4, 2.122983e2 at 1e-5,
    eigensolver 2.122883e2)."""
    exact = json.load(open(os.path.join(GOLDEN, "growth_rates_table3.json")))["eigensolver_pumping"]["tau"]
    gaps = []
    for eps in (3e-3, 1e-3):
        lam = leading_eigenvalue(E3, PR, RA, ETA, M12, 96, guess=214.0 - 9436.7j, n_r=145, pumping_eps=eps)
        gaps.append(lam.real - exact)
        assert abs(lam.imag - (-9436.7)) < 0.5
    assert gaps[0] > gaps[1] > 0
    assert 2.5 < gaps[0] / gaps[1] < 3.5
