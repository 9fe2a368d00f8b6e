"""Pins of the oracle's diagnostics against exact integrals and closed forms."""
import numpy as np
import numpy.polynomial.chebyshev as npc

from oracle import chebyshev as ch
from oracle.diagnostics import cc_weights, diagnostics, local_spacing
from oracle.geometry import gauss_lobatto
from oracle.stepper import IntegrationStepper


def test_clenshaw_curtis_weights_integrate_polynomials_exactly():
    n_r = 17
    x = gauss_lobatto(n_r)
    w = cc_weights(n_r)
    rng = np.random.default_rng(0)
    c = rng.standard_normal(n_r)
    exact = npc.chebval(1.0, npc.chebint(c)) - npc.chebval(-1.0, npc.chebint(c))
    assert np.isclose(w @ npc.chebval(x, c), exact, rtol=1e-13, atol=1e-13)
    assert np.isclose(w.sum(), 2.0)


def test_zonal_energy_of_a_polynomial_flow():
    """u_bar = (s - s_i)(s_o - s): E_Z = pi int u^2 s ds in closed form; E_K = E_Z."""
    st = IntegrationStepper(33, 12, 1e-3, 0.0, 1.0, 0.35, "CNAB2", 1e-4)
    ann = st.ops.ann
    s = ann.s_of_x(gauss_lobatto(33))
    u = (s - ann.s_i) * (ann.s_o - s)
    u_hat = ch.analysis(u, 33)[:st.n_c]
    z = np.zeros((st.g.M, st.n_c), complex)
    d = diagnostics(st.g, z, z, u_hat)
    P = np.polynomial.Polynomial
    p = P([-ann.s_i, 1]) * P([ann.s_o, -1])
    q = (p * p * P([0, 1])).integ()
    ez = np.pi * (q(ann.s_o) - q(ann.s_i))
    assert np.isclose(d["E_Z"], ez, rtol=1e-13)
    assert np.isclose(d["E_K"], ez, rtol=1e-13)
    Re = np.sqrt(2 * ez / (np.pi * (ann.s_o ** 2 - ann.s_i ** 2)))
    assert np.isclose(d["Re"], Re, rtol=1e-13)
    # CFL: |u_phi|/(s dphi) maximum over the grid
    assert np.isclose(d["cfl_phi"], np.max(np.abs(u) / (s * 2 * np.pi / 12)), rtol=1e-12)
    assert d["cfl_s"] == 0.0


def test_nusselt_of_a_polynomial_temperature():
    """theta_0 = (s - s_i)(s_o - s): d theta/ds at s_o = -(s_o - s_i) = -1."""
    st = IntegrationStepper(33, 12, 1e-3, 0.0, 1.0, 0.35, "CNAB2", 1e-4)
    ann = st.ops.ann
    s = ann.s_of_x(gauss_lobatto(33))
    th = np.zeros((st.g.M, st.n_c), complex)
    th[0] = ch.analysis((s - ann.s_i) * (ann.s_o - s), 33)[:st.n_c]
    d = diagnostics(st.g, np.zeros_like(th), th, np.zeros(st.n_c))
    assert np.isclose(d["Nu_minus_1"], -1.0 / ann.dTc_ds(ann.s_o), rtol=1e-12)
    assert d["E_K"] == 0.0


def test_local_spacing():
    s = np.array([3.0, 2.5, 1.5, 1.0])
    assert np.allclose(local_spacing(s), [0.5, 0.75, 0.75, 0.5])
