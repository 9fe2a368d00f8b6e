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


def test_energy_enstrophy_and_cfl_of_nonaxisymmetric_polynomial_flow():
    """m >= 1 parts of the diagnostics against a brute-force physical-space
    evaluation.  Psi_m = s^2 q_m(s) (m = 1, 2, 3) and u_bar = s p(s) make every
    field a polynomial in s:  psi = h^2 Psi (Section 3.2), u_s = (1/s) d psi/d phi,
    u_phi = u_bar - d psi/ds - beta psi (Eq. vel_def), omega = (1/s) d(s u_bar)/ds
    - L_beta psi with L_beta psi = Delta psi + (1/s) d(beta s psi)/ds (Eq. psi).
    Here they are built by polynomial arithmetic, taken to the physical grid by
    the literal sum of Eq. fft, and integrated with Gauss-Legendre nodes in s and
    the uniform rule in phi (exact for these trigonometric polynomials); the CFL
    rates are maxima over the Gauss-Lobatto x uniform grid of the closed forms.
    A wrong weight of the m >= 1 terms, of the radial velocity or of the
    vorticity changes one of E_K, Z or cfl_s."""
    from oracle import fourier as fo
    P = np.polynomial.Polynomial
    n_r, n_phi = 33, 24
    st = IntegrationStepper(n_r, n_phi, 1e-3, 0.0, 1.0, 0.35, "CNAB2", 1e-4)
    ann, g = st.ops.ann, st.g
    so2 = ann.s_o ** 2
    sP = P([0.0, 1.0])
    h2 = P([so2, 0.0, -1.0])
    rng = np.random.default_rng(5)
    q = {m: P(rng.standard_normal(4)) for m in (1, 2, 3)}      # real parts of Psi_m / s^2
    qi = {m: P(rng.standard_normal(4)) for m in (1, 2, 3)}     # imaginary parts
    p = P(rng.standard_normal(3))
    ubar = sP * p
    s_gl = ann.s_of_x(gauss_lobatto(n_r))
    psi_hat = np.zeros((g.M, st.n_c), complex)
    for m in (1, 2, 3):
        Psi = lambda s, m=m: s ** 2 * (q[m](s) + 1j * qi[m](s))
        psi_hat[m] = ch.analysis(Psi(s_gl), n_r)[:st.n_c]
    u_hat = ch.analysis(ubar(s_gl), n_r)[:st.n_c]
    d = diagnostics(g, psi_hat, np.zeros_like(psi_hat), u_hat)

    def fields(s):
        """(u_s, u_phi, omega) spectra [len(s), M] from the closed forms."""
        us = np.zeros((len(s), g.M), complex)
        up = np.zeros_like(us)
        om = np.zeros_like(us)
        up[:, 0] = ubar(s)
        om[:, 0] = (ubar + sP * ubar.deriv())(s) / s
        for m in (1, 2, 3):
            for part, qq in ((1.0, q[m]), (1j, qi[m])):
                Psi = sP ** 2 * qq
                psi = h2 * Psi
                us[:, m] += part * 1j * m * psi(s) / s
                up[:, m] += part * (-psi.deriv()(s) + (sP * Psi)(s))     # -beta psi = s Psi
                lap = psi.deriv(2)(s) + psi.deriv()(s) / s - m * m * psi(s) / s ** 2
                bsp = -(sP ** 2) * Psi                                   # beta s psi = -s^2 Psi
                om[:, m] += part * -(lap + bsp.deriv()(s) / s)
        return us, up, om

    xg, wg = np.polynomial.legendre.leggauss(48)
    s = ann.s_of_x(xg)
    ws = wg * ann.a * s                      # weights of int f s ds
    n_q = 64
    us, up, om = (fo.to_grid_direct(f, n_q) for f in fields(s))
    mean = lambda f2: 2 * np.pi * np.sum(ws[:, None] * f2) / n_q
    E_K = 0.5 * mean(us ** 2 + up ** 2)
    Z = mean(om ** 2)
    assert np.isclose(d["E_K"], E_K, rtol=1e-12)
    assert np.isclose(d["enstrophy"], Z, rtol=1e-12)
    assert np.isclose(d["Re"], np.sqrt(2 * E_K / (np.pi * (ann.s_o ** 2 - ann.s_i ** 2))), rtol=1e-12)
    usk, upk, _ = (fo.to_grid_direct(f, n_phi) for f in fields(s_gl))
    ds = np.empty(n_r)
    ds[1:-1] = 0.5 * (s_gl[:-2] - s_gl[2:])
    ds[0], ds[-1] = s_gl[0] - s_gl[1], s_gl[-2] - s_gl[-1]
    assert np.isclose(d["cfl_s"], np.max(np.abs(usk) / ds[:, None]), rtol=1e-12)
    assert np.isclose(d["cfl_phi"], np.max(np.abs(upk) / (s_gl[:, None] * 2 * np.pi / n_phi)), rtol=1e-12)
