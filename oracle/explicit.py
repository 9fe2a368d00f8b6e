"""Explicit terms of one stage, Chebyshev-integration formulation
(Section 2 Eqs. vort, uphi, temp; Section 3.2; dealiasing as stated below Eq. temp_int).

Test infrastructure only (see the package docstring).

From the state (Psi_hat, theta_hat, u_hat; paper coefficients, N_c per mode):
 1. radial grid, per m (regularised streamfunction of Section 3.2):
      v_m     = i m Psi_m                      (d Psi/d phi;  u_s = (h^2/s) v)
      u_phi_m = -h^2 dPsi_m/ds + 3 s Psi_m      (m >= 1),  u_phi_0 = u_bar
      omega_m = -L_I Psi_m                      (m >= 1),  omega_0 = (1/s) d(s u_bar)/ds
      theta_m
    derivatives by the dense Chebyshev differentiation matrix;
 2. physical grid by Eq. fft (N_phi points), the products
      v omega, u_phi omega, v theta, u_phi theta,
    and back by Eq. ifft keeping m <= N_m;
 3. flux-form divergences per m on the radial grid, with u_s = (h^2/s) v and
    beta u_s = -v (beta = -s/h^2):
      N_omega = (1/s) d/ds(h^2 [v omega]_m) + (i m/s)[u_phi omega]_m
      N_theta = (1/s) d/ds(h^2 [v theta]_m) + (i m/s)[u_phi theta]_m - [v theta]_m
      N_u     = [u_s omega]_0 = (h^2/s)[v omega]_0
    the radial derivative being that of the N_r-point Chebyshev interpolant
    (Eq. icheb, differentiate, Eq. cheb);
 4. Chebyshev coefficients by Eq. icheb, truncated to n < N_c;
 5. integrated right-hand sides (rows below q are zero):
      Psi:   C^I [ (Ra/Pr)(i m/s_o) theta_hat + N_omega_hat ]           (Eq. psi_int)
      theta: -D^I N_theta_hat - (alpha/ln eta) i m G^I Psi_hat          (Eq. temp_int)
      u_bar: -D^I N_u_hat                                                (Eq. uphi_int)
Ekman pumping (``g.pump_eps`` not None): the approximate F_eps of Eq. approx_pump
on the radial grid (``pumping.integration_grid``) joins step 3 as
N_omega - F_eps, and Upsilon_eps u_bar joins N_u.
Implicit buoyancy (``g.buoy_implicit``, Section 4): the buoyancy term leaves e_psi
and joins the implicit operator (``stepper.IntegrationStepper``).
"""
import numpy as np

from . import chebyshev as ch
from . import fourier as fo
from .geometry import gauss_lobatto
from .pumping import integration_grid


class Grid:
    def __init__(self, ops, n_phi):
        self.ops = ops
        self.n_r, self.n_c, self.n_phi = ops.n_r, ops.n_c, n_phi
        if n_phi % 3:
            raise ValueError("N_phi must be a multiple of 3")
        self.n_m = n_phi // 3
        self.M = self.n_m + 1
        ann = ops.ann
        self.x = gauss_lobatto(self.n_r)
        self.s = ann.s_of_x(self.x)
        self.h2 = ann.h2(self.s)
        self.m = np.arange(self.M)
        self.T = ch.tmat(self.n_r, self.n_r)
        self.Dn = ch.diff_matrix(self.n_r) / ann.a      # d/ds on plain coefficients
        self.pump_eps = None                             # Ekman pumping off
        self.buoy_implicit = False                       # buoyancy in the explicit terms


def radial_fields(g, psi_hat, theta_hat, u_hat):
    """Step 1: (v, u_phi, omega, theta) on the radial grid, arrays (N_r, M)."""
    n_r, n_c = g.n_r, g.n_c
    cp = np.zeros((n_r, g.M), complex)
    cp[:n_c] = ch.hat_to_plain(psi_hat.T, n_r)
    ct = np.zeros((n_r, g.M), complex)
    ct[:n_c] = ch.hat_to_plain(theta_hat.T, n_r)
    cu = np.zeros(n_r)
    cu[:n_c] = ch.hat_to_plain(u_hat, n_r)
    T, Dn = g.T, g.Dn
    Psi = T @ cp
    dPsi = T @ (Dn @ cp)
    d2Psi = T @ (Dn @ (Dn @ cp))
    s = g.s[:, None]
    h2 = g.h2[:, None]
    m = g.m[None, :]
    v = 1j * m * Psi
    uphi = -h2 * dPsi + 3 * s * Psi
    omega = -(h2 * d2Psi + (h2 / s - 5 * s) * dPsi - (6 + m * m * h2 / s ** 2) * Psi)
    ub = T @ cu
    dub = T @ (Dn @ cu)
    uphi[:, 0] = ub
    omega[:, 0] = dub + ub / g.s
    v[:, 0] = 0.0
    theta = T @ ct
    return v, uphi, omega, theta


def products(g, v, uphi, omega, theta):
    """Step 2: Fourier coefficients of v omega, u_phi omega, v theta, u_phi theta."""
    P = g.n_phi
    vg, ug, wg, tg = (fo.to_grid(f, P) for f in (v, uphi, omega, theta))
    return tuple(fo.to_spec(p, g.n_m) for p in (vg * wg, ug * wg, vg * tg, ug * tg))


def radial_derivative(g, f):
    """d/ds of the N_r-point interpolant of grid values f (N_r, ...)."""
    c = ch.hat_to_plain(ch.analysis(f, g.n_r), g.n_r)
    return g.T @ (g.Dn @ c)


def nonlinear_grid(g, vw, uw, vt, ut):
    """Step 3: N_omega, N_theta (N_r, M) and N_u (N_r,) on the radial grid."""
    s = g.s[:, None]
    h2 = g.h2[:, None]
    m = g.m[None, :]
    Nw = (radial_derivative(g, h2 * vw) + 1j * m * uw) / s
    Nt = (radial_derivative(g, h2 * vt) + 1j * m * ut) / s - vt
    Nu = (g.h2 / g.s) * vw[:, 0]
    return Nw, Nt, Nu


def nonlinear_hat(g, vw, uw, vt, ut):
    """Step 4: truncated Chebyshev coefficients (M, N_c) of N_omega, N_theta
    and (N_c,) of N_u."""
    Nw, Nt, Nu = nonlinear_grid(g, vw, uw, vt, ut)
    nc = g.n_c
    return (ch.analysis(Nw, g.n_r)[:nc].T, ch.analysis(Nt, g.n_r)[:nc].T,
            ch.analysis(Nu, g.n_r)[:nc].real)


def explicit_terms(g, psi_hat, theta_hat, u_hat, return_parts=False):
    """Step 5: integrated explicit right-hand sides (e_psi, e_theta, e_u)."""
    ops = g.ops
    v, uphi, omega, theta = radial_fields(g, psi_hat, theta_hat, u_hat)
    vw, uw, vt, ut = products(g, v, uphi, omega, theta)
    Nw_g, Nt_g, Nu_g = nonlinear_grid(g, vw, uw, vt, ut)
    if g.pump_eps is not None:
        F = integration_grid(g, psi_hat, u_hat, g.pump_eps)
        Nw_g = Nw_g - F
        Nu_g = Nu_g + F[:, 0].real
    nc = g.n_c
    Nw = ch.analysis(Nw_g, g.n_r)[:nc].T
    Nt = ch.analysis(Nt_g, g.n_r)[:nc].T
    Nu = ch.analysis(Nu_g, g.n_r)[:nc].real
    m = g.m[:, None]
    buoy = (ops.Ra / ops.Pr) * (1j * m / ops.ann.s_o) * theta_hat
    if g.buoy_implicit:
        buoy = np.zeros_like(buoy)
    e_psi = (ops.C @ (buoy + Nw).T).T
    e_psi[0] = 0.0
    e_theta = -(ops.D @ Nt.T).T - ops.tc_coef * 1j * m * (ops.G @ psi_hat.T).T
    e_u = -(ops.D @ Nu)
    if return_parts:
        return e_psi, e_theta, e_u, dict(v=v, uphi=uphi, omega=omega, theta=theta,
                                         vw=vw, uw=uw, vt=vt, ut=ut,
                                         Nw_grid=Nw_g, Nt_grid=Nt_g, Nu_grid=Nu_g,
                                         Nw=Nw, Nt=Nt, Nu=Nu)
    return e_psi, e_theta, e_u
