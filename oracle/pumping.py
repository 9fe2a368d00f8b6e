"""Ekman pumping (Section 2 Eqs. pumping_full and uphi; Section 3.2 Eq. approx_pump).

Test infrastructure only (see the package docstring).

Exact form, added to the right-hand side of the vorticity equation:
    F = -Upsilon [ omega - (beta/2) u_phi + beta (d/dphi - 5 s_o/(2h)) u_s ],
    Upsilon = (s_o/E)^(1/2) / h^(3/2),   h^2 = s_o^2 - s^2,
and -Upsilon u_bar on the right-hand side of the zonal-flow equation; both are
linear in the state and singular at s = s_o.  The zonal-flow nonlinear term gains
the self-interaction (E/2) Upsilon u_bar omega_0 of the zonal wind (Eq. uphicoll),
which stays explicit in both formulations.

Collocation (Section 3.1): the exact terms are implicit.  With u_s = (i m/s) psi,
u_phi = -psi' - beta psi (m >= 1) they are, per grid row,
    F = -Upsilon omega - (Upsilon beta/2) psi'
        + Upsilon (-beta^2/2 + beta m^2/s + i 5 m s_o beta/(2 h s)) psi,
and the outer-boundary row, where Upsilon is infinite, is a boundary-condition row
(its value is never used; it is set to 0 here).

Chebyshev integration (Section 3.2): the approximate F_eps of Eq. approx_pump,
    F_eps = Upsilon_eps [ L_I Psi + (s/2) Psi' - (3 s^2/(2 h_eps^2) + m^2
                          + 5 i m s_o/(2 h_eps)) Psi ],
    h_eps^2 = (s_o + eps)^2 - s^2,   Upsilon_eps = s_o^(1/2) E^(-1/2) h_eps^(-3/2),
is explicit: evaluated on the radial grid like a nonlinear term and entering the
integrated streamfunction equation as -F_eps (Eq. psiint).  Readings: L_I Psi is
-omega of the actual geometry (h, not h_eps), as the paper writes the operator
L_I unchanged; the zonal-flow term uses Upsilon_eps as well (the exact Upsilon
is infinite at s_o, where the integration method evaluates the explicit terms).
"""
import numpy as np

from . import chebyshev as ch


def upsilon(ann, E, s, eps=None):
    """Upsilon at radii s: exact (eps None, 0 where s = s_o) or Upsilon_eps."""
    s = np.asarray(s, dtype=float)
    if eps is None:
        h2 = ann.h2(s)
        out = np.zeros_like(s)
        ok = h2 > 0
        out[ok] = np.sqrt(ann.s_o / E) / h2[ok] ** 0.75
        return out
    he2 = (ann.s_o + eps) ** 2 - s ** 2
    return np.sqrt(ann.s_o / E) / he2 ** 0.75


def integration_grid(g, psi_hat, u_hat, eps):
    """F_eps on the radial grid (N_r, M) for m >= 1, and in column m = 0 the two
    zonal-flow terms Upsilon_eps u_bar (1 + (E/2) omega_0), omega_0 = u_bar' +
    u_bar/s, which enter as -D^I (N_u + ...)_hat (Eq. uphi_int)."""
    ops = g.ops
    ann = ops.ann
    n_r, n_c = g.n_r, g.n_c
    cp = np.zeros((n_r, g.M), complex)
    cp[:n_c] = ch.hat_to_plain(psi_hat.T, n_r)
    Psi = g.T @ cp
    dPsi = g.T @ (g.Dn @ cp)
    d2Psi = g.T @ (g.Dn @ (g.Dn @ cp))
    s = g.s[:, None]
    h2 = g.h2[:, None]
    m = g.m[None, :]
    LI = h2 * d2Psi + (h2 / s - 5 * s) * dPsi - (6 + m * m * h2 / s ** 2) * Psi
    he = np.sqrt((ann.s_o + eps) ** 2 - g.s ** 2)[:, None]
    ups = upsilon(ann, ops.E, g.s, eps)[:, None]
    F = ups * (LI + 0.5 * s * dPsi - (1.5 * s ** 2 / he ** 2 + m * m + 2.5j * m * ann.s_o / he) * Psi)
    cu = np.zeros(n_r)
    cu[:n_c] = ch.hat_to_plain(u_hat, n_r)
    ub = g.T @ cu
    w0 = g.T @ (g.Dn @ cu) + ub / g.s
    F[:, 0] = ups[:, 0] * ub * (1.0 + 0.5 * ops.E * w0)
    return F


def integration_matrix(g, m, eps):
    """Psi_hat (N_c) -> truncated Chebyshev coefficients of F_eps (N_c), mode m >= 1:
    the linear map the explicit stage applies (for the onset pencil)."""
    n_c = g.n_c
    out = np.zeros((n_c, n_c), complex)
    for j in range(n_c):
        p = np.zeros((g.M, n_c), complex)
        p[m, j] = 1.0
        F = integration_grid(g, p, np.zeros(n_c), eps)[:, m]
        out[:, j] = ch.analysis(F, g.n_r)[:n_c]
    return out


def collocation_blocks(o, m):
    """Exact pumping rows of the collocation vorticity equation for mode m >= 1 as
    matrices on (omega_hat, psi_hat): (F_omega, F_psi), and the zonal-flow block
    F_u (-Upsilon T).  o: CollocationOperators."""
    ups = upsilon(o.ann, o.E, o.s)
    ups[0] = 0.0                      # s_o: a boundary-condition row
    beta = o.beta
    s = o.s
    h = np.sqrt(np.maximum(o.ann.h2(s), 0.0))
    hs = np.where(h > 0, h * s, 1.0)
    Fw = -ups[:, None] * o.T
    diag = ups * (-0.5 * beta ** 2 + beta * m * m / s) + 1j * ups * 2.5 * m * o.ann.s_o * beta / hs
    Fpsi = -(0.5 * ups * beta)[:, None] * o.T1 + diag[:, None] * o.T
    Fu = -ups[:, None] * o.T
    return Fw, Fpsi, Fu
