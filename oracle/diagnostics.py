"""Diagnostics of a state (Section 6.2 and the definitions around Eq. cfl).

Test infrastructure only (see the package docstring).

  E_K = (1/2) <u_s^2 + u_phi^2> = E_Z + 2 pi sum_{m>=1} int (|u_s,m|^2 + |u_phi,m|^2) s ds
  E_Z = (1/2) <u_bar^2> = pi int u_bar^2 s ds
  Z   = <omega^2> = 2 pi [ int omega_0^2 s ds + 2 sum_{m>=1} int |omega_m|^2 s ds ]
  Re  = [2 E_K / (pi (s_o^2 - s_i^2))]^(1/2),   Ro = Re E
  Nu - 1 = (d theta_0/ds)(s_o) / (dT_c/ds)(s_o)   (reading: the paper defines no
           Nusselt number; this is the heat flux through the outer wall relative to
           conduction)
  CFL rates: max |u_s|/ds_k and max |u_phi|/(s_k dphi) over the physical grid,
           dphi = 2 pi/N_phi, ds_k the local Gauss-Lobatto spacing (half the
           distance between the two neighbours; one-sided at the walls)
with <f> = int int f s ds dphi (Section 5).  The radial integrals use
Clenshaw-Curtis quadrature on the N_r Gauss-Lobatto points: the weights integrate
the N_r-point Chebyshev interpolant exactly.
"""
import numpy as np

from . import chebyshev as ch
from . import fourier as fo
from .explicit import radial_fields


def cc_weights(n_r):
    """Weights w_k with sum_k w_k f(x_k) = int_{-1}^{1} of the interpolant of f:
    int T_n dx = 2/(1-n^2) (n even), 0 (n odd), applied to Eq. icheb."""
    n = np.arange(n_r)
    tint = np.where(n % 2 == 0, 2.0 / (1.0 - n.astype(float) ** 2 + (n % 2)), 0.0)
    # plain coefficients of the interpolant: c = hat_to_plain(analysis(f))
    # => int = sum_n tint_n c_n = sum_k w_k f_k
    A = ch.hat_to_plain(ch.analysis(np.eye(n_r), n_r), n_r)   # (n, k)
    return tint @ A


def local_spacing(s):
    d = np.empty_like(s)
    d[1:-1] = 0.5 * (s[:-2] - s[2:])
    d[0] = s[0] - s[1]
    d[-1] = s[-2] - s[-1]
    return d


def diagnostics(g, psi_hat, theta_hat, u_hat):
    ops = g.ops
    ann = ops.ann
    v, uphi, omega, theta = radial_fields(g, psi_hat, theta_hat, u_hat)
    s = g.s
    us = (g.h2 / s)[:, None] * v
    w = cc_weights(g.n_r) * ann.a * s                       # weights of int f s ds
    wm = np.full(g.M, 2.0)
    wm[0] = 1.0
    E_Z = np.pi * np.sum(w * np.abs(uphi[:, 0]) ** 2)
    E_K = E_Z + 2 * np.pi * np.sum(w[:, None] * (np.abs(us[:, 1:]) ** 2 + np.abs(uphi[:, 1:]) ** 2))
    Z = 2 * np.pi * np.sum(w[:, None] * wm[None, :] * np.abs(omega) ** 2)
    Re = np.sqrt(2 * E_K / (np.pi * (ann.s_o ** 2 - ann.s_i ** 2)))
    c0 = np.zeros(g.n_r)
    c0[:g.n_c] = ch.hat_to_plain(theta_hat[0].real, g.n_r)
    dth_o = np.sum(np.arange(g.n_r) ** 2 * c0) / ann.a          # T_n'(1) = n^2
    nu_m1 = dth_o / ann.dTc_ds(ann.s_o)
    usg = fo.to_grid(us, g.n_phi)
    upg = fo.to_grid(uphi, g.n_phi)
    ds = local_spacing(s)
    dphi = 2 * np.pi / g.n_phi
    cfl_s = np.max(np.abs(usg) / ds[:, None])
    cfl_phi = np.max(np.abs(upg) / (s[:, None] * dphi))
    return dict(E_K=E_K, E_Z=E_Z, enstrophy=Z, Nu=1.0 + nu_m1, Nu_minus_1=nu_m1, Re=Re, Ro=Re * ops.E,
                cfl_s=cfl_s, cfl_phi=cfl_phi)
