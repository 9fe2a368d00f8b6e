"""Galerkin-basis variant of the Chebyshev-integration solve (Appendix B, with the
integrated systems of Section 3.2).

Test infrastructure only (see the package docstring).

Instead of carrying the boundary conditions as tau rows, the unknowns are
expanded in bases that satisfy them:
  streamfunction  Psi = sum_{n < N_c-4} x_n phi_n,  phi_n = sum_{i=0..4} gamma_i^n T_{n+i}
                  with the closed-form gamma of Appendix B (Psi = 0 at both walls,
                  Psi''' = 0 at s_o and Psi' = 0 at s_i: the four tau rows);
  temperature and zonal flow  f = sum_{n < N_c-2} x_n (T_{n+2} - T_n)  (zero at
                  both walls).
With S the stencil matrix (plain coefficients c = S x) and the tau rows dropped
(P_4, P_2: rows k >= 4, resp. k >= 2 of the integrated equations), each implicit
system becomes square and banded,
    P_4 (A^I_m - g dt B^I_m) S_Psi x = P_4 r      (8 diagonals below, 12 above),
    P_2 (D^I - g dt F^I_m/Pr) S_D x = P_2 r,  P_2 (D^I - g dt E^I) S_D x = P_2 r
                                                   (4 below, 6 above),
solved here by banded LU with partial pivoting (LAPACK gbsv through
scipy.linalg.solve_banded) after scaling each row to unit maximum (which leaves
the solution unchanged).  The columns of S span exactly the coefficient vectors
that meet the boundary conditions, so the solution is that of the tau system;
only the linear algebra differs.  The time schemes, explicit terms, mass and
implicit operators are those of ``stepper.IntegrationStepper``.
"""
import numpy as np
import scipy.linalg as sl

from . import chebyshev as ch
from .stepper import IntegrationStepper


def gamma_psi(n):
    """gamma_0..gamma_4 of phi_n (Appendix B), gamma_0 = 1."""
    n = float(n)
    den = 2 * n ** 4 + 20 * n ** 3 + 78 * n ** 2 + 140 * n + 95
    q = n * n + 4 * n + 5
    return np.array([
        1.0,
        8 * (n + 1) * q / den,
        -2 * (n + 2) * (2 * n ** 4 + 16 * n ** 3 + 58 * n ** 2 + 104 * n + 75) / ((n + 3) * den),
        -8 * (n + 1) * q / den,
        (n + 1) * (2 * n ** 4 + 12 * n ** 3 + 30 * n ** 2 + 36 * n + 15) / ((n + 3) * den),
    ])


def stencil_psi(n_c):
    """Plain-coefficient stencil S_Psi (n_c x (n_c - 4)): column n is phi_n."""
    S = np.zeros((n_c, n_c - 4))
    for n in range(n_c - 4):
        S[n:n + 5, n] = gamma_psi(n)
    return S


def stencil_dir(n_c):
    """Plain-coefficient stencil S_D (n_c x (n_c - 2)): column n is T_{n+2} - T_n."""
    S = np.zeros((n_c, n_c - 2))
    for n in range(n_c - 2):
        S[n, n] = -1.0
        S[n + 2, n] = 1.0
    return S


def band_extent(G):
    """(lower, upper) half bandwidths of the nonzero pattern of G."""
    i, j = np.nonzero(G)
    d = i - j
    return int(max(d.max(), 0)), int(max(-d.min(), 0))


def galerkin_matrix(L, q, S, n_r):
    """P_q L S in plain coefficients: L acts on f_hat (columns scaled by C w_n), so
    f_hat = (S x) / (C w)."""
    hs = ch.hat_scale(n_r, L.shape[1])
    return L[q:, :] @ (S / hs[:, None])


def _banded(G, kl, ku):
    n = G.shape[0]
    ab = np.zeros((kl + ku + 1, n), dtype=G.dtype)
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[ku + i - j, j] = G[i, j]
    return ab


class _BandSystem:
    """G x = b by LAPACK's banded LU with partial pivoting, rows scaled to unit max."""

    def __init__(self, G, kl, ku):
        self.r = 1.0 / np.abs(G).max(axis=1)
        self.kl, self.ku = kl, ku
        self.ab = _banded(G * self.r[:, None], kl, ku)

    def solve(self, b):
        return sl.solve_banded((self.kl, self.ku), self.ab, b * self.r)


class GalerkinStepper(IntegrationStepper):
    """IntegrationStepper with the implicit systems solved in the Galerkin bases."""

    KL_PSI, KU_PSI, KL_DIR, KU_DIR = 8, 12, 4, 6

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        nc = self.n_c
        self.S_psi = stencil_psi(nc)
        self.S_dir = stencil_dir(nc)

    def _hat(self, c):
        return ch.plain_to_hat(c, self.ops.n_r)

    def lu(self, gamma):
        if gamma not in self._lu:
            gdt = gamma * self.dt
            ops, n_r = self.ops, self.ops.n_r
            lp = [None] + [_BandSystem(galerkin_matrix(ops.A(m) - gdt * ops.B(m), 4, self.S_psi, n_r),
                                       self.KL_PSI, self.KU_PSI) for m in range(1, self.g.M)]
            lt = [_BandSystem(galerkin_matrix(ops.D - gdt * ops.F(m) / ops.Pr, 2, self.S_dir, n_r),
                              self.KL_DIR, self.KU_DIR) for m in range(self.g.M)]
            lu_ = _BandSystem(galerkin_matrix(ops.D - gdt * ops.Ez, 2, self.S_dir, n_r), self.KL_DIR, self.KU_DIR)
            self._lu[gamma] = (lp, lt, lu_)
        return self._lu[gamma]

    def solve(self, gamma, rhs):
        lp, lt, lu_ = self.lu(gamma)
        rp, rt, ru = (np.array(r) for r in rhs)
        th = np.stack([self._hat(self.S_dir @ lt[m].solve(rt[m][2:])) for m in range(self.g.M)])
        if self.buoy_implicit:
            # the temperature first; its buoyancy joins the streamfunction rows
            gdt = gamma * self.dt
            for m in range(1, self.g.M):
                rp[m] = rp[m] + gdt * self._buoyancy(m, th[m])
        psi = np.zeros_like(rp)
        for m in range(1, self.g.M):
            psi[m] = self._hat(self.S_psi @ lp[m].solve(rp[m][4:]))
        u = self._hat(self.S_dir @ lu_.solve(ru[2:])).real
        return psi, th, u
