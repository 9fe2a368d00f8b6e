"""Chebyshev-collocation formulation of the step (Section 3.1; Eqs. psiomcoll,
uphicoll, tempcoll, bcs_coll_dirichlet, bcs_coll_neumann).

Test infrastructure only (see the package docstring).

Unknowns per mode (N_c = N_r, paper coefficients with both ends halved):
omega_hat and psi_hat (m >= 1), theta_hat, and u_hat (m = 0).  With T, T', T''
the Chebyshev polynomials and their s-derivatives at the Gauss-Lobatto points,
and Ekman pumping off (Upsilon = 0; with ``pumping`` the exact terms of
``pumping.collocation_blocks`` join A^C, B^C and the zonal-flow operator, all
implicit):
  A^C = T'' + T'/s - (m^2/s^2) T
  B^C = -(2/E)(i m beta/s) T
  C^C = T'' + (beta + 1/s) T' + (dbeta/ds + beta/s - m^2/s^2) T
  (reading: the printed -(dbeta/ds + beta/s + m^2/s^2) contradicts the definition
  L_beta psi = Delta psi + (1/s) d(beta s psi)/ds; the definition is used)
  vorticity rows:  d/dt (T omega) = A^C omega - B^C psi + e_omega
  constraint rows: T omega + C^C psi = 0
  e_omega = -(Ra/Pr)(i m/s_o) theta - N_omega
  temperature:     d/dt (T theta) = (1/Pr)(T'' + T'/s - m^2 T/s^2) theta + e_theta,
  e_theta = -(i m/s) dT_c/ds psi - N_theta       (reading: -u_s dT_c/ds, as Eq. temp)
  zonal flow:      d/dt (T u) = (T'' + T'/s - T/s^2) u + e_u,   e_u = -N_u
at the interior points; the four streamfunction conditions replace the first
and last rows of both blocks (reading: Neumann in the vorticity block,
Dirichlet in the constraint block), Dirichlet rows close temperature and zonal
flow.  Nonlinear terms in flux form with v = d psi/d phi = s u_s:
  N_omega = (1/s) d(v omega)/ds + (i m/s)[u_phi omega]_m
  N_theta = (1/s) d(v theta)/ds + (i m/s)[u_phi theta]_m + (beta/s)[v theta]_m
  N_u     = [v omega]_0 / s,   u_phi = u_bar - dpsi/ds - beta psi
(beta psi and beta-terms are set to 0 at s_o, where psi = 0 and the rows are
boundary rows).  Systems solved by dense LU with row scaling and one
refinement step, as in ``stepper``.
"""
import numpy as np
import scipy.linalg as sl

from . import chebyshev as ch
from . import fourier as fo
from .geometry import Annulus, gauss_lobatto
from .operators import bc_rows_plain
from .onset import leading_of_pencil
from .pumping import collocation_blocks, upsilon
from .stepper import ImexScheme
from . import schemes


class CollocationOperators:
    def __init__(self, n_r, eta, E, Pr, Ra, pumping=False):
        self.n_r = self.n_c = n_r
        self.pumping = bool(pumping)
        self.ann = ann = Annulus(eta)
        self.E, self.Pr, self.Ra = float(E), float(Pr), float(Ra)
        N = n_r
        x = gauss_lobatto(N)
        self.s = s = ann.s_of_x(x)
        h2 = ann.h2(s)
        h2[0] = 0.0
        self.beta = np.zeros(N)
        self.beta[1:] = -s[1:] / h2[1:]
        self.dbeta = np.zeros(N)
        self.dbeta[1:] = -(ann.s_o ** 2 + s[1:] ** 2) / h2[1:] ** 2
        sc = ch.hat_scale(N, N)[None, :]
        Tp = ch.tmat(N, N)
        Dn = ch.diff_matrix(N) / ann.a
        self.T = Tp * sc
        self.T1 = (Tp @ Dn) * sc
        self.T2 = (Tp @ Dn @ Dn) * sc
        si = (1.0 / s)[:, None]
        self.Q = self.T2 + si * self.T1                      # T'' + T'/s
        self.tc = ann.dTc_ds(s)
        self.bc = {k: bc_rows_plain(N, k) * sc[0] for k in ("dir_o", "dir_i", "neu_o", "neu_i")}

    def A(self, m):
        return self.Q - (m * m / self.s ** 2)[:, None] * self.T

    def pump(self, m):
        """(F_omega, F_psi) of the exact Ekman pumping for mode m (zeros when off)."""
        if not self.pumping or m == 0:
            z = np.zeros_like(self.T)
            return z, z
        Fw, Fpsi, _ = collocation_blocks(self, m)
        return Fw, Fpsi

    def Bdiag(self, m):
        """B^C = diag(bdiag) T."""
        return -(2.0 / self.E) * 1j * m * self.beta / self.s

    def C(self, m):
        s = self.s
        return (self.T2 + (self.beta + 1.0 / s)[:, None] * self.T1
                + (self.dbeta + self.beta / s - m * m / s ** 2)[:, None] * self.T)

    def Lt(self, m):
        return (self.Q - (m * m / self.s ** 2)[:, None] * self.T) / self.Pr

    def Lu(self):
        L = self.Q - (1.0 / self.s ** 2)[:, None] * self.T
        if self.pumping:
            L = L + collocation_blocks(self, 1)[2]
        return L

    def lhs_wpsi(self, m, gdt):
        N = self.n_r
        L = np.zeros((2 * N, 2 * N), complex)
        Fw, Fpsi = self.pump(m)
        L[:N, :N] = self.T - gdt * (self.A(m) + Fw)
        L[:N, N:] = gdt * (self.Bdiag(m)[:, None] * self.T - Fpsi)
        L[N:, :N] = self.T
        L[N:, N:] = self.C(m)
        for row in (0, N - 1, N, 2 * N - 1):
            L[row, :] = 0.0
        L[0, N:] = self.bc["neu_o"]
        L[N - 1, N:] = self.bc["neu_i"]
        L[N, N:] = self.bc["dir_o"]
        L[2 * N - 1, N:] = self.bc["dir_i"]
        return L

    def lhs_dir(self, Lin, gdt):
        L = (self.T - gdt * Lin).astype(complex)
        L[0] = self.bc["dir_o"]
        L[-1] = self.bc["dir_i"]
        return L


class CollocationStepper(ImexScheme):
    """State tuple (omega_hat, psi_hat, theta_hat, u_hat); mass/imp/explicit return
    grid-row tuples (omega rows, constraint rows, theta rows, u rows)."""

    def __init__(self, n_r, n_phi, E, Ra, Pr, eta, scheme, dt, pumping=False, buoy_implicit=False):
        if scheme not in schemes.SCHEME_ID:
            raise ValueError(scheme)
        self.ops = CollocationOperators(n_r, eta, E, Pr, Ra, pumping)
        # implicit buoyancy (Section 4): -(Ra/Pr)(i m/s_o) theta joins the implicit
        # operator of the vorticity rows; the temperature is solved first
        self.buoy_implicit = bool(buoy_implicit)
        self.n_c = n_r
        if n_phi % 3:
            raise ValueError("N_phi must be a multiple of 3")
        self.n_phi, self.n_m, self.M = n_phi, n_phi // 3, n_phi // 3 + 1
        self.scheme, self.dt = scheme, float(dt)
        self._lu = {}
        self.n_done = 0
        self.hist_y, self.hist_e = [], []
        z = np.zeros((self.M, n_r), complex)
        self.y = (z.copy(), z.copy(), z.copy(), np.zeros(n_r))

    def set_state(self, omega, psi, theta, u):
        self.y = (np.array(omega, complex), np.array(psi, complex), np.array(theta, complex),
                  np.array(u, float))
        self.y[0][0] = 0.0
        self.y[1][0] = 0.0
        self.n_done = 0
        self.hist_y, self.hist_e = [], []

    def vorticity_from_psi(self, psi):
        """omega_hat = Eq. icheb of -L_beta psi on the grid; at s_o the beta terms
        take their limit for psi = dpsi/ds = 0 there: L_beta psi -> (5/4) psi''."""
        o = self.ops
        out = np.zeros_like(psi)
        for m in range(1, self.M):
            p = o.T @ psi[m]
            p2 = o.T2 @ psi[m]
            L = o.C(m) @ psi[m]
            L[0] = 1.25 * p2[0]
            out[m] = ch.analysis(-L, o.n_r)
        return out

    # -- grid rows ----------------------------------------------------------
    def mass(self, y):
        w, psi, th, u = y
        T = self.ops.T
        mw = (T @ w.T).T
        mw[0] = 0.0
        return mw, np.zeros_like(psi), (T @ th.T).T, T @ u

    def imp(self, y):
        w, psi, th, u = y
        o = self.ops
        iw = np.stack([o.A(m) @ w[m] - o.Bdiag(m) * (o.T @ psi[m]) + o.pump(m)[0] @ w[m] + o.pump(m)[1] @ psi[m]
                       for m in range(self.M)])
        if self.buoy_implicit:
            iw = iw + np.stack([self._buoyancy(m, th[m]) for m in range(self.M)])
        iw[0] = 0.0
        it = np.stack([o.Lt(m) @ th[m] for m in range(self.M)])
        return iw, np.zeros_like(psi), it, o.Lu() @ u

    def explicit(self, y):
        w, psi, th, u = y
        o = self.ops
        N = o.n_r
        s = o.s[:, None]
        m = np.arange(self.M)[None, :]
        P = (o.T @ psi.T)
        dP = (o.T1 @ psi.T)
        W = (o.T @ w.T)
        TH = (o.T @ th.T)
        ub = o.T @ u
        dub = o.T1 @ u
        v = 1j * m * P
        bpsi = o.beta[:, None] * P
        bpsi[0] = 0.0
        uphi = -dP - bpsi
        uphi[:, 0] = ub
        W[:, 0] = dub + ub / o.s
        v[:, 0] = 0.0
        prods = []
        for a, b in ((v, W), (uphi, W), (v, TH), (uphi, TH)):
            prods.append(fo.to_spec(fo.to_grid(a, self.n_phi) * fo.to_grid(b, self.n_phi), self.n_m))
        vw, uw, vt, ut = prods
        deriv = lambda f: o.T1 @ ch.analysis(f, N)
        Nw = (deriv(vw) + 1j * m * uw) / s
        bt = o.beta[:, None] * vt / s
        bt[0] = 0.0
        Nt = (deriv(vt) + 1j * m * ut) / s + bt
        Nu = vw[:, 0] / o.s
        if o.pumping:   # self-interaction of the zonal wind (Eq. uphicoll), explicit
            ups = upsilon(o.ann, o.E, o.s)
            ups[0] = 0.0
            Nu = Nu + 0.5 * o.E * ups * ub * W[:, 0]
        ew = -(o.Ra / o.Pr) * (1j * m / o.ann.s_o) * TH - Nw
        if self.buoy_implicit:
            ew = -Nw
        et = -(1j * m / s) * o.tc[:, None] * P - Nt
        eu = -Nu
        ew[:, 0] = 0.0
        for a in (ew, et):
            a[0] = 0.0
            a[-1] = 0.0
        eu = eu.real.copy()
        eu[0] = eu[-1] = 0.0
        return ew.T, np.zeros_like(psi), et.T, eu

    def _buoyancy(self, m, theta_m):
        """-(Ra/Pr)(i m/s_o) theta on the grid rows (vorticity equation, Eq. psiomcoll)."""
        o = self.ops
        return -(o.Ra / o.Pr) * (1j * m / o.ann.s_o) * (o.T @ theta_m)

    # -- solve --------------------------------------------------------------
    @staticmethod
    def _factor(L):
        r = 1.0 / np.abs(L).max(axis=1)
        return sl.lu_factor(L * r[:, None]), r, L

    @staticmethod
    def _solve(fac, b):
        lu, r, L = fac
        x = sl.lu_solve(lu, b * r)
        return x + sl.lu_solve(lu, (b - L @ x) * r)

    def lu(self, gamma):
        if gamma not in self._lu:
            o = self.ops
            gdt = gamma * self.dt
            lw = [None] + [self._factor(o.lhs_wpsi(m, gdt)) for m in range(1, self.M)]
            lt = [self._factor(o.lhs_dir(o.Lt(m), gdt)) for m in range(self.M)]
            lu_ = self._factor(o.lhs_dir(o.Lu(), gdt).real)
            self._lu[gamma] = (lw, lt, lu_)
        return self._lu[gamma]

    def solve(self, gamma, rhs):
        lw, lt, lu_ = self.lu(gamma)
        rw, _, rt, ru = (np.array(r) for r in rhs)
        N = self.n_c
        rt[:, 0] = rt[:, -1] = 0.0
        th = np.stack([self._solve(lt[m], rt[m]) for m in range(self.M)])
        if self.buoy_implicit:
            gdt = gamma * self.dt
            for m in range(1, self.M):
                rw[m] = rw[m] + gdt * self._buoyancy(m, th[m])
        w = np.zeros_like(rw)
        psi = np.zeros_like(rw)
        for m in range(1, self.M):
            b = np.zeros(2 * N, complex)
            b[1:N - 1] = rw[m, 1:N - 1]
            x = self._solve(lw[m], b)
            w[m], psi[m] = x[:N], x[N:]
        ru[0] = ru[-1] = 0.0
        u = self._solve(lu_, ru)
        return w, psi, th, u

    def grid_state(self):
        """u_s, u_phi, omega, theta Fourier coefficients on the radial grid."""
        w, psi, th, u = self.y
        o = self.ops
        m = np.arange(self.M)[None, :]
        P = o.T @ psi.T
        bpsi = o.beta[:, None] * P
        bpsi[0] = 0.0
        us = 1j * m * P / o.s[:, None]
        uphi = -(o.T1 @ psi.T) - bpsi
        uphi[:, 0] = o.T @ u
        W = o.T @ w.T
        W[:, 0] = o.T1 @ u + (o.T @ u) / o.s
        return us, uphi, W, o.T @ th.T


def collocation_pencil(E, Pr, Ra, eta, m, n_r, pumping=False):
    """Linearised Eqs. psiomcoll and tempcoll for normal modes exp(i m phi +
    lambda t): unknowns (omega_hat, psi_hat, theta_hat); boundary rows carry no
    mass.  ``pumping``: the exact Ekman pumping of Eq. pumping_full."""
    o = CollocationOperators(n_r, eta, E, Pr, Ra, pumping)
    Fw, Fpsi = o.pump(m)
    N = n_r
    L = np.zeros((3 * N, 3 * N), complex)
    M = np.zeros((3 * N, 3 * N), complex)
    M[:N, :N] = o.T
    L[:N, :N] = o.A(m) + Fw
    L[:N, N:2 * N] = -o.Bdiag(m)[:, None] * o.T + Fpsi
    L[:N, 2 * N:] = -(Ra / Pr) * (1j * m / o.ann.s_o) * o.T
    L[N:2 * N, :N] = o.T
    L[N:2 * N, N:2 * N] = o.C(m)
    M[2 * N:, 2 * N:] = o.T
    L[2 * N:, 2 * N:] = o.Lt(m)
    L[2 * N:, N:2 * N] = -(1j * m / o.s * o.tc)[:, None] * o.T
    rows = {0: ("neu_o", N), N - 1: ("neu_i", N), N: ("dir_o", N), 2 * N - 1: ("dir_i", N),
            2 * N: ("dir_o", 2 * N), 3 * N - 1: ("dir_i", 2 * N)}
    for r, (kind, c0) in rows.items():
        M[r] = 0.0
        L[r] = 0.0
        L[r, c0:c0 + N] = o.bc[kind]
    return L, M


def leading_eigenvalue_collocation(E, Pr, Ra, eta, m, n_r, guess=None, pumping=False):
    return leading_of_pencil(*collocation_pencil(E, Pr, Ra, eta, m, n_r, pumping), guess)


def leading_mode_collocation(E, Pr, Ra, eta, m, n_r, guess=None, pumping=False):
    """Leading eigenvalue and eigenvector (omega_hat, psi_hat, theta_hat), unit
    2-norm, by inverse iteration at the refined eigenvalue."""
    L, M = collocation_pencil(E, Pr, Ra, eta, m, n_r, pumping)
    lam = leading_of_pencil(L, M, guess)
    lu = sl.lu_factor(L - lam * M)
    x = np.ones(3 * n_r, complex)
    for _ in range(3):
        x = sl.lu_solve(lu, M @ x)
        x /= np.linalg.norm(x)
    return lam, x[:n_r], x[n_r:2 * n_r], x[2 * n_r:]
