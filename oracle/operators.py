"""Radial operators of the two spectral formulations (Section 3).

Test infrastructure only (see the package docstring).

Chebyshev integration method (Section 3.2):
  A^I_m = int^4 s^4 L_I,  B^I_m = int^4 s^4 (Delta L_I + (2/E) i m),  C^I = int^4 s^4
                                                          (Eq. psi_int and below)
  D^I = int^2 s^2,  E^I = s^2 - 3 int s  (= int^2 s^2 (Delta - 1/s^2) at m = 0),
  F^I_m = int^2 s^2 Delta                          (Eqs. uphi_int, temp_int and below)
  G^I = int^2 h^2 : the conduction term of Eq. temp_int,
        D^I [i m (h^2/s) dT_c/ds Psi] = (alpha/ln eta) i m int^2 h^2 Psi,
        since s^2 (h^2/s)(alpha/(s ln eta)) = (alpha/ln eta) h^2 is a polynomial.
  with L_I Psi = Delta(h^2 Psi) - (1/s) d/ds(s^2 Psi)      (definition of L_I)
  and Delta = d2/ds2 + (1/s) d/ds - m^2/s^2 on one Fourier mode.

The construction follows the paper's recipe: multiply by s^q, write every term as
(polynomial) x (derivative), then integrate by parts until no derivative is left:
    int^q (Q d^p f) = sum_{j=0..p} (-1)^j binom(p,j) int^(q-p+j) (Q^(j) f)
(rows k >= q; lower rows only collect constants of integration and are replaced by
boundary-condition rows).  Every remaining term is an integral of a polynomial
times f, i.e. a product of the exact banded matrices of Eq. int1 and of
multiplication by x.  Rows below q are returned as zero.

Tau boundary rows (Eqs. bcs_coll_dirichlet, bcs_coll_neumann, bc_d3psi_coll).

Chebyshev collocation method (Section 3.1, Eqs. psiomcoll, uphicoll, tempcoll):
dense real matrices T, T', T'' at the Gauss-Lobatto points.

All returned matrices act on the paper's f_hat coefficients (columns scaled by
C w_n) and produce plain Chebyshev coefficients of the integrated equation.
"""
from math import comb

import numpy as np
import numpy.polynomial.polynomial as P
import scipy.sparse as sp

from . import chebyshev as ch
from .geometry import Annulus, gauss_lobatto


# ---------------------------------------------------------------------------
# Differential operators with Laurent-polynomial coefficients in s.
# key (p, i, j) -> coefficient of  mu^j s^i d^p/ds^p,  mu = m^2.
# ---------------------------------------------------------------------------

def _falling(i, k):
    out = 1.0
    for t in range(k):
        out *= (i - t)
    return out


def op_compose(A, B):
    """(A o B) f by the Leibniz rule d^p (s^i g) = sum_k binom(p,k) (s^i)^(k) d^(p-k) g."""
    out = {}
    for (p1, i1, j1), a in A.items():
        for (p2, i2, j2), b in B.items():
            for k in range(p1 + 1):
                f = _falling(i2, k)
                if f == 0.0:
                    continue
                key = (p1 - k + p2, i1 + i2 - k, j1 + j2)
                out[key] = out.get(key, 0.0) + a * b * comb(p1, k) * f
    return {k: v for k, v in out.items() if v != 0.0}


def op_add(*ops):
    out = {}
    for op in ops:
        for k, v in op.items():
            out[k] = out.get(k, 0.0) + v
    return {k: v for k, v in out.items() if v != 0.0}


def op_scale(A, c):
    return {k: c * v for k, v in A.items()}


def op_mul_spow(A, q):
    """Multiply an operator on the left by s^q."""
    return {(p, i + q, j): v for (p, i, j), v in A.items()}


def laplacian():
    return {(2, 0, 0): 1.0, (1, -1, 0): 1.0, (0, -2, 1): -1.0}


def L_I(s_o):
    """L_I Psi = Delta(h^2 Psi) - (1/s)(s^2 Psi)' = h^2 Psi'' + (h^2/s - 5s) Psi'
    - (6 + m^2 h^2/s^2) Psi, built here by composition from its definition."""
    h2 = {(0, 0, 0): s_o ** 2, (0, 2, 0): -1.0}          # multiplication by h^2
    lap_h2 = op_compose(laplacian(), h2)
    s2 = {(0, 2, 0): 1.0}
    d_s2 = op_compose({(1, 0, 0): 1.0}, s2)               # d/ds (s^2 .)
    return op_add(lap_h2, op_scale(op_mul_spow(d_s2, -1), -1.0))


# ---------------------------------------------------------------------------
# Integrated (banded) operators
# ---------------------------------------------------------------------------

def _poly_in_x(coeffs_s, ann):
    """sum_i c_i s^i with s = a x + b, as power-basis coefficients in x."""
    out = np.zeros(1)
    lin = np.array([ann.b, ann.a])
    powk = np.array([1.0])
    maxi = max(coeffs_s) if coeffs_s else 0
    for i in range(maxi + 1):
        c = coeffs_s.get(i, 0.0)
        if c != 0.0:
            out = P.polyadd(out, c * powk)
        powk = P.polymul(powk, lin)
    return out


def _poly_matrix(coef_x, X):
    """Q(X) for Q in the power basis (Horner); X sparse, result dense."""
    K = X.shape[0]
    R = np.zeros((K, K))
    for c in coef_x[::-1]:
        R = X @ R
        R[np.diag_indices(K)] += c
    return R


def integrated_operator(op, q, ann, n_c, mu_power):
    """Plain-coefficient matrix (n_c x n_c, rows < q zero) of int^q_s s^0 op, for
    the mu^mu_power part of ``op`` (which must have no negative powers of s)."""
    # gather polynomial coefficients per derivative order
    by_p = {}
    for (p, i, j), v in op.items():
        if j != mu_power:
            continue
        if i < 0:
            raise ValueError("operator still singular: multiply by a higher power of s")
        by_p.setdefault(p, {})
        by_p[p][i] = by_p[p].get(i, 0.0) + v
    if not by_p:
        return np.zeros((n_c, n_c))
    maxdeg = max(max(d) for d in by_p.values())
    Kp = n_c + 2 * (maxdeg + q) + 8
    # x-multiplication and integration are tri-/bidiagonal: stored sparse
    X = sp.csr_matrix(ch.xmul_matrix(Kp))
    J = sp.csr_matrix(ch.int_matrix(Kp))
    Jpow = [sp.identity(Kp, format="csr")]
    for _ in range(q):
        Jpow.append((J @ Jpow[-1]).tocsr())
    M = np.zeros((Kp, Kp))
    for p, cs in by_p.items():
        if p > q:
            raise ValueError("derivative order exceeds the number of integrations")
        Qx = _poly_in_x(cs, ann) * ann.a ** (-p)       # d/ds = (1/a) d/dx
        for j in range(p + 1):
            Qj = P.polyder(Qx, j) if j > 0 else Qx
            if len(Qj) == 0 or not np.any(Qj):
                continue
            M += (-1) ** j * comb(p, j) * (Jpow[q - p + j] @ _poly_matrix(Qj, X))
    M *= ann.a ** q                                     # int ds = a int dx
    out = M[:n_c, :n_c].copy()
    out[:q, :] = 0.0
    return out


def multiplication_operator(coeffs_s, ann, n_c, q_int):
    """int^q_int of (polynomial in s) x f, plain coefficients, rows < q_int zero."""
    return integrated_operator({(0, i, 0): c for i, c in coeffs_s.items()},
                               q_int, ann, n_c, 0)


# ---------------------------------------------------------------------------
# Tau rows, in plain coefficients
# ---------------------------------------------------------------------------

def bc_rows_plain(n_c, kind):
    n = np.arange(n_c, dtype=float)
    sgn = (-1.0) ** n
    if kind == "dir_o":
        return np.ones(n_c)
    if kind == "dir_i":
        return sgn.copy()
    if kind == "neu_o":
        return n ** 2
    if kind == "neu_i":
        return -sgn * n ** 2
    if kind == "d3_o":
        return n ** 2 * (n ** 2 - 1) * (n ** 2 - 4)
    raise ValueError(kind)


class IntegrationOperators:
    """All banded operators of the Chebyshev-integration formulation for one
    problem, acting on the paper's f_hat coefficients (columns scaled by C w_n)."""

    def __init__(self, n_r, n_c, eta, E, Pr, Ra):
        self.n_r, self.n_c = n_r, n_c
        self.ann = ann = Annulus(eta)
        self.E, self.Pr, self.Ra = float(E), float(Pr), float(Ra)
        sc = ch.hat_scale(n_r, n_c)[None, :]
        s_o = ann.s_o

        LI4 = op_mul_spow(L_I(s_o), 4)
        lap_LI4 = op_mul_spow(op_compose(laplacian(), L_I(s_o)), 4)
        self.A0 = integrated_operator(LI4, 4, ann, n_c, 0) * sc
        self.A2 = integrated_operator(LI4, 4, ann, n_c, 1) * sc
        self.B0 = integrated_operator(lap_LI4, 4, ann, n_c, 0) * sc
        self.B2 = integrated_operator(lap_LI4, 4, ann, n_c, 1) * sc
        self.B4 = integrated_operator(lap_LI4, 4, ann, n_c, 2) * sc
        self.C = multiplication_operator({4: 1.0}, ann, n_c, 4) * sc
        self.D = multiplication_operator({2: 1.0}, ann, n_c, 2) * sc
        lap2 = op_mul_spow(laplacian(), 2)
        self.F0 = integrated_operator(lap2, 2, ann, n_c, 0) * sc
        self.F2 = integrated_operator(lap2, 2, ann, n_c, 1) * sc
        # zonal flow: s^2 (Delta - 1/s^2) at m = 0
        zon = op_add({k: v for k, v in lap2.items() if k[2] == 0}, {(0, 0, 0): -1.0})
        self.Ez = integrated_operator(zon, 2, ann, n_c, 0) * sc
        self.G = multiplication_operator({0: s_o ** 2, 2: -1.0}, ann, n_c, 2) * sc

        self.bc_psi = np.stack([bc_rows_plain(n_c, k) for k in
                                ("dir_o", "dir_i", "d3_o", "neu_i")]) * sc
        self.bc_dir = np.stack([bc_rows_plain(n_c, k) for k in
                                ("dir_o", "dir_i")]) * sc
        self.tc_coef = ann.alpha / np.log(ann.eta)

    # m-dependent assemblies
    def A(self, m):
        return self.A0 + m * m * self.A2

    def B(self, m):
        mu = float(m * m)
        return (self.B0 + mu * self.B2 + mu * mu * self.B4) + 1j * m * (2.0 / self.E) * self.C

    def F(self, m):
        return self.F0 + m * m * self.F2

    # left-hand sides with the tau rows on top
    def lhs_psi(self, m, gdt):
        L = (self.A(m) - gdt * self.B(m)).astype(complex)
        L[:4, :] = self.bc_psi
        return L

    def lhs_theta(self, m, gdt):
        L = self.D - gdt * self.F(m) / self.Pr
        L = L.copy()
        L[:2, :] = self.bc_dir
        return L

    def lhs_uphi(self, gdt):
        L = (self.D - gdt * self.Ez).copy()
        L[:2, :] = self.bc_dir
        return L
