"""One IMEX time step of the Chebyshev-integration / tau formulation
(Sections 3.2 and 4; Eqs. psi_int, uphi_int, temp_int, multistep1, dirks).

Test infrastructure only (see the package docstring).

Unknowns per Fourier mode m: Psi_hat_m (m >= 1; Psi_0 = 0), theta_hat_m, and
u_hat (m = 0 zonal flow), each with N_c = floor(2 (N_r - 1)/3) coefficients.
Semi-discrete system (rows k >= q of the q-times integrated equations):
    A^I_m dPsi/dt = B^I_m Psi + e_psi
    D^I dtheta/dt = (F^I_m/Pr) theta + e_theta
    D^I du/dt     = E^I u + e_u
the explicit parts e_* coming from ``explicit.explicit_terms``.  The implicit
systems carry the tau rows on top (4 for Psi, 2 for theta and u) with zero right
hand side.  They are solved here by dense LU with partial pivoting after scaling
every row to unit maximum: the tau rows grow like n^6 (the third-derivative row)
while the integrated rows shrink like n^-4, and pivoting on the unscaled matrix
loses up to 8 digits at n_r = 257 (row scaling leaves the solution unchanged).
One step of iterative refinement with an FP64 residual follows (at n_r = 2049 it
takes the solution from ~1e-11 to ~1e-13 of an extended-precision reference).
``bordered_solve`` is the Appendix A algorithm, kept separate and pinned against
the dense solve.
"""
import numpy as np
import scipy.linalg as sl

from .explicit import Grid, explicit_terms
from .operators import IntegrationOperators
from . import schemes


def n_c_integration(n_r):
    return (2 * (n_r - 1)) // 3


def bordered_solve(Mat, f, p):
    """Appendix A: (A B; C D)(psi1; psi2) = (g; h) with A of size p x p.
    D x = h, D y = C, M = A - B y, M psi1 = g - B x, psi2 = x - y psi1."""
    A = Mat[:p, :p]
    B = Mat[:p, p:]
    C = Mat[p:, :p]
    D = Mat[p:, p:]
    g, h = f[:p], f[p:]
    x = np.linalg.solve(D, h)
    y = np.linalg.solve(D, C)
    Ms = A - B @ y
    psi1 = np.linalg.solve(Ms, g - B @ x)
    psi2 = x - y @ psi1
    return np.concatenate([psi1, psi2])


class ImexScheme:
    """Scheme logic of Eqs. multistep1 and dirks on tuples of per-field arrays;
    subclasses provide mass(y), imp(y), explicit(y) and solve(gamma, rhs)."""

    @staticmethod
    def _axpy(acc, c, v):
        return tuple(a + c * b for a, b in zip(acc, v))

    def step(self):
        if self.scheme in schemes.MULTISTEP:
            self._step_multistep()
        else:
            self._step_dirk()
        self.n_done += 1
        return self.y

    def _step_multistep(self):
        a, b0, bI, bE = schemes.multistep_coeffs(self.scheme, self.n_done)
        dt = self.dt
        e_n = self.explicit(self.y)
        ys = [self.y] + self.hist_y
        es = [e_n] + self.hist_e
        zero = tuple(np.zeros_like(v) for v in self.mass(self.y))
        rhs = zero
        for j, aj in enumerate(a):
            rhs = self._axpy(rhs, aj, self.mass(ys[j]))
        for j, bj in enumerate(bI):
            if bj != 0.0:
                rhs = self._axpy(rhs, dt * bj, self.imp(ys[j]))
        for j, bj in enumerate(bE):
            rhs = self._axpy(rhs, dt * bj, es[j])
        y_new = self.solve(b0, rhs)
        keep = 2
        self.hist_y = ys[:keep]
        self.hist_e = es[:keep]
        self.y = y_new

    def _step_dirk(self):
        aI, aE = schemes.dirk_tableau(self.scheme)
        nu = aI.shape[0] - 1
        dt = self.dt
        ys = [self.y]
        es, imps = [], {}
        rhs0 = self.mass(self.y)
        for i in range(1, nu + 1):
            es.append(self.explicit(ys[i - 1]))
            rhs = rhs0
            for j in range(i):
                if aE[i, j] != 0.0:
                    rhs = self._axpy(rhs, dt * aE[i, j], es[j])
                if aI[i, j] != 0.0:
                    if j not in imps:
                        imps[j] = self.imp(ys[j])
                    rhs = self._axpy(rhs, dt * aI[i, j], imps[j])
            ys.append(self.solve(aI[i, i], rhs))
        self.y = ys[nu]


class IntegrationStepper(ImexScheme):
    def __init__(self, n_r, n_phi, E, Ra, Pr, eta, scheme, dt, pumping_eps=None, buoy_implicit=False):
        if scheme not in schemes.SCHEME_ID:
            raise ValueError(scheme)
        self.n_c = n_c_integration(n_r)
        self.ops = IntegrationOperators(n_r, self.n_c, eta, E, Pr, Ra)
        self.g = Grid(self.ops, n_phi)
        self.g.pump_eps = pumping_eps       # Ekman pumping, explicit (Eq. approx_pump)
        # implicit buoyancy (Section 4): (Ra/Pr)(i m/s_o) C^I theta joins the implicit
        # operator of the streamfunction equation; the temperature is advanced first
        self.buoy_implicit = bool(buoy_implicit)
        self.g.buoy_implicit = self.buoy_implicit
        self.scheme, self.dt = scheme, float(dt)
        self._lu = {}
        self.n_done = 0
        self.hist_y, self.hist_e = [], []
        M, nc = self.g.M, self.n_c
        self.y = (np.zeros((M, nc), complex), np.zeros((M, nc), complex), np.zeros(nc))

    # -- state ---------------------------------------------------------------
    def set_state(self, psi, theta, u):
        self.y = (np.array(psi, complex), np.array(theta, complex), np.array(u, float))
        self.y[0][0] = 0.0
        self.n_done = 0
        self.hist_y, self.hist_e = [], []

    # -- operators -----------------------------------------------------------
    def mass(self, y):
        psi, th, u = y
        ops = self.ops
        mp = np.stack([ops.A(m) @ psi[m] for m in range(self.g.M)])
        mp[0] = 0.0
        return mp, (ops.D @ th.T).T, ops.D @ u

    def imp(self, y):
        psi, th, u = y
        ops = self.ops
        ip = np.stack([ops.B(m) @ psi[m] for m in range(self.g.M)])
        if self.buoy_implicit:
            ip = ip + np.stack([self._buoyancy(m, th[m]) for m in range(self.g.M)])
        ip[0] = 0.0
        it = np.stack([ops.F(m) @ th[m] for m in range(self.g.M)]) / ops.Pr
        return ip, it, ops.Ez @ u

    def explicit(self, y):
        return explicit_terms(self.g, *y)

    def _buoyancy(self, m, theta_m):
        """(Ra/Pr)(i m/s_o) C^I theta_m, the buoyancy term of Eq. psi_int."""
        ops = self.ops
        return (ops.Ra / ops.Pr) * (1j * m / ops.ann.s_o) * (ops.C @ theta_m)

    @staticmethod
    def _factor(L):
        """LU of the row-scaled matrix; returns (lu, row scales)."""
        r = 1.0 / np.abs(L).max(axis=1)
        return sl.lu_factor(L * r[:, None]), r

    @staticmethod
    def _solve(fac, b):
        lu, r = fac
        return sl.lu_solve(lu, b * r)

    def lu(self, gamma):
        if gamma not in self._lu:
            gdt = gamma * self.dt
            ops = self.ops
            lp = [None] + [(self._factor(L), L) for L in (ops.lhs_psi(m, gdt) for m in range(1, self.g.M))]
            lt = [(self._factor(L), L) for L in (ops.lhs_theta(m, gdt).astype(complex) for m in range(self.g.M))]
            Lu = ops.lhs_uphi(gdt)
            lu_ = (self._factor(Lu), Lu)
            self._lu[gamma] = (lp, lt, lu_)
        return self._lu[gamma]

    @classmethod
    def _solve_refined(cls, fac, L, b):
        x = cls._solve(fac, b)
        return x + cls._solve(fac, b - L @ x)

    def solve(self, gamma, rhs):
        lp, lt, lu_ = self.lu(gamma)
        rp, rt, ru = (np.array(r) for r in rhs)
        rp[:, :4] = 0.0
        rt[:, :2] = 0.0
        ru[:2] = 0.0
        th = np.stack([self._solve_refined(*lt[m], rt[m]) for m in range(self.g.M)])
        if self.buoy_implicit:
            # (Mass - g Lin) y = r with Lin_psi = B Psi + buoyancy(theta): the
            # temperature is solved first, its buoyancy moves to the right-hand side
            gdt = gamma * self.dt
            for m in range(1, self.g.M):
                rp[m] = rp[m] + gdt * self._buoyancy(m, th[m])
            rp[:, :4] = 0.0
        psi = np.zeros_like(rp)
        for m in range(1, self.g.M):
            psi[m] = self._solve_refined(*lp[m], rp[m])
        u = self._solve_refined(*lu_, ru)
        return psi, th, u
