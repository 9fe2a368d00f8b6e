"""Linear onset of convection (Section 6.1, Eq. lin), solved with the
Chebyshev-integration operators of this oracle.

Test infrastructure only (see the package docstring).

For one azimuthal wavenumber m, normal modes f ~ exp(i m phi + lambda t) of the
linearised equations satisfy the generalised eigenproblem
    lambda A^I Psi = B^I Psi + (Ra/Pr)(i m/s_o) C^I theta
    lambda D^I theta = (1/Pr) F^I theta - (alpha/ln eta) i m G^I Psi
with the tau rows of the boundary conditions (zero mass).  Reading: the printed
Eq. lin omits the 1/Pr of the diffusion term that Eq. temp carries; the paper's own
eigenvalues (tau = 6.149994e2, omega_d = -9.536952e3 at E = 3e-6, Pr = 0.025,
Ra = 1e7, m = 12) are reproduced only with 1/Pr, so 1/Pr is kept.

lambda = tau + i omega_d.  The tau method adds spurious eigenvalues of huge
modulus; they are discarded (|lambda| > 1e8) and the leading eigenvalue is then
refined by shift-and-invert around the QZ estimate.
"""
import numpy as np
import scipy.linalg as sl
from scipy.optimize import brentq

from .operators import IntegrationOperators


def pencil(E, Pr, Ra, eta, m, n_c, n_r=None, pumping_eps=None):
    """(L, M) in the f_hat coordinates of a radial grid of n_r points (the
    eigenvalues do not depend on n_r, the column scaling of the vectors does).
    pumping_eps: the approximate Ekman pumping F_eps of Eq. approx_pump, the
    linear map of the explicit stage (grid values, Eq. icheb, truncation), which
    enters the streamfunction rows as -C^I F_eps (Eq. psiint)."""
    n_r = int(1.5 * n_c) + 2 if n_r is None else n_r
    op = IntegrationOperators(n_r, n_c, eta, E, Pr, Ra)
    n = n_c
    L = np.zeros((2 * n, 2 * n), complex)
    M = np.zeros((2 * n, 2 * n), complex)
    M[:n, :n] = op.A(m)
    L[:n, :n] = op.B(m)
    if pumping_eps is not None:
        from .explicit import Grid
        from .pumping import integration_matrix
        g = Grid(op, 3 * (m + 1))
        L[:n, :n] -= op.C @ integration_matrix(g, m, pumping_eps)
    L[:n, n:] = (Ra / Pr) * (1j * m / op.ann.s_o) * op.C
    M[n:, n:] = op.D
    L[n:, n:] = op.F(m) / Pr
    L[n:, :n] = -op.tc_coef * 1j * m * op.G
    M[:4, :] = 0.0
    L[:4, :] = 0.0
    L[:4, :n] = op.bc_psi
    M[n:n + 2, :] = 0.0
    L[n:n + 2, :] = 0.0
    L[n:n + 2, n:] = op.bc_dir
    return L, M


def leading_eigenvalue(E, Pr, Ra, eta, m, n_c, guess=None, n_r=None, pumping_eps=None):
    return leading_of_pencil(*pencil(E, Pr, Ra, eta, m, n_c, n_r, pumping_eps), guess)


def leading_of_pencil(L, M, guess=None):
    """Eigenvalue of L x = lambda M x of largest real part among the finite ones
    (QZ estimate unless ``guess`` is given), refined by shift-and-invert."""
    if guess is None:
        w = sl.eig(L, M, right=False)
        w = w[np.isfinite(w) & (np.abs(w) < 1e8)]
        guess = w[np.argmax(w.real)]
    lu = sl.lu_factor(L - guess * M)
    mu = sl.eigvals(sl.lu_solve(lu, M))
    mu = mu[np.abs(mu) > 1e-300]
    lam = guess + 1.0 / mu
    lam = lam[np.abs(lam) < 1e8]
    return lam[np.argmin(np.abs(lam - guess))]


def leading_mode(E, Pr, Ra, eta, m, n_c, n_r=None, guess=None, pumping_eps=None):
    """Leading eigenvalue and its eigenvector (Psi_hat, theta_hat), unit 2-norm,
    by inverse iteration at the refined eigenvalue."""
    L, M = pencil(E, Pr, Ra, eta, m, n_c, n_r, pumping_eps)
    lam = leading_of_pencil(L, M, guess)
    lu = sl.lu_factor(L - lam * M)
    x = np.ones(2 * n_c, complex)
    for _ in range(3):
        x = sl.lu_solve(lu, M @ x)
        x /= np.linalg.norm(x)
    return lam, x[:n_c], x[n_c:]


def critical_rayleigh_m(E, Pr, eta, m, n_c, ra_lo, ra_hi, rtol=1e-9, eigenvalue=None):
    """Ra at which the leading growth rate of mode m crosses zero, bracketed by
    [ra_lo, ra_hi].  ``eigenvalue(m, ra)``, when given, returns the leading
    eigenvalue of another discretisation of Eq. lin (default: the
    integration/tau pencil of this module)."""
    lead = eigenvalue or (lambda mm, ra: leading_eigenvalue(E, Pr, ra, eta, mm, n_c))
    ra = brentq(lambda r: lead(m, r).real, ra_lo, ra_hi, rtol=rtol)
    return ra, lead(m, ra)


def critical_rayleigh(E, Pr, eta, m_values, n_c, ra_lo, ra_hi, eigenvalue=None):
    """Minimum over m of the marginal Ra: returns (Ra_c, m_c, omega_d)."""
    best = None
    for m in m_values:
        ra, lam = critical_rayleigh_m(E, Pr, eta, m, n_c, ra_lo, ra_hi, eigenvalue=eigenvalue)
        if best is None or ra < best[0]:
            best = (ra, m, lam.imag)
    return best


def leading_eigenvalue_arnoldi(E, Pr, Ra, eta, m, n_c, guess, k=6):
    """Eigenvalues nearest ``guess`` by Arnoldi iteration on (L - guess M)^{-1} M;
    returns the one of largest real part among them."""
    from scipy.sparse.linalg import LinearOperator, eigs
    L, M = pencil(E, Pr, Ra, eta, m, n_c)
    lu = sl.lu_factor(L - guess * M)
    n = L.shape[0]
    op = LinearOperator((n, n), matvec=lambda x: sl.lu_solve(lu, M @ x), dtype=complex)
    mu = eigs(op, k=k, return_eigenvectors=False, tol=1e-13)
    lam = guess + 1.0 / mu
    lam = lam[np.abs(lam) < 1e8]
    return lam[np.argmax(lam.real)]


def marginal_rayleigh(E, Pr, eta, m, n_c, ra0, guess=None, rtol=1e-10, eigenvalue=None):
    """Ra at which the leading growth rate of mode m vanishes, by bracketing from
    ra0 with factor-2 steps and then Brent's method; returns (Ra, lambda).

    ``eigenvalue(ra, g)``, when given, replaces the integration/tau pencil of this
    module: it returns the eigenvalue of the discretised Eq. lin nearest the
    branch guess g (g = i omega_d of the previous evaluation, or ``guess`` first;
    None: the leading one).  This lets the same root finder run on the
    collocation pencil, with or without Ekman pumping."""
    state = {"g": guess}
    memo = {}

    def tau(ra):
        if ra in memo:
            return memo[ra]
        if eigenvalue is not None:
            lam = eigenvalue(ra, state["g"])
            state["g"] = 1j * lam.imag
            memo[ra] = lam.real
            return lam.real
        lam = None
        if state["g"] is not None:
            lam = leading_eigenvalue_arnoldi(E, Pr, ra, eta, m, n_c, state["g"])
            # accept only a continuation of the same branch
            if abs(lam.imag - state["g"].imag) > 0.2 * abs(state["g"].imag) + 1.0:
                lam = None
        if lam is None:
            lam = leading_eigenvalue(E, Pr, ra, eta, m, n_c)
        state["g"] = 1j * lam.imag
        memo[ra] = lam.real
        return lam.real

    lo = hi = ra0
    t0 = tau(ra0)
    if t0 < 0:
        while True:
            hi *= 2.0
            if tau(hi) > 0:
                break
            lo = hi
    else:
        while True:
            lo /= 2.0
            if tau(lo) < 0:
                break
            hi = lo
    ra = brentq(tau, lo, hi, rtol=rtol)
    if eigenvalue is not None:
        return ra, eigenvalue(ra, state["g"])
    lam = leading_eigenvalue(E, Pr, ra, eta, m, n_c, guess=state["g"])
    return ra, lam
