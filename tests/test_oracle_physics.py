"""Pins of the oracle's linear physics, time schemes, bordered solve and
nonlinear terms against values the paper prints, closed forms and exact
analytic evaluation."""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.optimize import brentq
from scipy.special import jv, yv

from oracle import chebyshev as ch
from oracle import schemes
from oracle.explicit import explicit_terms
from oracle.geometry import Annulus, gauss_lobatto
from oracle.onset import leading_eigenvalue, leading_mode
from oracle.stepper import IntegrationStepper, bordered_solve


# ---------------------------------------------------------------- onset ----
def test_onset_eigenvalue_matches_the_paper():
    """Table 3 (LSB row, without Ekman pumping): E = 3e-6, Pr = 0.025, Ra = 1e7,
    eta = 0.35, m = 12: tau = 6.149994e2, omega_d = -9.536952e3."""
    lam = leading_eigenvalue(3e-6, 0.025, 1e7, 0.35, 12, 192, guess=615.0 - 9537.0j)
    assert abs(lam.real - 614.9994) < 1e-6 * 615.0
    assert abs(lam.imag - (-9536.952)) < 1e-6 * 9537.0


def test_dns_from_eigenmode_grows_at_the_eigenvalue():
    """Section 6.1 validation on a coarse grid: a time-stepped run started from the
    onset solver's leading m = 12 eigenmode (E = 3e-6, Ra = 1e7, Pr = 0.025) grows
    and drifts at that eigenvalue.  The stepper and the onset pencil are assembled
    separately (explicit buoyancy and T_c coupling on the grid in the stepper,
    matrix blocks in the pencil), so a wrong sign or factor in either fails here.
    CNAB2 with dt = 2e-7: the splitting error in lambda is O((lambda dt)^2 lambda)."""
    n_r, n_phi, dt, m = 65, 48, 2e-7, 12
    nc = (2 * (n_r - 1)) // 3
    lam, p, th = leading_mode(3e-6, 0.025, 1e7, 0.35, m, nc, n_r=n_r, guess=615.0 - 9537.0j)
    st = IntegrationStepper(n_r, n_phi, 3e-6, 1e7, 0.025, 0.35, "CNAB2", dt)
    P = np.zeros((n_phi // 3 + 1, nc), complex)
    T = np.zeros_like(P)
    a = 1e-8 / np.max(np.abs(th))       # weakly nonlinear: products are O(1e-16)
    P[m], T[m] = a * p, a * th
    st.set_state(P, T, np.zeros(nc))
    K1, K2 = 20, 220
    for k in range(K2):
        st.step()
        if k + 1 == K1:
            z1 = np.vdot(T[m], st.y[1][m]) / np.vdot(T[m], T[m])
    z2 = np.vdot(T[m], st.y[1][m]) / np.vdot(T[m], T[m])
    est = np.log(z2 / z1) / ((K2 - K1) * dt)
    assert abs(est.real - lam.real) < 1e-5 * abs(lam)
    assert abs(est.imag - lam.imag) < 1e-5 * abs(lam)
    # the run stays on the eigenvector (other directions only from the splitting)
    assert np.linalg.norm(st.y[1][m] - z2 * T[m]) < 1e-5 * np.linalg.norm(st.y[1][m])


# -------------------------------------------------------------- schemes ----
@pytest.mark.parametrize("exact", [schemes.ars443_exact, schemes.bpr353_exact])
def test_dirk_tableau_is_third_order_and_stiffly_accurate(exact):
    aI, aE = exact()
    nu = 4
    c = [sum(r) for r in aI]
    assert c == [sum(r) for r in aE]                       # same abscissae
    bI, bE = aI[nu], aE[nu]                                 # stiffly accurate: b = last row
    assert aI[nu][nu] == aI[1][1] == aI[2][2] == aI[3][3]   # singly diagonal
    from fractions import Fraction as Fr
    for b, A in ((bI, aI), (bE, aE)):
        assert sum(b) == 1
        assert sum(bi * ci for bi, ci in zip(b, c)) == Fr(1, 2)
        assert sum(bi * ci * ci for bi, ci in zip(b, c)) == Fr(1, 3)
        assert sum(b[i] * A[i][j] * c[j] for i in range(5) for j in range(5)) == Fr(1, 6)
    # coupling conditions of the additive pair
    assert sum(bI[i] * aE[i][j] * c[j] for i in range(5) for j in range(5)) == Fr(1, 6)
    assert sum(bE[i] * aI[i][j] * c[j] for i in range(5) for j in range(5)) == Fr(1, 6)


def test_bpr353_term_counts_match_table1():
    """Table 1: BPR353 computes five implicit and three explicit terms per step
    (columns of the tableaux with a nonzero entry), ARS443 four implicit ones."""
    cols = lambda A: sum(1 for j in range(5) if any(A[i][j] != 0 for i in range(5)))
    aI, aE = schemes.bpr353_exact()
    assert (cols(aI), cols(aE)) == (5, 3)
    assert cols(schemes.ars443_exact()[0]) == 4


def _scalar_run(name, lam_i, lam_e, dt, T, exact_start=False):
    """y' = lam_i y + lam_e y with the scheme coefficients (Eqs. multistep1, dirks).
    exact_start: seed the multistep history with exact values (no start-up steps)."""
    n = int(round(T / dt))
    y = 1.0 + 0j
    if name in schemes.MULTISTEP:
        ys, es = [], []
        k0 = 0
        if exact_start:
            lam = lam_i + lam_e
            for k in (1, 2):
                yk = np.exp(-lam * k * dt)
                ys = ys + [yk]
                es = es + [lam_e * yk]
            k0 = 10
        for k in range(n):
            a, b0, bI, bE = schemes.multistep_coeffs(name, k + k0)
            ys = [y] + ys
            es = [lam_e * y] + es
            rhs = sum(aj * ys[j] for j, aj in enumerate(a))
            rhs += dt * sum(bj * lam_i * ys[j] for j, bj in enumerate(bI))
            rhs += dt * sum(bj * es[j] for j, bj in enumerate(bE))
            y = rhs / (1 - b0 * dt * lam_i)
        return y
    aI, aE = schemes.dirk_tableau(name)
    for _ in range(n):
        st = [y]
        for i in range(1, 5):
            r = y + dt * sum(aE[i, j] * lam_e * st[j] + aI[i, j] * lam_i * st[j] for j in range(i))
            st.append(r / (1 - aI[i, i] * dt * lam_i))
        y = st[4]
    return y


@pytest.mark.parametrize("name,order,exact_start", [
    ("CNAB2", 2, False), ("SBDF2", 2, True), ("SBDF3", 3, True), ("ARS443", 3, False), ("BPR353", 3, False),
    # with the lower-order start-up steps the global error of SBDF2/SBDF3 is that
    # of the first SBDF1 step, O(dt^2) (the paper notes the start-up penalty)
    ("SBDF2", 2, False), ("SBDF3", 2, False)])
def test_scheme_orders_on_scalar_imex_problem(name, order, exact_start):
    lam_i, lam_e, T = -3.0 + 1.0j, 0.5 - 2.0j, 1.0
    exact = np.exp((lam_i + lam_e) * T)
    dts = [0.02, 0.01, 0.005]
    err = [abs(_scalar_run(name, lam_i, lam_e, dt, T, exact_start) - exact) for dt in dts]
    slopes = [np.log2(err[i] / err[i + 1]) for i in range(2)]
    assert min(slopes) > order - 0.35, (slopes, err)
    assert max(slopes) < order + 0.5, (slopes, err)


# ---------------------------------------------------- linear diffusion ----
def _bessel_mode(ann, m):
    f = lambda k: jv(m, k * ann.s_o) * yv(m, k * ann.s_i) - jv(m, k * ann.s_i) * yv(m, k * ann.s_o)
    ks = np.linspace(0.5, 12, 400)
    v = f(ks)
    i = np.nonzero(np.sign(v[:-1]) != np.sign(v[1:]))[0][0]
    k = brentq(f, ks[i], ks[i + 1], xtol=1e-15)
    prof = lambda s: jv(m, k * s) * yv(m, k * ann.s_i) - jv(m, k * ann.s_i) * yv(m, k * s)
    return k, prof


@pytest.mark.parametrize("scheme,order", [("CNAB2", 2), ("ARS443", 3), ("BPR353", 3)])
def test_temperature_operator_decays_annulus_eigenmode(scheme, order):
    """With Psi = u_bar = 0 the temperature obeys d theta/dt = Delta theta/Pr; the
    Dirichlet annulus mode J_m(ks)Y_m(ks_i) - J_m(ks_i)Y_m(ks) decays as
    exp(-k^2 t/Pr).  Checks D^I, F^I_m, the tau rows and the stepper."""
    n_r, n_phi, m, Pr, T = 65, 12, 3, 1.0, 0.02
    ann = Annulus(0.35)
    k, prof = _bessel_mode(ann, m)
    s = ann.s_of_x(gauss_lobatto(n_r))
    nc = (2 * (n_r - 1)) // 3
    th0 = np.zeros((n_phi // 3 + 1, nc), complex)
    th0[m] = ch.analysis(prof(s), n_r)[:nc]
    errs = []
    for dt in (2e-3, 1e-3):
        st = IntegrationStepper(n_r, n_phi, 1e-3, 0.0, Pr, 0.35, scheme, dt)
        st.set_state(np.zeros_like(th0), th0, np.zeros(nc))
        for _ in range(int(round(T / dt))):
            st.step()
        ref = th0[m] * np.exp(-k * k * T / Pr)
        errs.append(np.linalg.norm(st.y[1][m] - ref) / np.linalg.norm(ref))
    assert errs[1] < 1e-4
    assert np.log2(errs[0] / errs[1]) > order - 0.3


# ------------------------------------------------------- bordered solve ----
def test_bordered_solve_equals_dense_solve_on_tau_systems():
    st = IntegrationStepper(65, 24, 1e-4, 1e6, 1.0, 0.35, "CNAB2", 1e-6)
    rng = np.random.default_rng(9)
    for m in (1, 3, 8):
        L = st.ops.lhs_psi(m, 0.5e-6)
        f = rng.standard_normal(L.shape[0]) + 1j * rng.standard_normal(L.shape[0])
        f[:4] = 0
        ref = np.linalg.solve(L, f)
        got = bordered_solve(L, f, 4)
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
        Lt = st.ops.lhs_theta(m, 0.5e-6)
        ft = f.copy(); ft[:2] = 0
        assert np.allclose(bordered_solve(Lt, ft, 2), np.linalg.solve(Lt, ft), rtol=1e-11, atol=0)


# -------------------------------------------------- nonlinear terms -------
def test_flux_divergences_match_analytic_evaluation():
    """N_omega = div(u omega), N_theta = div(u theta) + beta u_s theta and
    N_u = mean(u_s omega) evaluated symbolically from the definitions of Section 2
    and 3.2 (u_s = (h^2/s) dPsi/dphi, u_phi = u_bar - h^2 dPsi/ds + 3 s Psi,
    omega = (1/s) d(s u_bar)/ds - L_I Psi, beta = -s/h^2) agree with the oracle's
    grid values for low-degree fields."""
    sp = pytest.importorskip("sympy")
    n_r, n_phi = 33, 24
    ann = Annulus(0.35)
    st = IntegrationStepper(n_r, n_phi, 1e-3, 0.0, 1.0, 0.35, "CNAB2", 1e-4)
    nc, M = st.n_c, st.g.M
    x = gauss_lobatto(n_r)
    rng = np.random.default_rng(11)
    # Psi_1, Psi_2, theta_1, theta_2 and u_bar as low-degree polynomials in x
    cps = {m: rng.standard_normal(4) + 1j * rng.standard_normal(4) for m in (1, 2)}
    cts = {m: rng.standard_normal(4) + 1j * rng.standard_normal(4) for m in (1, 2)}
    cu = rng.standard_normal(4)
    psi = np.zeros((M, nc), complex)
    th = np.zeros((M, nc), complex)
    for m in (1, 2):
        psi[m, :4] = ch.plain_to_hat(cps[m], n_r)[:4]
        th[m, :4] = ch.plain_to_hat(cts[m], n_r)[:4]
    u = np.zeros(nc)
    u[:4] = ch.plain_to_hat(cu, n_r)[:4]
    _, _, _, parts = explicit_terms(st.g, psi, th, u, return_parts=True)

    s, phi = sp.symbols("s phi", real=True)
    X = (s - ann.b) / ann.a
    T = [sp.Integer(1), X, 2 * X ** 2 - 1, 4 * X ** 3 - 3 * X]

    def series(c):
        return sum(sp.nsimplify(0) + complex(c[i]) * T[i] for i in range(4))

    h2 = ann.s_o ** 2 - s ** 2
    Psi = sum(2 * sp.re(series(cps[m]) * sp.exp(sp.I * m * phi)) for m in (1, 2))
    Psi = sum(series(cps[m]) * sp.exp(sp.I * m * phi) + sp.conjugate(series(cps[m])) * sp.exp(-sp.I * m * phi)
              for m in (1, 2))
    Th = sum(series(cts[m]) * sp.exp(sp.I * m * phi) + sp.conjugate(series(cts[m])) * sp.exp(-sp.I * m * phi)
             for m in (1, 2))
    ub = sum(float(cu[i]) * T[i] for i in range(4))

    def lap(f):
        return sp.diff(f, s, 2) + sp.diff(f, s) / s + sp.diff(f, phi, 2) / s ** 2

    LI = lap(h2 * Psi) - sp.diff(s ** 2 * Psi, s) / s
    us = h2 / s * sp.diff(Psi, phi)
    up = ub - h2 * sp.diff(Psi, s) + 3 * s * Psi
    om = sp.diff(s * ub, s) / s - LI
    beta = -s / h2
    Nw = sp.diff(s * us * om, s) / s + sp.diff(up * om, phi) / s
    Nt = sp.diff(s * us * Th, s) / s + sp.diff(up * Th, phi) / s + beta * us * Th
    Nu_f = us * om
    fw = sp.lambdify((s, phi), Nw, "numpy")
    ft = sp.lambdify((s, phi), Nt, "numpy")
    fu = sp.lambdify((s, phi), Nu_f, "numpy")
    sk = ann.s_of_x(x)[1:]                      # outer wall excluded (beta singular there)
    P = 64
    ph = 2 * np.pi * np.arange(P) / P
    S, PH = np.meshgrid(sk, ph, indexing="ij")
    for f, key, mmax in ((fw, "Nw_grid", 4), (ft, "Nt_grid", 4)):
        vals = np.asarray(f(S, PH), dtype=complex).real
        spec = np.fft.fft(vals, axis=1)[:, :mmax + 1] / P
        got = parts[key][1:, :mmax + 1]
        assert np.allclose(got, spec, rtol=0, atol=1e-10 * np.abs(spec).max()), key
    vals = np.asarray(fu(S, PH), dtype=complex).real.mean(axis=1)
    assert np.allclose(parts["Nu_grid"][1:], vals, rtol=0, atol=1e-10 * np.abs(vals).max())


def test_tau_solve_is_accurate_against_extended_precision_refinement():
    """The oracle's solve of the streamfunction tau system (n_r = 257, E = 1e-5,
    dt = 1e-7) agrees with a solution iteratively refined with residuals in
    extended precision."""
    st = IntegrationStepper(257, 12, 1e-5, 1e8, 1.0, 0.35, "CNAB2", 1e-7)
    rng = np.random.default_rng(12)
    nc = st.n_c
    for m in (1, 3):
        L = st.ops.lhs_psi(m, 0.5e-7)
        c = np.zeros(nc, complex)
        c[:30] = (rng.standard_normal(30) + 1j * rng.standard_normal(30)) / (1 + np.arange(30)) ** 3
        f = st.ops.A(m) @ c
        f[:4] = 0
        x = st._solve_refined(st._factor(L), L, f)
        xr = x.copy()
        Ll = L.astype(np.clongdouble)
        for _ in range(4):
            r = (f.astype(np.clongdouble) - Ll @ xr.astype(np.clongdouble)).astype(complex)
            xr = xr + st._solve(st._factor(L), r)
        assert np.linalg.norm(x - xr) <= 1e-13 * np.linalg.norm(xr)


# --------------------------------------------------- implicit buoyancy ----
def test_implicit_buoyancy_solve_equals_the_coupled_dense_solve():
    """Section 4: with the buoyancy term implicit, the stage system of mode m is
    [A - g B, -g (Ra/Pr)(i m/s_o) C^I; 0, D - g F/Pr] (tau rows on top of each
    block) and the temperature is advanced first.  The stepper's block-ordered
    solve equals a dense solve of the coupled 2 N_c system."""
    n_r, n_phi, gamma, dt = 33, 24, 0.5, 3e-4
    st = IntegrationStepper(n_r, n_phi, 1e-3, 2e5, 0.7, 0.35, "CNAB2", dt, buoy_implicit=True)
    ops, nc, M = st.ops, st.n_c, st.g.M
    rng = np.random.default_rng(4)
    rp = (rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))) / (1 + np.arange(nc)) ** 2
    rt = (rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))) / (1 + np.arange(nc)) ** 2
    ru = rng.standard_normal(nc) / (1 + np.arange(nc)) ** 2
    psi, th, u = st.solve(gamma, (rp, rt, ru))
    gdt = gamma * dt
    for m in (1, 3, M - 1):
        L = np.zeros((2 * nc, 2 * nc), complex)
        L[:nc, :nc] = ops.lhs_psi(m, gdt)
        cpl = -gdt * (ops.Ra / ops.Pr) * (1j * m / ops.ann.s_o) * ops.C
        cpl[:4] = 0.0
        L[:nc, nc:] = cpl
        L[nc:, nc:] = ops.lhs_theta(m, gdt)
        b = np.concatenate([rp[m], rt[m]])
        b[:4] = 0.0
        b[nc:nc + 2] = 0.0
        x = np.linalg.solve(L, b)
        ref = np.concatenate([psi[m], th[m]])
        assert np.linalg.norm(ref - x) <= 1e-9 * np.linalg.norm(x)


def test_implicit_buoyancy_run_keeps_second_order_at_the_eigenvalue():
    """The eigenmode run of test_dns_from_eigenmode_grows_at_the_eigenvalue with
    the buoyancy implicit: CNAB2 still converges to the eigenvalue at second order."""
    n_r, n_phi, m = 65, 48, 12
    nc = (2 * (n_r - 1)) // 3
    lam, p, th = leading_mode(3e-6, 0.025, 1e7, 0.35, m, nc, n_r=n_r, guess=615.0 - 9537.0j)
    errs = []
    for dt, K1, K2 in ((4e-7, 10, 110), (2e-7, 20, 220)):
        st = IntegrationStepper(n_r, n_phi, 3e-6, 1e7, 0.025, 0.35, "CNAB2", dt, buoy_implicit=True)
        P = np.zeros((n_phi // 3 + 1, nc), complex)
        T = np.zeros_like(P)
        a = 1e-8 / np.max(np.abs(th))
        P[m], T[m] = a * p, a * th
        st.set_state(P, T, np.zeros(nc))
        for k in range(K2):
            st.step()
            if k + 1 == K1:
                z1 = np.vdot(T[m], st.y[1][m]) / np.vdot(T[m], T[m])
        z2 = np.vdot(T[m], st.y[1][m]) / np.vdot(T[m], T[m])
        errs.append(abs(np.log(z2 / z1) / ((K2 - K1) * dt) - lam) / abs(lam))
    assert errs[1] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 5.0
