"""Pins of the oracle's Chebyshev-collocation formulation (Section 3.1): the
paper's onset eigenvalue, decay of annulus eigenmodes, a manufactured solve, and
agreement with the independently pinned Chebyshev-integration formulation."""
import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle.collocation import CollocationStepper, leading_eigenvalue_collocation
from oracle.explicit import radial_fields
from oracle.geometry import Annulus, gauss_lobatto
from oracle.stepper import IntegrationStepper
from tests.test_oracle_physics import _bessel_mode


def test_collocation_onset_eigenvalue_matches_the_paper():
    """Table 3 (without Ekman pumping): E = 3e-6, Pr = 0.025, Ra = 1e7, eta = 0.35,
    m = 12: tau = 6.149994e2, omega_d = -9.536952e3.  Fixes A^C, B^C, C^C (with
    the sign of dbeta/ds + beta/s taken from the definition of L_beta), the
    buoyancy and conduction couplings and the boundary rows."""
    lam = leading_eigenvalue_collocation(3e-6, 0.025, 1e7, 0.35, 12, 129, guess=615.0 - 9537.0j)
    assert abs(lam.real - 614.9994) < 1e-6 * 615.0
    assert abs(lam.imag - (-9536.952)) < 1e-6 * 9537.0


def _decay_errors(field, scheme, m, rate, prof, n_r=49, T=0.02, dts=(2e-3, 1e-3)):
    ann = Annulus(0.35)
    s = ann.s_of_x(gauss_lobatto(n_r))
    n_phi = 3 * max(4, m + 1)
    M = n_phi // 3 + 1
    f0 = ch.analysis(prof(s), n_r)
    errs = []
    for dt in dts:
        st = CollocationStepper(n_r, n_phi, 1e-3, 0.0, 1.0, 0.35, scheme, dt)
        z = np.zeros((M, n_r), complex)
        th = z.copy()
        u = np.zeros(n_r)
        if field == "theta":
            th[m] = f0
        else:
            u = f0.copy()
        st.set_state(z, z.copy(), th, u)
        for _ in range(int(round(T / dt))):
            st.step()
        got = st.y[2][m] if field == "theta" else st.y[3]
        ref = f0 * np.exp(-rate * T)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return errs


@pytest.mark.parametrize("scheme,order", [("CNAB2", 2), ("ARS443", 3)])
def test_collocation_temperature_decays_annulus_eigenmode(scheme, order):
    """psi = u_bar = 0: d theta/dt = Delta theta/Pr; the Dirichlet mode
    J_m(ks)Y_m(ks_i) - J_m(ks_i)Y_m(ks) decays as exp(-k^2 t) (Pr = 1)."""
    ann = Annulus(0.35)
    k, prof = _bessel_mode(ann, 3)
    errs = _decay_errors("theta", scheme, 3, k * k, prof)
    assert errs[1] < 1e-4
    assert np.log2(errs[0] / errs[1]) > order - 0.3


@pytest.mark.parametrize("scheme,order", [("CNAB2", 2), ("SBDF3", 2)])
def test_collocation_zonal_flow_decays_annulus_eigenmode(scheme, order):
    """psi = theta = 0: d u/dt = Delta u - u/s^2 (Eq. uphi without pumping); the
    no-slip mode J_1(ks)Y_1(ks_i) - J_1(ks_i)Y_1(ks) decays as exp(-k^2 t)."""
    ann = Annulus(0.35)
    k, prof = _bessel_mode(ann, 1)
    errs = _decay_errors("u", scheme, 1, k * k, prof)
    assert errs[1] < 1e-4
    assert np.log2(errs[0] / errs[1]) > order - 0.3


def test_collocation_solve_recovers_manufactured_solution():
    """psi = (1-x^2)^2 p(x) meets the four boundary conditions; omega takes -L_beta psi
    at the interior points and free values at the walls.  Building the right-hand
    side from the operators and solving must give both fields back."""
    n_r, m, gdt = 33, 5, 3e-4
    st = CollocationStepper(n_r, 24, 1e-4, 0.0, 1.0, 0.35, "CNAB2", 2 * gdt)
    o = st.ops
    x = gauss_lobatto(n_r)
    rng = np.random.default_rng(4)
    p = np.polynomial.chebyshev.chebval(x, rng.standard_normal(8) + 1j * rng.standard_normal(8))
    psi = ch.analysis((1 - x * x) ** 2 * p, n_r)
    w = -(o.C(m) @ psi)
    w[0], w[-1] = 0.7 - 0.2j, -1.1 + 0.4j
    w_hat = ch.analysis(w, n_r)
    L = o.lhs_wpsi(m, gdt)
    rhs = (L @ np.concatenate([w_hat, psi]))[:n_r]
    y = tuple(np.zeros((st.M, n_r), complex) for _ in range(3)) + (np.zeros(n_r),)
    R = list(y)
    R[0] = R[0].copy()
    R[0][m] = rhs
    w_s, psi_s, _, _ = st.solve(0.5, tuple(R))
    assert np.linalg.norm(psi_s[m] - psi) < 1e-12 * np.linalg.norm(psi)
    assert np.linalg.norm(w_s[m] - w_hat) < 1e-10 * np.linalg.norm(w_hat)


def _paired_runs(n_r, scheme, dt, nsteps, n_phi=24, E=1e-3, Ra=1e5, amp=1e-2, seed=3):
    """The same smooth initial state in both formulations: Psi = (1+x)^2 (1-x)^4 p
    (Psi = dPsi/ds = 0 at s_i, Psi = ... = d^3Psi/ds^3 = 0 at s_o), psi = h^2 Psi,
    theta and u_bar vanishing at both walls."""
    rng = np.random.default_rng(seed)
    x = gauss_lobatto(n_r)
    nc = (2 * (n_r - 1)) // 3
    M = n_phi // 3 + 1

    def poly(K=6):
        c = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) / np.arange(1, K + 1) ** 2
        return np.polynomial.chebyshev.chebval(x, c)

    Psig = np.zeros((n_r, M), complex)
    thg = np.zeros((n_r, M), complex)
    for m in range(1, 4):
        Psig[:, m] = amp * (1 + x) ** 2 * (1 - x) ** 4 * poly()
    for m in range(0, 4):
        thg[:, m] = amp * (1 - x * x) * poly()
    thg[:, 0] = thg[:, 0].real
    ug = amp * (1 - x * x) * poly().real
    st = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt)
    st.set_state(ch.analysis(Psig, n_r)[:nc].T, ch.analysis(thg, n_r)[:nc].T, ch.analysis(ug, n_r)[:nc])
    cs = CollocationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt)
    psih = ch.analysis(st.g.h2[:, None] * Psig, n_r).T
    cs.set_state(cs.vorticity_from_psi(psih), psih, ch.analysis(thg, n_r).T, ch.analysis(ug, n_r))

    def differences():
        v, uphi, om, th = radial_fields(st.g, *st.y)
        us = (st.g.h2 / st.g.s)[:, None] * v
        us_c, up_c, om_c, th_c = cs.grid_state()
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(a)
        return dict(us=rel(us, us_c), uphi=rel(uphi, up_c), omega=rel(om, om_c), theta=rel(th, th_c))

    d0 = differences()
    for _ in range(nsteps):
        st.step()
        cs.step()
    return d0, differences()


def test_collocation_and_integration_formulations_agree():
    """Both formulations discretise the same equations (no Ekman pumping): from the
    same smooth state the initial fields coincide to rounding, and after 100 SBDF2
    steps they differ by a spatial truncation error that falls by orders of
    magnitude from n_r = 33 to 65.  (With CNAB2 the undamped stiff modes of the
    wall layers keep a resolution-independent difference in omega at the walls.)"""
    d0, d33 = _paired_runs(33, "SBDF2", 2e-4, 100)
    assert max(d0.values()) < 1e-10
    _, d65 = _paired_runs(65, "SBDF2", 2e-4, 100)
    for f in ("us", "uphi", "theta"):
        assert d65[f] < 1e-4, (f, d65)
        assert d65[f] < d33[f] / 10, (f, d33, d65)
    assert d65["omega"] < d33["omega"] / 5


def test_collocation_implicit_buoyancy_solve_equals_the_coupled_dense_solve():
    """Section 4 in the collocation formulation: the stage system couples the
    vorticity rows to the new temperature through -g(-(Ra/Pr)(i m/s_o)) T theta;
    the block-ordered solve (temperature first) equals a dense solve of the
    coupled 3N system."""
    from oracle.collocation import CollocationStepper
    N, n_phi, gamma, dt = 17, 24, 0.5, 2e-4
    st = CollocationStepper(N, n_phi, 1e-3, 2e5, 0.7, 0.35, "CNAB2", dt, buoy_implicit=True)
    o, M = st.ops, st.M
    rng = np.random.default_rng(8)
    rw = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    rt = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    ru = rng.standard_normal(N)
    w, psi, th, u = st.solve(gamma, (rw, np.zeros_like(rw), rt, ru))
    gdt = gamma * dt
    for m in (1, 4, M - 1):
        L = np.zeros((3 * N, 3 * N), complex)
        L[:2 * N, :2 * N] = o.lhs_wpsi(m, gdt)
        cpl = -gdt * (-(o.Ra / o.Pr) * (1j * m / o.ann.s_o)) * o.T
        cpl[0] = cpl[N - 1] = 0.0
        L[:N, 2 * N:] = cpl
        L[2 * N:, 2 * N:] = o.lhs_dir(o.Lt(m), gdt)
        b = np.zeros(3 * N, complex)
        b[1:N - 1] = rw[m, 1:N - 1]
        b[2 * N + 1:3 * N - 1] = rt[m, 1:N - 1]
        x = np.linalg.solve(L, b)
        ref = np.concatenate([w[m], psi[m], th[m]])
        assert np.linalg.norm(ref - x) <= 1e-9 * np.linalg.norm(x)
