"""Discrete adjoint of the Chebyshev-integration time step (Sections 3.2 and 4):
reverse-mode derivative of a time-averaged Nusselt number through CNAB2 steps,
with respect to the initial state and to Ra.

Test infrastructure only (see the package docstring).

Inner product: the real part of the Hermitian product over the stored arrays,
<a, b> = Re sum conj(a) b (coefficients m = 0..N_m, n < N_c).  Every map below is
real-linear; the adjoint X* of each satisfies <l, X d> = <X* l, d>.  For a
complex-linear map with matrix X this is the conjugate transpose.

Forward (stepper.IntegrationStepper, CNAB2 with the start-up rule):
    r_0 = A y_0 + dt E(y_0),   r_n = A y_n + dt (3/2 E(y_n) - 1/2 E(y_{n-1})),
    y_{n+1} = S^{-1} P r_n,
with A = Mass + (dt/2) Lin (per field), S the tau system of weight dt/2 and P the
projection that zeroes its tau rows.  For J = sum_{n=1..K} j_n(y_n):
    lambda_K = g_K,   rho_n = P S^{-H} lambda_{n+1},
    lambda_n = g_n + A^H rho_n + J_E(y_n)* [dt (c_n rho_n - 1/2 rho_{n+1})],
with c_0 = 1, c_n = 3/2 and rho_K = 0; lambda_0 = dJ/dy_0 and
dJ/dRa = sum_n < dt (c_n rho_n - 1/2 rho_{n+1}), dE/dRa(y_n) >.

J_E(y)* is the adjoint of the explicit stage of ``explicit.explicit_terms``, taken
backwards through its steps: the integrated right-hand sides (C^I, D^I, G^I
transposed, conjugated where complex), truncation (zero padding), Eq. icheb
(its transpose), the flux divergences, the azimuthal transforms (Eq. ifft and
Eq. fft transposed) with the product rule on the grid, and the radial fields
(Chebyshev synthesis and derivatives transposed).  Only the real parts of the
m = 0 spectra enter the grid fields (the transforms are real), and the adjoint
keeps that.
"""
import numpy as np

from . import chebyshev as ch
from . import fourier as fo


def _radial_mats(g):
    """Real matrices (N_r x N_c) mapping f_hat to grid values of f, f', f''."""
    n_r, n_c = g.n_r, g.n_c
    P = np.zeros((n_r, n_c))
    P[:n_c, :n_c] = np.diag(ch.hat_scale(n_r, n_c))
    S0 = g.T @ P
    S1 = g.T @ (g.Dn @ P)
    S2 = g.T @ (g.Dn @ (g.Dn @ P))
    return S0, S1, S2


def _analysis_matrix(n_r):
    return ch.analysis(np.eye(n_r), n_r)       # f_hat = A f


def _radial_derivative_matrix(g):
    """Grid -> grid d/ds of the interpolant (``explicit.radial_derivative``)."""
    A = _analysis_matrix(g.n_r)
    return g.T @ (g.Dn @ ch.hat_to_plain(A, g.n_r))


def _to_grid_adjoint(fbar, n_m):
    """Adjoint of fourier.to_grid: real grid adjoint (..., n_phi) -> spectra
    (..., n_m + 1): m = 0 gets sum_j (real), m >= 1 gets 2 sum_j fbar e^{-i m phi}."""
    R = np.fft.rfft(fbar, axis=-1)[..., :n_m + 1]
    out = 2.0 * R
    out[..., 0] = R[..., 0].real
    return out


def _to_spec_adjoint(Pbar, n_phi):
    """Adjoint of fourier.to_spec: spectra (..., n_m + 1) -> real grid adjoint
    fbar_j = (1/n_phi) Re sum_m Pbar_m e^{i m phi_j}."""
    n_m = Pbar.shape[-1] - 1
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    E = np.exp(1j * np.outer(np.arange(n_m + 1), phi))
    return np.real(np.tensordot(Pbar, E, axes=(-1, 0))) / n_phi


def explicit_adjoint(g, psi_hat, theta_hat, u_hat, e_bar):
    """J_E(y)* applied to e_bar = (ebar_psi, ebar_theta, ebar_u): returns the
    adjoint (psi_bar, theta_bar, u_bar) with the shapes of the state, and the
    derivative dE/dRa of the explicit terms (for the Ra gradient)."""
    from .explicit import radial_fields
    ops = g.ops
    n_r, nc, M, n_phi = g.n_r, g.n_c, g.M, g.n_phi
    ep, et, eu = (np.array(x) for x in e_bar)
    ep = ep.astype(complex)
    ep[0] = 0.0
    m = g.m[:, None]
    s = g.s[:, None]
    h2 = g.h2[:, None]
    # e_psi = C^I (buoy + Nw_hat), buoy = (Ra/Pr)(i m/s_o) theta_hat
    q = (ops.C.T @ ep.T).T                                    # adjoint of (buoy + Nw_hat)
    theta_bar = np.conj((ops.Ra / ops.Pr) * (1j * m / ops.ann.s_o)) * q
    Nw_hat_bar = q
    # e_theta = -D^I Nt_hat - tc i m G^I psi_hat
    Nt_hat_bar = -(ops.D.T @ et.T).T
    psi_bar = np.conj(-ops.tc_coef * 1j * m) * (ops.G.T @ et.T).T
    # e_u = -D^I Re(Nu_hat)
    Nu_hat_bar = -(ops.D.T @ eu)
    # truncation and Eq. icheb: hat = (A grid)[:nc]
    A = _analysis_matrix(n_r)
    pad = lambda x: np.concatenate([x, np.zeros((n_r - nc,) + x.shape[1:], x.dtype)])
    Nw_bar = A.T @ pad(Nw_hat_bar.T)                          # (n_r, M)
    Nt_bar = A.T @ pad(Nt_hat_bar.T)
    Nu_bar = A.T @ pad(Nu_hat_bar)
    # flux divergences (explicit.nonlinear_grid)
    Dg = _radial_derivative_matrix(g)
    vw_bar = h2 * (Dg.T @ (Nw_bar / s))
    uw_bar = np.conj(1j * m.T) * Nw_bar / s
    vt_bar = h2 * (Dg.T @ (Nt_bar / s)) - Nt_bar
    ut_bar = np.conj(1j * m.T) * Nt_bar / s
    vw_bar[:, 0] += (g.h2 / g.s) * Nu_bar.real
    # azimuthal products: p = f_a f_b on the grid, spectra by Eq. fft (to_spec)
    v, uphi, omega, theta = radial_fields(g, psi_hat, theta_hat, u_hat)
    vg, ug, wg, tg = (fo.to_grid(f, n_phi) for f in (v, uphi, omega, theta))
    pvw, puw, pvt, put = (_to_spec_adjoint(x, n_phi) for x in (vw_bar, uw_bar, vt_bar, ut_bar))
    vgb = wg * pvw + tg * pvt
    ugb = wg * puw + tg * put
    wgb = vg * pvw + ug * puw
    tgb = vg * pvt + ug * put
    v_bar, uphi_bar, omega_bar, th_grid_bar = (_to_grid_adjoint(x, g.n_m) for x in (vgb, ugb, wgb, tgb))
    # radial fields (explicit.radial_fields); m = 0 uses only real parts
    S0, S1, S2 = _radial_mats(g)
    v_bar[:, 0] = 0.0
    a0 = np.conj(1j * m.T) * v_bar + 3 * s * uphi_bar + (6 + m.T ** 2 * h2 / s ** 2) * omega_bar
    a1 = -h2 * uphi_bar - (h2 / s - 5 * s) * omega_bar
    a2 = -h2 * omega_bar
    pb = S0.T @ a0 + S1.T @ a1 + S2.T @ a2                     # (nc, M)
    pb[:, 0] = 0.0
    psi_bar = psi_bar + pb.T
    psi_bar[0] = 0.0
    theta_bar = theta_bar + (S0.T @ th_grid_bar).T
    ub = S0.T @ uphi_bar[:, 0].real + S1.T @ omega_bar[:, 0].real + S0.T @ (omega_bar[:, 0].real / g.s)
    u_bar = ub
    # dE/dRa: only the buoyancy term of e_psi
    dE_dRa = (ops.C @ ((1.0 / ops.Pr) * (1j * m / ops.ann.s_o) * theta_hat).T).T
    dE_dRa[0] = 0.0
    return (psi_bar, theta_bar, u_bar), dE_dRa


def nusselt_gradient(g):
    """Gradient of Nu - 1 = (d theta_0/ds)(s_o)/(dT_c/ds)(s_o) with respect to
    theta_hat (only the real parts of the m = 0 coefficients enter):
    d/ds at s_o of sum_n c_n T_n is (1/a) sum_n n^2 c_n, c_n = C w_n theta_hat_0n."""
    ann = g.ops.ann
    nc = g.n_c
    n = np.arange(nc)
    w = ch.hat_scale(g.n_r, nc) * n ** 2 / ann.a / ann.dTc_ds(ann.s_o)
    gt = np.zeros((g.M, nc), complex)
    gt[0] = w
    return gt


def nusselt_minus_one(g, theta_hat):
    return float(np.sum(nusselt_gradient(g)[0].real * theta_hat[0].real))


def adjoint_cnab2(stepper, y0, K):
    """J = (1/K) sum_{n=1..K} (Nu_n - 1) after K CNAB2 steps from y0 = (psi_hat,
    theta_hat, u_hat).  Returns (J, dJ/dy0 as (psi_bar, theta_bar, u_bar), dJ/dRa)."""
    if stepper.scheme != "CNAB2":
        raise ValueError("the adjoint is written for CNAB2")
    g = stepper.g
    ops = stepper.ops
    dt = stepper.dt
    gN = nusselt_gradient(g) / K
    stepper.set_state(*y0)
    ys = [tuple(np.array(x) for x in stepper.y)]
    J = 0.0
    for _ in range(K):
        stepper.step()
        ys.append(tuple(np.array(x) for x in stepper.y))
        J += nusselt_minus_one(g, stepper.y[1]) / K
    gamma = 0.5
    lp, lt, lu_ = stepper.lu(gamma)

    def s_inv_h(lam):
        """P S^{-H} lam for the three fields."""
        lpsi, lth, lu = lam
        rp = np.zeros_like(lpsi)
        for mm in range(1, g.M):
            L = lp[mm][1]
            rp[mm] = np.linalg.solve(L.conj().T, lpsi[mm])
        rt = np.stack([np.linalg.solve(lt[mm][1].conj().T, lth[mm]) for mm in range(g.M)])
        ru = np.linalg.solve(lu_[1].T, lu)
        rp[:, :4] = 0.0
        rt[:, :2] = 0.0
        ru[:2] = 0.0
        return rp, rt, ru

    def a_h(rho):
        """(Mass + (dt/2) Lin)^H rho."""
        rp, rt, ru = rho
        out_p = np.zeros_like(rp)
        for mm in range(1, g.M):
            A = ops.A(mm) + 0.5 * dt * ops.B(mm)
            out_p[mm] = A.conj().T @ rp[mm]
        out_t = np.stack([(ops.D + 0.5 * dt * ops.F(mm) / ops.Pr).T @ rt[mm] for mm in range(g.M)])
        out_u = (ops.D + 0.5 * dt * ops.Ez).T @ ru
        return out_p, out_t, out_u

    zero = tuple(np.zeros_like(x) for x in ys[0])
    lam = (zero[0], gN.copy(), zero[2])           # lambda_K
    rho_next = zero
    dRa = 0.0
    for n in range(K - 1, -1, -1):
        rho = s_inv_h(lam)
        c = 1.0 if n == 0 else 1.5
        w = tuple(dt * (c * a - 0.5 * b) for a, b in zip(rho, rho_next))
        (jp, jt, ju), dE = explicit_adjoint(g, *ys[n], w)
        ap, at, au = a_h(rho)
        dRa += float(np.real(np.vdot(w[0], dE)))
        gn = gN if n >= 1 else np.zeros_like(gN)
        lam = (ap + jp, gn + at + jt, au + ju)
        rho_next = rho
    return J, lam, dRa
