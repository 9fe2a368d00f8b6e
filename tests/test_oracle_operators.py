"""Pins of the oracle's Chebyshev-integration operators (Section 3.2, Eqs. psi_int,
uphi_int, temp_int; Appendix B) against exact rational arithmetic, the paper's
bandwidths, its closed form for E^I and its Galerkin coefficients."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle.operators import IntegrationOperators, bc_rows_plain

ETA = Fr(7, 20)          # radius ratio 0.35 exactly
S_O = 1 / (1 - ETA)      # 20/13
S_I = ETA / (1 - ETA)    # 7/13
A = (S_O - S_I) / 2      # 1/2
B = (S_O + S_I) / 2      # 27/26


# --- exact Laurent polynomials in s: dict power -> Fraction -----------------
def padd(*ps):
    out = {}
    for p in ps:
        for k, v in p.items():
            out[k] = out.get(k, 0) + v
    return {k: v for k, v in out.items() if v != 0}


def pmul(p, q):
    out = {}
    for i, a in p.items():
        for j, b in q.items():
            out[i + j] = out.get(i + j, 0) + a * b
    return {k: v for k, v in out.items() if v != 0}


def pscale(p, c):
    return {k: c * v for k, v in p.items()}


def pder(p):
    return {k - 1: k * v for k, v in p.items() if k != 0}


def pint(p):
    assert all(k >= 0 for k in p)
    return {k + 1: v / (k + 1) for k, v in p.items()}


S1 = {1: Fr(1)}
H2 = {0: S_O * S_O, 2: Fr(-1)}


def lap(f, mu):
    """Delta f = f'' + f'/s - mu f/s^2 on one Fourier mode (mu = m^2)."""
    return padd(pder(pder(f)), pmul({-1: Fr(1)}, pder(f)), pscale(pmul({-2: Fr(1)}, f), -mu))


def L_I(f, mu):
    """L_I f = Delta(h^2 f) - (1/s) d/ds (s^2 f)   (definition in Section 3.2)."""
    return padd(lap(pmul(H2, f), mu), pscale(pmul({-1: Fr(1)}, pder(pmul({2: Fr(1)}, f))), -1))


def cheb_T_in_s(n):
    """T_n(x) with x = (s - B)/A as an exact polynomial in s."""
    x = {0: -B / A, 1: 1 / A}
    t0, t1 = {0: Fr(1)}, x
    if n == 0:
        return t0
    for _ in range(n - 1):
        t0, t1 = t1, padd(pscale(pmul(x, t1), 2), pscale(t0, -1))
    return t1


def s_poly_to_plain_cheb(p, K):
    """Exact Chebyshev coefficients (in x) of a polynomial in s, length K."""
    # to power basis in x: s = A x + B
    deg = max(p)
    xs = [{0: Fr(1)}]
    for _ in range(deg):
        xs.append(pmul(xs[-1], {0: B, 1: A}))
    px = {}
    for k, v in p.items():
        px = padd(px, pscale(xs[k], v))
    # power -> Chebyshev by peeling the top degree
    c = [Fr(0)] * max(K, deg + 1)
    rem = dict(px)
    Tx = [{0: Fr(1)}, {1: Fr(1)}]
    while len(Tx) <= deg:
        Tx.append(padd(pscale(pmul({1: Fr(1)}, Tx[-1]), 2), pscale(Tx[-2], -1)))
    for d in range(deg, -1, -1):
        lead = rem.get(d, 0)
        if lead == 0:
            continue
        coef = lead / Tx[d][d]
        c[d] = coef
        rem = padd(rem, pscale(Tx[d], -coef))
    return c[:K]


@pytest.mark.parametrize("mu", [0, 1, 4])
def test_integrated_operators_equal_exact_integrals(mu):
    """Rows k >= q of A^I, B^I, C^I applied to T_n equal the Chebyshev coefficients
    of int^q s^q (operator T_n) computed in exact rational arithmetic."""
    n_r, n_c = 21, 12
    ops = IntegrationOperators(n_r, n_c, 0.35, 1e-3, 1.0, 1.0)
    sc = ch.hat_scale(n_r, n_c)
    A_or = (ops.A0 + mu * ops.A2) / sc[None, :]
    B_or = (ops.B0 + mu * ops.B2 + mu * mu * ops.B4) / sc[None, :]
    C_or = ops.C / sc[None, :]
    F_or = (ops.F0 + mu * ops.F2) / sc[None, :]
    for n in range(n_c):
        f = cheb_T_in_s(n)
        for name, op_f, q, mat in (
            ("A", pmul({4: Fr(1)}, L_I(f, mu)), 4, A_or),
            ("B", pmul({4: Fr(1)}, lap(L_I(f, mu), mu)), 4, B_or),
            ("C", pmul({4: Fr(1)}, f), 4, C_or),
            ("F", pmul({2: Fr(1)}, lap(f, mu)), 2, F_or),
        ):
            if not op_f:
                ref = np.zeros(n_c)
            else:
                assert min(op_f) >= 0, name
                g = op_f
                for _ in range(q):
                    g = pint(g)
                ref = np.array([float(v) for v in s_poly_to_plain_cheb(g, n_c)])
            got = mat[:, n]
            scale = max(np.abs(ref[q:]).max(), np.abs(mat[q:]).max())  # operator magnitude
            assert np.allclose(got[q:], ref[q:], rtol=0, atol=1e-13 * scale), (name, n)


def test_bandwidths_match_the_paper():
    """A^I, C^I: 17; B^I without the (2/E) i m term: 13; D^I: 9; E^I, F^I: 5
    (bandwidths stated in Section 3.2)."""
    ops = IntegrationOperators(65, 42, 0.35, 1e-4, 1.0, 1e6)

    def width(M, q):
        r = np.arange(M.shape[0])[:, None]
        c = np.arange(M.shape[1])[None, :]
        nz = (np.abs(M) > 1e-14 * np.abs(M).max()) & (r >= q)
        d = (c - r)[nz]
        return d.max() - d.min() + 1

    assert width(ops.A(5), 4) == 17
    assert width(ops.B0 + 25 * ops.B2 + 625 * ops.B4, 4) == 13
    assert width(ops.C, 4) == 17
    assert width(ops.D, 2) == 9
    assert width(ops.Ez, 2) == 5
    assert width(ops.F(5), 2) == 5
    # the assembled streamfunction matrix: 4 full tau rows above +-8 bands
    L = ops.lhs_psi(5, 1e-3)
    assert (np.abs(L[:4, 3:]) > 0).all()          # dense rows (T_0..T_2 vanish in f''')
    assert width(L[4:], 0) == 17


def test_zonal_operator_is_the_closed_form_of_the_paper():
    """E^I = s^2 - 3 int s (Section 3.2, below Eq. temp_int)."""
    n_r, n_c = 33, 21
    ops = IntegrationOperators(n_r, n_c, 0.35, 1e-3, 1.0, 1.0)
    a, b = ops.ann.a, ops.ann.b
    K = n_c + 10
    X = ch.xmul_matrix(K)
    J = ch.int_matrix(K)
    I = np.eye(K)
    S = a * X + b * I
    E_ref = (S @ S - 3 * a * (J @ S))[:n_c, :n_c] * ch.hat_scale(n_r, n_c)[None, :]
    assert np.allclose(ops.Ez[2:], E_ref[2:], atol=1e-14)


def test_galerkin_basis_of_appendix_b_satisfies_the_tau_rows():
    """gamma_i^n of Appendix B make phi_n = sum_i gamma_i T_{n+i} satisfy the four
    streamfunction tau rows (Eqs. bcs_coll_dirichlet, bcs_coll_neumann, bc_d3psi_coll)."""
    K = 30
    rows = [bc_rows_plain(K, k) for k in ("dir_o", "dir_i", "d3_o", "neu_i")]
    for n in range(0, K - 5):
        den = 2 * n ** 4 + 20 * n ** 3 + 78 * n ** 2 + 140 * n + 95
        g = np.zeros(K)
        g[n] = 1.0
        g[n + 1] = 8 * (n + 1) * (n * n + 4 * n + 5) / den
        g[n + 2] = -2 * (n + 2) * (2 * n ** 4 + 16 * n ** 3 + 58 * n ** 2 + 104 * n + 75) / ((n + 3) * den)
        g[n + 3] = -8 * (n + 1) * (n * n + 4 * n + 5) / den
        g[n + 4] = (n + 1) * (2 * n ** 4 + 12 * n ** 3 + 30 * n ** 2 + 36 * n + 15) / ((n + 3) * den)
        for r in rows:
            assert abs(r @ g) <= 1e-12 * np.abs(r * g).sum()


def test_tau_rows_evaluate_the_boundary_values():
    """The tau rows are f(1), f(-1), f'''(1), f'(-1) on plain coefficients."""
    import numpy.polynomial.chebyshev as npc
    rng = np.random.default_rng(7)
    c = rng.standard_normal(15)
    assert np.isclose(bc_rows_plain(15, "dir_o") @ c, npc.chebval(1.0, c))
    assert np.isclose(bc_rows_plain(15, "dir_i") @ c, npc.chebval(-1.0, c))
    assert np.isclose(bc_rows_plain(15, "neu_i") @ c, npc.chebval(-1.0, npc.chebder(c)))
    assert np.isclose(bc_rows_plain(15, "d3_o") @ c, 15 * npc.chebval(1.0, npc.chebder(c, 3)))
