"""Pins of the oracle's transforms (Section 3, Eqs. fft, ifft, cheb, icheb, int1)
against definitions and independent library routines."""
import numpy as np
import numpy.polynomial.chebyshev as npc

from oracle import chebyshev as ch
from oracle import fourier as fo
from oracle.geometry import gauss_lobatto


def test_tmat_is_cosine_of_gauss_lobatto_angle():
    # T_n(x_k) = cos(n arccos x_k) = cos(pi n k/(N_r-1))  (Section 3)
    n_r = 17
    x = gauss_lobatto(n_r)
    T = ch.tmat(n_r, n_r)
    assert np.allclose(T, np.cos(np.outer(np.arccos(np.clip(x, -1, 1)), np.arange(n_r))), atol=1e-14)


def test_cheb_pair_is_involution():
    # Eqs. cheb/icheb with C = sqrt(2/(N_r-1)) and double primes: icheb(cheb(f)) = f
    rng = np.random.default_rng(0)
    for n_r in (9, 33, 65):
        f = rng.standard_normal((n_r, 3)) + 1j * rng.standard_normal((n_r, 3))
        assert np.allclose(ch.synthesis(ch.analysis(f, n_r), n_r), f, atol=1e-13)
        assert np.allclose(ch.analysis(ch.synthesis(f, n_r), n_r), f, atol=1e-13)


def test_analysis_recovers_polynomial_coefficients_exactly():
    # samples of a polynomial of degree < N_r: plain coefficients recovered
    n_r = 33
    rng = np.random.default_rng(1)
    c = rng.standard_normal(20)
    x = gauss_lobatto(n_r)
    vals = npc.chebval(x, c)
    got = ch.hat_to_plain(ch.analysis(vals, n_r), n_r)
    assert np.allclose(got[:20], c, atol=1e-13)
    assert np.allclose(got[20:], 0.0, atol=1e-13)


def test_diff_matrix_matches_numpy_chebder():
    rng = np.random.default_rng(2)
    c = rng.standard_normal(25)
    D = ch.diff_matrix(25)
    ref = npc.chebder(c)
    assert np.allclose((D @ c)[:24], ref, atol=1e-12)
    assert abs((D @ c)[24]) < 1e-15


def test_derivative_at_walls():
    # T_n'(+-1) = (+-1)^(n+1) n^2  (Neumann tau rows of Section 3.1)
    K = 12
    D = ch.diff_matrix(K)
    for n in range(K):
        e = np.zeros(K); e[n] = 1
        d = D @ e
        assert np.isclose(npc.chebval(1.0, d), n * n)
        assert np.isclose(npc.chebval(-1.0, d), (-1) ** (n + 1) * n * n)


def test_int_matrix_inverts_derivative_above_row_zero():
    # Eq. int1: integrating the derivative returns f up to the constant (row 0)
    rng = np.random.default_rng(3)
    c = np.zeros(30); c[:20] = rng.standard_normal(20)
    J = ch.int_matrix(30); D = ch.diff_matrix(30)
    assert np.allclose((J @ (D @ c))[1:], c[1:], atol=1e-13)
    ref = npc.chebint(c[:20])
    assert np.allclose((J @ c)[1:21], ref[1:21], atol=1e-14)


def test_xmul_matches_numpy():
    rng = np.random.default_rng(4)
    c = np.zeros(12); c[:10] = rng.standard_normal(10)
    ref = np.zeros(12); r = npc.chebmulx(c[:10]); ref[:len(r)] = r
    assert np.allclose(ch.xmul_matrix(12) @ c, ref, atol=1e-15)


def test_fourier_numpy_path_matches_direct_sums():
    rng = np.random.default_rng(5)
    n_phi, n_m = 48, 16
    fm = rng.standard_normal((3, n_m + 1)) + 1j * rng.standard_normal((3, n_m + 1))
    fm[:, 0] = fm[:, 0].real
    g = fo.to_grid(fm, n_phi)
    assert np.allclose(g, fo.to_grid_direct(fm, n_phi), atol=1e-12)
    assert np.allclose(fo.to_spec(g, n_m), fo.to_spec_direct(g, n_m), atol=1e-13)
    assert np.allclose(fo.to_spec(g, n_m), fm, atol=1e-13)


def test_fourier_single_mode_closed_form():
    # f_m = a for one m >= 1: f(phi) = 2 Re{a e^{i m phi}}  (Eq. fft)
    n_phi, n_m, m, a = 24, 8, 3, 0.7 - 0.2j
    fm = np.zeros(n_m + 1, complex); fm[m] = a
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    assert np.allclose(fo.to_grid(fm, n_phi), 2 * np.real(a * np.exp(1j * m * phi)), atol=1e-14)


def test_product_of_band_limited_fields_is_alias_free():
    # N_phi = 3 N_m (the paper's choice): products of two degree-N_m fields are
    # alias-free for m < N_m; the top mode m = N_m receives the alias of 2 N_m.
    rng = np.random.default_rng(6)
    n_m = 10; n_phi = 3 * n_m
    a = rng.standard_normal(n_m + 1) + 1j * rng.standard_normal(n_m + 1); a[0] = a[0].real
    b = rng.standard_normal(n_m + 1) + 1j * rng.standard_normal(n_m + 1); b[0] = b[0].real
    big = 8 * n_m
    ref = fo.to_spec(fo.to_grid(a, big) * fo.to_grid(b, big), n_m)
    got = fo.to_spec(fo.to_grid(a, n_phi) * fo.to_grid(b, n_phi), n_m)
    assert np.allclose(got[:n_m], ref[:n_m], atol=1e-12)
    assert not np.allclose(got[n_m], ref[n_m], atol=1e-12)
