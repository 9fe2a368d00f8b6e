"""Chebyshev series on the Gauss-Lobatto grid (Section 3, Eqs. cheb and icheb; the
integral identity Eq. int1).

Test infrastructure only (see the package docstring).

Two coefficient conventions appear:

* the paper's ``f_hat``:  f(x_k) = C sum''_{n<N_c} f_hat_n T_n(x_k), with
  C = [2/(N_r-1)]^(1/2) and the double prime halving the n = 0 and n = N_r-1
  terms (Eq. cheb).  The analysis sum Eq. icheb has the same form, so the pair is
  an involution.  When N_c < N_r the n = N_r-1 term is absent and only n = 0 is
  halved.
* plain coefficients ``c``:  f(x) = sum_n c_n T_n(x), i.e. c_n = C w_n f_hat_n with
  w_0 = w_{N_r-1} = 1/2 and w_n = 1 otherwise.  The operators below act on ``c``.
"""
import numpy as np


def tmat(n_r, n_c):
    """T_kn = T_n(x_k) = cos(pi n k/(N_r-1)), k < N_r, n < n_c."""
    k = np.arange(n_r)[:, None]
    n = np.arange(n_c)[None, :]
    return np.cos(np.pi * n * k / (n_r - 1))


def norm_c(n_r):
    return np.sqrt(2.0 / (n_r - 1))


def dp_weights(n_r, length):
    """Double-prime weights of a sum over indices 0..length-1 in a transform of
    N_r points: 1/2 at 0 and at N_r-1, 1 elsewhere."""
    w = np.ones(length)
    w[0] = 0.5
    if length >= n_r:
        w[n_r - 1] = 0.5
    return w


def analysis(f_grid, n_r):
    """Eq. icheb: f_hat_n = C sum''_k f(x_k) T_n(x_k), n = 0..N_r-1.
    ``f_grid`` has the radial index first; further axes are carried along."""
    f_grid = np.asarray(f_grid)
    T = tmat(n_r, n_r)
    wk = dp_weights(n_r, n_r)
    wf = f_grid * wk.reshape((-1,) + (1,) * (f_grid.ndim - 1))
    return norm_c(n_r) * np.tensordot(T.T, wf, axes=(1, 0))


def synthesis(f_hat, n_r):
    """Eq. cheb: f(x_k) = C sum''_n f_hat_n T_n(x_k); ``f_hat`` has the
    coefficient index first (length n_c <= N_r)."""
    f_hat = np.asarray(f_hat)
    n_c = f_hat.shape[0]
    T = tmat(n_r, n_c)
    wn = dp_weights(n_r, n_c)
    wf = f_hat * wn.reshape((-1,) + (1,) * (f_hat.ndim - 1))
    return norm_c(n_r) * np.tensordot(T, wf, axes=(1, 0))


def hat_to_plain(f_hat, n_r):
    f_hat = np.asarray(f_hat)
    w = dp_weights(n_r, f_hat.shape[0]).reshape((-1,) + (1,) * (f_hat.ndim - 1))
    return norm_c(n_r) * w * f_hat


def plain_to_hat(c, n_r):
    c = np.asarray(c)
    w = dp_weights(n_r, c.shape[0]).reshape((-1,) + (1,) * (c.ndim - 1))
    return c / (norm_c(n_r) * w)


def hat_scale(n_r, n_c):
    """Diagonal of the map f_hat -> c (length n_c)."""
    return norm_c(n_r) * dp_weights(n_r, n_c)


def diff_matrix(K):
    """d/dx on plain coefficients (closed form, e.g. Canuto et al. Eq. 2.4.22):
    (f')_j = (2/c_j) sum_{n>j, n+j odd} n c_n,  c_0 = 2, c_j = 1 (j > 0)."""
    D = np.zeros((K, K))
    for j in range(K):
        cj = 2.0 if j == 0 else 1.0
        for n in range(j + 1, K, 2):
            D[j, n] = 2.0 * n / cj
    return D


def xmul_matrix(K):
    """Multiplication by x on plain coefficients: x T_n = (T_{n+1} + T_{|n-1|})/2,
    x T_0 = T_1.  Truncated to K x K (callers pad)."""
    X = np.zeros((K, K))
    for n in range(K):
        if n == 0:
            if K > 1:
                X[1, 0] = 1.0
            continue
        if n + 1 < K:
            X[n + 1, n] += 0.5
        X[n - 1, n] += 0.5
    return X


def int_matrix(K):
    """Indefinite integration on plain coefficients from Eq. int1:
    int T_n = [T_{n+1}/(n+1) - T_{n-1}/(n-1)]/2 (n > 1), int T_0 = T_1,
    int T_1 = T_2/4; the constant of integration (row 0) is set to zero.
    Row k >= 1: F_k = (c_{k-1} (1 + delta_{k1}) - c_{k+1})/(2k)."""
    J = np.zeros((K, K))
    for k in range(1, K):
        J[k, k - 1] += (2.0 if k == 1 else 1.0) / (2.0 * k)
        if k + 1 < K:
            J[k, k + 1] -= 1.0 / (2.0 * k)
    return J


def eval_series(c, x):
    """sum_n c_n T_n(x) by the three-term recurrence (used by tests only)."""
    x = np.asarray(x, dtype=float)
    t0 = np.ones_like(x)
    out = c[0] * t0
    if len(c) == 1:
        return out
    t1 = x.copy()
    out = out + c[1] * t1
    for n in range(2, len(c)):
        t0, t1 = t1, 2 * x * t1 - t0
        out = out + c[n] * t1
    return out
