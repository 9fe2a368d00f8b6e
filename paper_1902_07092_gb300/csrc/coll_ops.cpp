// Host-side set-up of the Chebyshev-collocation formulation (Section 3.1,
// Eqs. psiomcoll, uphicoll, tempcoll with the boundary rows of Eqs.
// bcs_coll_dirichlet and bcs_coll_neumann) of Gastine, pizza, GJI 2019.
//
// The device keeps every collocation field as its values on the Gauss-Lobatto
// grid, so the systems are written for grid unknowns: with D1, D2 the
// differentiation matrices of the N-point interpolant (d/ds, d^2/ds^2), the
// vorticity-streamfunction system for mode m and implicit weight g = gamma dt is
//   rows k = 1..N-2:  omega_k - g [D2 omega + D1 omega/s - m^2 omega/s^2]_k
//                     + g b_k psi_k = r_k,      b_k = -(2/E) i m beta_k/s_k
//   rows 0, N-1:      (D1 psi)_0 = 0, (D1 psi)_{N-1} = 0           (Neumann)
//   rows N+k:         omega_k + [D2 psi + (beta + 1/s) D1 psi
//                     + (dbeta/ds + beta/s - m^2/s^2) psi]_k = 0   (k = 1..N-2)
//   rows N, 2N-1:     psi_0 = 0, psi_{N-1} = 0                      (Dirichlet)
// (the B^C term of Eq. psiomcoll is diag(b) T; C^C is L_beta, whose printed
// sign of dbeta/ds + beta/s contradicts the definition of L_beta; the
// definition is used).  Temperature and zonal flow:
//   rows k = 1..N-2:  f_k - g kappa [D2 f + D1 f/s - q f/s^2]_k = r_k,  rows 0, N-1: f = 0
// with (kappa, q) = (1/Pr, m^2) and (1, 1).  Only the interior rows of the right
// hand side are ever nonzero, so only the N-2 matching columns of each inverse
// are kept; they are computed by LU with row equilibration and partial
// pivoting, followed by one step of iterative refinement in FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "host_ops.h"

namespace pz {

CollGrid coll_grid(int n_r, const Geom& g) {
    CollGrid c;
    const int N = n_r, K = n_r - 1;
    c.N = N;
    c.s.resize(N);
    c.beta.assign(N, 0.0);
    c.dbeta.assign(N, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    const double S = g.s_o * g.s_o;
    for (int k = 0; k < N; ++k) {
        const double x = (double)cosl(pi * (long double)k / (long double)K);
        c.s[k] = g.a * x + g.b;
        if (k > 0) {
            const double h2 = S - c.s[k] * c.s[k];
            c.beta[k] = -c.s[k] / h2;
            c.dbeta[k] = -(S + c.s[k] * c.s[k]) / (h2 * h2);
        }
    }
    // first-derivative matrix of the Gauss-Lobatto interpolant (in x):
    //   D_ij = (c_i/c_j) (-1)^(i+j) / (x_i - x_j),  c_0 = c_K = 2, else 1,
    // with x_i - x_j = -2 sin(pi (i+j)/2K) sin(pi (i-j)/2K) and the diagonal from
    // the vanishing derivative of a constant (negative row sum).
    std::vector<double> D((size_t)N * N);
    for (int i = 0; i < N; ++i) {
        long double sum = 0.0L;
        for (int j = 0; j < N; ++j) {
            if (i == j) continue;
            const long double ci = (i == 0 || i == K) ? 2.0L : 1.0L;
            const long double cj = (j == 0 || j == K) ? 2.0L : 1.0L;
            const long double dx =
                -2.0L * sinl(pi * (long double)(i + j) / (2.0L * K)) * sinl(pi * (long double)(i - j) / (2.0L * K));
            const long double v = (ci / cj) * (((i + j) & 1) ? -1.0L : 1.0L) / dx;
            D[(size_t)i * N + j] = (double)v;
            sum += v;
        }
        D[(size_t)i * N + i] = (double)(-sum);
    }
    const double ia = 1.0 / g.a;
    c.D1.resize((size_t)N * N);
    for (size_t i = 0; i < c.D1.size(); ++i) c.D1[i] = D[i] * ia;
    // D2 = D1 D1, its diagonal again from the row sums
    c.D2.assign((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i) {
        double* row = &c.D2[(size_t)i * N];
        for (int k = 0; k < N; ++k) {
            const double a = c.D1[(size_t)i * N + k];
            const double* rk = &c.D1[(size_t)k * N];
            for (int j = 0; j < N; ++j) row[j] += a * rk[j];
        }
        long double sum = 0.0L;
        for (int j = 0; j < N; ++j)
            if (j != i) sum += row[j];
        row[i] = (double)(-sum);
    }
    // synthesis matrix T_kn = C w_n T_n(x_k) (Eq. cheb); it is an involution, so
    // it is also the analysis matrix of Eq. icheb
    c.T.resize((size_t)N * N);
    const double C = std::sqrt(2.0 / (double)K);
    for (int k = 0; k < N; ++k)
        for (int n = 0; n < N; ++n) {
            const double w = (n == 0 || n == K) ? 0.5 : 1.0;
            const long long kn = (long long)k * n % (2LL * K);
            c.T[(size_t)k * N + n] = C * w * (double)cosl(pi * (long double)kn / (long double)K);
        }
    return c;
}

namespace {

// Dense row-major n x n matrix with split real / imaginary planes (im empty for
// a real matrix) and LU with partial pivoting in place.
struct Dense {
    int n = 0;
    bool cx = false;
    std::vector<double> re, im;
    std::vector<int> piv;
};

bool lu_factor(Dense& A) {
    const int n = A.n;
    A.piv.resize(n);
    double* re = A.re.data();
    double* im = A.cx ? A.im.data() : nullptr;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = -1.0;
        for (int i = k; i < n; ++i) {
            const double a = re[(size_t)i * n + k], b = im ? im[(size_t)i * n + k] : 0.0;
            const double v = a * a + b * b;
            if (v > best) {
                best = v;
                p = i;
            }
        }
        if (!(best > 0.0)) return false;
        A.piv[k] = p;
        if (p != k) {
            std::swap_ranges(re + (size_t)k * n, re + (size_t)(k + 1) * n, re + (size_t)p * n);
            if (im) std::swap_ranges(im + (size_t)k * n, im + (size_t)(k + 1) * n, im + (size_t)p * n);
        }
        const double pr = re[(size_t)k * n + k], pi_ = im ? im[(size_t)k * n + k] : 0.0;
        const double den = pr * pr + pi_ * pi_;
        const double ir = pr / den, ii = -pi_ / den;  // 1 / pivot
        const double* rk = re + (size_t)k * n;
        const double* ik = im ? im + (size_t)k * n : nullptr;
        for (int i = k + 1; i < n; ++i) {
            double* ri = re + (size_t)i * n;
            const double ar = ri[k];
            if (!im) {
                const double l = ar * ir;
                ri[k] = l;
                if (l == 0.0) continue;
                for (int j = k + 1; j < n; ++j) ri[j] -= l * rk[j];
            } else {
                double* ji = im + (size_t)i * n;
                const double ai = ji[k];
                const double lr = ar * ir - ai * ii, li = ar * ii + ai * ir;
                ri[k] = lr;
                ji[k] = li;
                if (lr == 0.0 && li == 0.0) continue;
                for (int j = k + 1; j < n; ++j) {
                    const double br = rk[j], bi = ik[j];
                    ri[j] -= lr * br - li * bi;
                    ji[j] -= lr * bi + li * br;
                }
            }
        }
    }
    return true;
}

// Solve A X = B in place for B row-major n x nr (split planes like A).
void lu_solve(const Dense& A, int nr, double* bre, double* bim) {
    const int n = A.n;
    const double* re = A.re.data();
    const double* im = A.cx ? A.im.data() : nullptr;
    for (int k = 0; k < n; ++k) {
        const int p = A.piv[k];
        if (p != k) {
            std::swap_ranges(bre + (size_t)k * nr, bre + (size_t)(k + 1) * nr, bre + (size_t)p * nr);
            if (bim) std::swap_ranges(bim + (size_t)k * nr, bim + (size_t)(k + 1) * nr, bim + (size_t)p * nr);
        }
    }
    auto axpy = [&](int dst, int src, double lr, double li) {
        double* dr = bre + (size_t)dst * nr;
        const double* sr = bre + (size_t)src * nr;
        if (!bim) {
            for (int j = 0; j < nr; ++j) dr[j] -= lr * sr[j];
            return;
        }
        double* di = bim + (size_t)dst * nr;
        const double* si = bim + (size_t)src * nr;
        for (int j = 0; j < nr; ++j) {
            const double xr = sr[j], xi = si[j];
            dr[j] -= lr * xr - li * xi;
            di[j] -= lr * xi + li * xr;
        }
    };
    for (int i = 1; i < n; ++i)
        for (int k = 0; k < i; ++k) {
            const double lr = re[(size_t)i * n + k], li = im ? im[(size_t)i * n + k] : 0.0;
            if (lr != 0.0 || li != 0.0) axpy(i, k, lr, li);
        }
    for (int i = n - 1; i >= 0; --i) {
        for (int k = i + 1; k < n; ++k) {
            const double ur = re[(size_t)i * n + k], ui = im ? im[(size_t)i * n + k] : 0.0;
            if (ur != 0.0 || ui != 0.0) axpy(i, k, ur, ui);
        }
        const double pr = re[(size_t)i * n + i], pi_ = im ? im[(size_t)i * n + i] : 0.0;
        const double den = pr * pr + pi_ * pi_;
        const double ir = pr / den, ii = -pi_ / den;
        double* dr = bre + (size_t)i * nr;
        if (!bim) {
            for (int j = 0; j < nr; ++j) dr[j] *= ir;
        } else {
            double* di = bim + (size_t)i * nr;
            for (int j = 0; j < nr; ++j) {
                const double xr = dr[j], xi = di[j];
                dr[j] = xr * ir - xi * ii;
                di[j] = xr * ii + xi * ir;
            }
        }
    }
}

// Columns X = A0^{-1} E of the inverse, E holding one unit vector per column:
// rows[c] is the row of the nonzero of column c.  A0 is left unchanged.
bool inverse_columns(const Dense& A0, const std::vector<int>& rows, std::vector<double>& xre,
                     std::vector<double>& xim) {
    const int n = A0.n, nr = (int)rows.size();
    const bool cx = A0.cx;
    std::vector<double> scale(n);
    Dense A = A0;
    for (int i = 0; i < n; ++i) {
        double mx = 0.0;
        for (int j = 0; j < n; ++j) {
            const double a = A0.re[(size_t)i * n + j], b = cx ? A0.im[(size_t)i * n + j] : 0.0;
            mx = std::max(mx, std::sqrt(a * a + b * b));
        }
        if (!(mx > 0.0)) return false;
        scale[i] = 1.0 / mx;
        for (int j = 0; j < n; ++j) {
            A.re[(size_t)i * n + j] *= scale[i];
            if (cx) A.im[(size_t)i * n + j] *= scale[i];
        }
    }
    if (!lu_factor(A)) return false;
    xre.assign((size_t)n * nr, 0.0);
    if (cx) xim.assign((size_t)n * nr, 0.0);
    for (int c = 0; c < nr; ++c) xre[(size_t)rows[c] * nr + c] = scale[rows[c]];
    lu_solve(A, nr, xre.data(), cx ? xim.data() : nullptr);
    // one refinement step: R = E - A0 X (skipping the zero entries of A0), X += A^{-1} R
    std::vector<double> rre((size_t)n * nr, 0.0), rim;
    if (cx) rim.assign((size_t)n * nr, 0.0);
    for (int c = 0; c < nr; ++c) rre[(size_t)rows[c] * nr + c] = 1.0;
    for (int i = 0; i < n; ++i) {
        double* dr = &rre[(size_t)i * nr];
        double* di = cx ? &rim[(size_t)i * nr] : nullptr;
        for (int k = 0; k < n; ++k) {
            const double ar = A0.re[(size_t)i * n + k], ai = cx ? A0.im[(size_t)i * n + k] : 0.0;
            if (ar == 0.0 && ai == 0.0) continue;
            const double* sr = &xre[(size_t)k * nr];
            if (!cx) {
                for (int j = 0; j < nr; ++j) dr[j] -= ar * sr[j];
            } else {
                const double* si = &xim[(size_t)k * nr];
                for (int j = 0; j < nr; ++j) {
                    dr[j] -= ar * sr[j] - ai * si[j];
                    di[j] -= ar * si[j] + ai * sr[j];
                }
            }
        }
        for (int j = 0; j < nr; ++j) {
            dr[j] *= scale[i];
            if (cx) di[j] *= scale[i];
        }
    }
    lu_solve(A, nr, rre.data(), cx ? rim.data() : nullptr);
    for (size_t i = 0; i < xre.size(); ++i) xre[i] += rre[i];
    if (cx)
        for (size_t i = 0; i < xim.size(); ++i) xim[i] += rim[i];
    return true;
}

}  // namespace

bool dense_inverse(int n, const std::vector<cplx>& A, std::vector<cplx>& inv) {
    Dense D;
    D.n = n;
    D.cx = true;
    D.re.resize((size_t)n * n);
    D.im.resize((size_t)n * n);
    for (size_t i = 0; i < D.re.size(); ++i) {
        D.re[i] = A[i].real();
        D.im[i] = A[i].imag();
    }
    std::vector<int> rows(n);
    for (int i = 0; i < n; ++i) rows[i] = i;
    std::vector<double> xr, xi;
    if (!inverse_columns(D, rows, xr, xi)) return false;
    inv.resize((size_t)n * n);
    for (size_t i = 0; i < inv.size(); ++i) inv[i] = cplx(xr[i], xi[i]);
    return true;
}

bool dense_inverse(int n, const std::vector<double>& A, std::vector<double>& inv) {
    Dense D;
    D.n = n;
    D.cx = false;
    D.re = A;
    std::vector<int> rows(n);
    for (int i = 0; i < n; ++i) rows[i] = i;
    std::vector<double> xi;
    return inverse_columns(D, rows, inv, xi);
}

void coll_pumping(CollGrid& c, const Geom& g, double E) {
    const int N = c.N;
    c.ups.assign(N, 0.0);
    c.c5.assign(N, 0.0);
    const double S = g.s_o * g.s_o;
    for (int k = 1; k < N; ++k) {
        const double s = c.s[k], h = std::sqrt(S - s * s);
        c.ups[k] = std::sqrt(g.s_o / E) / (h * std::sqrt(h));
        c.c5[k] = 2.5 * g.s_o * c.beta[k] / (h * s);
    }
}

bool coll_inverse_wpsi(const CollGrid& c, double E, int m, double gdt, std::vector<cplx>& G) {
    const int N = c.N, n = 2 * N;
    Dense A;
    A.n = n;
    A.cx = true;
    A.re.assign((size_t)n * n, 0.0);
    A.im.assign((size_t)n * n, 0.0);
    const double mu = (double)m * m, dm = (double)m;
    auto R = [&](int i, int j) -> double& { return A.re[(size_t)i * n + j]; };
    for (int k = 1; k + 1 < N; ++k) {
        const double s = c.s[k], is = 1.0 / s;
        for (int j = 0; j < N; ++j) {
            double v = -gdt * (c.D2[(size_t)k * N + j] + c.D1[(size_t)k * N + j] * is);
            if (j == k) v += 1.0 + gdt * mu * is * is;
            R(k, j) = v;
            // constraint row: L_beta psi
            double w = c.D2[(size_t)k * N + j] + (c.beta[k] + is) * c.D1[(size_t)k * N + j];
            if (j == k) w += c.dbeta[k] + c.beta[k] * is - mu * is * is;
            R(N + k, N + j) = w;
        }
        // g b_k psi_k, b_k = -(2/E) i m beta_k / s_k
        A.im[(size_t)k * n + N + k] = gdt * (-2.0 / E) * dm * c.beta[k] * is;
        R(N + k, k) = 1.0;
        if (!c.ups.empty()) {
            // exact Ekman pumping F = -U omega - (U beta/2) psi'
            //   + U (-beta^2/2 + beta m^2/s + i m c5) psi, moved to the left as -g F
            const double U = c.ups[k], b = c.beta[k];
            R(k, k) += gdt * U;
            for (int j = 0; j < N; ++j) R(k, N + j) += gdt * 0.5 * U * b * c.D1[(size_t)k * N + j];
            R(k, N + k) -= gdt * U * (-0.5 * b * b + b * mu * is);
            A.im[(size_t)k * n + N + k] -= gdt * U * dm * c.c5[k];
        }
    }
    for (int j = 0; j < N; ++j) {
        R(0, N + j) = c.D1[j];
        R(N - 1, N + j) = c.D1[(size_t)(N - 1) * N + j];
    }
    R(N, N) = 1.0;
    R(2 * N - 1, 2 * N - 1) = 1.0;
    std::vector<int> rows;
    for (int k = 1; k + 1 < N; ++k) rows.push_back(k);
    std::vector<double> xr, xi;
    if (!inverse_columns(A, rows, xr, xi)) return false;
    G.resize(xr.size());
    for (size_t i = 0; i < xr.size(); ++i) G[i] = cplx(xr[i], xi[i]);
    return true;
}

bool coll_inverse_dir(const CollGrid& c, double kappa, double q, double gdt, std::vector<double>& G, bool pump) {
    const int N = c.N;
    Dense A;
    A.n = N;
    A.cx = false;
    A.re.assign((size_t)N * N, 0.0);
    for (int k = 1; k + 1 < N; ++k) {
        const double is = 1.0 / c.s[k];
        for (int j = 0; j < N; ++j) {
            double v = -gdt * kappa * (c.D2[(size_t)k * N + j] + c.D1[(size_t)k * N + j] * is);
            if (j == k) v += 1.0 + gdt * kappa * q * is * is + ((pump && !c.ups.empty()) ? gdt * c.ups[k] : 0.0);
            A.re[(size_t)k * N + j] = v;
        }
    }
    A.re[0] = 1.0;
    A.re[(size_t)N * N - 1] = 1.0;
    std::vector<int> rows;
    for (int k = 1; k + 1 < N; ++k) rows.push_back(k);
    std::vector<double> xi;
    return inverse_columns(A, rows, G, xi);
}

}  // namespace pz
