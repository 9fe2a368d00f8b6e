// Host-side operator construction for the Chebyshev-integration method
// (Section 3.2, Eqs. psi_int, uphi_int, temp_int of Gastine, pizza, GJI 2019).
//
// Each operator is  int^q_s ( sum_p P_p(s) d^p/ds^p ),  P_p polynomials in s.
// With s = a x + b the coefficients become Chebyshev series Q_p(x) (times
// a^{-p}); integrating by parts until no derivative remains gives, in the rows
// k >= q that survive the tau rows,
//   int^q (Q d^p f) = sum_{j=0..p} (-1)^j binom(p,j) int^(q-p+j) (Q^(j) f).
// Columns are built one basis polynomial T_n at a time with the product rule
// T_i T_n = (T_{i+n} + T_{|i-n|})/2 and the integral identity Eq. int1.
//
// The coefficient polynomials were derived by hand from the definitions
//   L_I Psi = Delta(h^2 Psi) - (1/s) d/ds(s^2 Psi),
//   Delta = d^2/ds^2 + (1/s) d/ds - m^2/s^2,  h^2 = S - s^2,  S = s_o^2:
//   s^4 L_I          = (S s^4 - s^6) D^2 + (S s^3 - 6 s^5) D - 6 s^4 + m^2 (s^4 - S s^2)
//   s^4 Delta L_I    = (S s^4 - s^6) D^4 + (2 S s^3 - 11 s^5) D^3
//                      + (-28 s^4 - S s^2) D^2 + (S s - 12 s^3) D
//                      + m^2 [ (2 s^4 - 2 S s^2) D^2 + (2 S s + 7 s^3) D + 6 s^2 - 4 S ]
//                      + m^4 (S - s^2)
//   s^2 Delta        = s^2 D^2 + s D - m^2
//   s^2 (Delta - 1/s^2) at m = 0 = s^2 D^2 + s D - 1          (E^I)
//   C^I: s^4 (q = 4); D^I: s^2 (q = 2); G^I: h^2 (q = 2).
#include "host_ops.h"

#include <cmath>
#include <map>

namespace pz {

Geom make_geom(double eta) {
    Geom g;
    g.eta = eta;
    g.s_o = 1.0 / (1.0 - eta);
    g.s_i = eta / (1.0 - eta);
    g.a = 0.5 * (g.s_o - g.s_i);
    g.b = 0.5 * (g.s_o + g.s_i);
    return g;
}

double tc_coefficient(double eta) {
    double r = std::sqrt(1.0 - eta * eta);
    double alpha = eta / (1.0 - eta) * (std::asinh(r / eta) / r - 1.0);
    return alpha / std::log(eta);
}

namespace {

// polynomial in s: power -> coefficient
using SPoly = std::map<int, double>;
// operator: derivative order -> polynomial coefficient
using SOp = std::map<int, SPoly>;

struct OpDef {
    int q;
    SOp op;
};

OpDef op_def(int id, double S) {
    OpDef d;
    switch (id) {
        case OP_A0:
            d.q = 4;
            d.op[2] = {{4, S}, {6, -1.0}};
            d.op[1] = {{3, S}, {5, -6.0}};
            d.op[0] = {{4, -6.0}};
            break;
        case OP_A2:
            d.q = 4;
            d.op[0] = {{4, 1.0}, {2, -S}};
            break;
        case OP_B0:
            d.q = 4;
            d.op[4] = {{4, S}, {6, -1.0}};
            d.op[3] = {{3, 2.0 * S}, {5, -11.0}};
            d.op[2] = {{4, -28.0}, {2, -S}};
            d.op[1] = {{1, S}, {3, -12.0}};
            break;
        case OP_B2:
            d.q = 4;
            d.op[2] = {{4, 2.0}, {2, -2.0 * S}};
            d.op[1] = {{1, 2.0 * S}, {3, 7.0}};
            d.op[0] = {{2, 6.0}, {0, -4.0 * S}};
            break;
        case OP_B4:
            d.q = 4;
            d.op[0] = {{0, S}, {2, -1.0}};
            break;
        case OP_C:
            d.q = 4;
            d.op[0] = {{4, 1.0}};
            break;
        case OP_D:
            d.q = 2;
            d.op[0] = {{2, 1.0}};
            break;
        case OP_F0:
            d.q = 2;
            d.op[2] = {{2, 1.0}};
            d.op[1] = {{1, 1.0}};
            break;
        case OP_F2:
            d.q = 2;
            d.op[0] = {{0, -1.0}};
            break;
        case OP_EZ:
            d.q = 2;
            d.op[2] = {{2, 1.0}};
            d.op[1] = {{1, 1.0}};
            d.op[0] = {{0, -1.0}};
            break;
        case OP_G:
            d.q = 2;
            d.op[0] = {{0, S}, {2, -1.0}};
            break;
        default:
            d.q = 0;
    }
    return d;
}

// Chebyshev series of b + a x raised to the power k, for k = 0..kmax.
std::vector<std::vector<double>> s_powers(const Geom& g, int kmax) {
    std::vector<std::vector<double>> pw(kmax + 1);
    pw[0] = {1.0};
    for (int k = 1; k <= kmax; ++k) {
        const auto& p = pw[k - 1];
        std::vector<double> r(p.size() + 1, 0.0);
        for (size_t i = 0; i < p.size(); ++i) {
            // (b + a x) * p_i T_i,  x T_i = (T_{i+1} + T_{|i-1|})/2,  x T_0 = T_1
            r[i] += g.b * p[i];
            if (i == 0) {
                r[1] += g.a * p[i];
            } else {
                r[i + 1] += 0.5 * g.a * p[i];
                r[i - 1] += 0.5 * g.a * p[i];
            }
        }
        pw[k] = r;
    }
    return pw;
}

std::vector<double> cheb_derivative(const std::vector<double>& c) {
    int n = (int)c.size();
    if (n <= 1) return {0.0};
    std::vector<double> d(n, 0.0);  // d[n-1] = 0
    for (int k = n - 1; k >= 1; --k) {
        double next = (k + 1 < n) ? d[k + 1] : 0.0;
        d[k - 1] = next + 2.0 * k * c[k];
    }
    d[0] *= 0.5;
    d.resize(n - 1);
    return d;
}

// in place: integrate plain coefficients over the window [lo, hi]; constant 0.
void integrate(std::vector<double>& c, int& lo, int& hi, int Kp) {
    int nlo = std::max(1, lo - 1), nhi = std::min(Kp - 1, hi + 1);
    std::vector<double> F(nhi - nlo + 1, 0.0);
    for (int k = nlo; k <= nhi; ++k) {
        double cm = (k - 1 >= lo && k - 1 <= hi) ? c[k - 1] : 0.0;
        double cp = (k + 1 >= lo && k + 1 <= hi) ? c[k + 1] : 0.0;
        F[k - nlo] = ((k == 1 ? 2.0 : 1.0) * cm - cp) / (2.0 * k);
    }
    for (int k = lo; k <= hi; ++k) c[k] = 0.0;
    for (int k = nlo; k <= nhi; ++k) c[k] = F[k - nlo];
    c[0] = 0.0;
    lo = nlo;
    hi = nhi;
}

double binom(int p, int j) {
    double r = 1.0;
    for (int t = 1; t <= j; ++t) r = r * (p - j + t) / t;
    return r;
}

}  // namespace

int op_q(int id) { return op_def(id, 1.0).q; }

int op_h(int id) {
    switch (id) {
        case OP_A0: case OP_A2: case OP_C: return 8;
        case OP_B0: case OP_B2: case OP_B4: return 6;
        case OP_D: case OP_G: return 4;
        default: return 2;
    }
}

std::vector<double> build_operator(int id, int n_r, int n_c, const Geom& g) {
    OpDef def = op_def(id, g.s_o * g.s_o);
    const int q = def.q;
    int maxdeg = 0;
    for (auto& kv : def.op)
        for (auto& t : kv.second) maxdeg = std::max(maxdeg, t.first);
    const int Kp = n_c + 2 * (maxdeg + q) + 8;
    auto pw = s_powers(g, maxdeg);

    std::vector<double> M((size_t)n_c * n_c, 0.0);
    std::vector<double> work(Kp);
    for (auto& kv : def.op) {
        const int p = kv.first;
        // Q_p(x) = a^{-p} P_p(a x + b) as a Chebyshev series
        std::vector<double> Q(maxdeg + 1, 0.0);
        for (auto& t : kv.second)
            for (size_t i = 0; i < pw[t.first].size(); ++i) Q[i] += t.second * pw[t.first][i];
        const double ap = std::pow(g.a, -p);
        for (auto& v : Q) v *= ap;
        std::vector<double> Qj = Q;
        for (int j = 0; j <= p; ++j) {
            const double coef = ((j & 1) ? -1.0 : 1.0) * binom(p, j);
            const int r = q - p + j;
            const int dq = (int)Qj.size() - 1;
            for (int n = 0; n < n_c; ++n) {
                std::fill(work.begin(), work.end(), 0.0);
                int lo = Kp, hi = -1;
                for (int i = 0; i <= dq; ++i) {
                    if (Qj[i] == 0.0) continue;
                    const double v = 0.5 * Qj[i];
                    const int k1 = i + n, k2 = std::abs(i - n);
                    work[k1] += v;
                    work[k2] += v;
                    lo = std::min(lo, std::min(k1, k2));
                    hi = std::max(hi, std::max(k1, k2));
                }
                if (hi < 0) continue;
                for (int t = 0; t < r; ++t) integrate(work, lo, hi, Kp);
                for (int k = std::max(lo, q); k <= std::min(hi, n_c - 1); ++k)
                    M[(size_t)k * n_c + n] += coef * work[k];
            }
            Qj = cheb_derivative(Qj);
        }
    }
    const double aq = std::pow(g.a, q);
    const double C = std::sqrt(2.0 / (n_r - 1));
    for (int k = 0; k < n_c; ++k)
        for (int n = 0; n < n_c; ++n) {
            double w = (n == 0 || n == n_r - 1) ? 0.5 : 1.0;
            M[(size_t)k * n_c + n] = (k < q) ? 0.0 : M[(size_t)k * n_c + n] * aq * C * w;
        }
    return M;
}

std::vector<double> to_band(const std::vector<double>& dense, int n_c, int h) {
    const int W = 2 * h + 1;
    std::vector<double> b((size_t)n_c * W, 0.0);
    for (int k = 0; k < n_c; ++k)
        for (int d = 0; d < W; ++d) {
            int n = k - h + d;
            if (n >= 0 && n < n_c) b[(size_t)k * W + d] = dense[(size_t)k * n_c + n];
        }
    return b;
}

static std::vector<double> tau_rows(int n_r, int n_c, const int* kinds, int p) {
    const double C = std::sqrt(2.0 / (n_r - 1));
    std::vector<double> r((size_t)p * n_c);
    for (int i = 0; i < p; ++i)
        for (int n = 0; n < n_c; ++n) {
            double dn = n, sg = (n & 1) ? -1.0 : 1.0, v = 0.0;
            switch (kinds[i]) {
                case 0: v = 1.0; break;                                             // f(1)
                case 1: v = sg; break;                                              // f(-1)
                case 2: v = dn * dn * (dn * dn - 1.0) * (dn * dn - 4.0); break;     // f'''(1)
                case 3: v = -sg * dn * dn; break;                                    // f'(-1)
            }
            double w = (n == 0 || n == n_r - 1) ? 0.5 : 1.0;
            r[(size_t)i * n_c + n] = v * C * w;
        }
    return r;
}

std::vector<double> tau_rows_psi(int n_r, int n_c) {
    const int k[4] = {0, 1, 2, 3};
    return tau_rows(n_r, n_c, k, 4);
}

std::vector<double> tau_rows_dir(int n_r, int n_c) {
    const int k[2] = {0, 1};
    return tau_rows(n_r, n_c, k, 2);
}

// Sums in twice the working precision (Ogita, Rump and Oishi 2005, "Accurate sum
// and dot product"): a product a b is split exactly as p + e with
// e = fma(a, b, -p), a sum s + p exactly as s' + t by Knuth's two-sum; the
// leading parts accumulate in hi, the errors in lo.  The library is built with
// floating-point contraction off, so p and the sums are rounded as written.
struct Acc2 {
    double hi = 0.0, lo = 0.0;
    void add(double v) {
        const double s = hi + v, bb = s - hi;
        lo += (hi - (s - bb)) + (v - bb);
        hi = s;
    }
    void add_prod(double a, double b) {
        const double p = a * b;
        lo += std::fma(a, b, -p);
        add(p);
    }
    double value() const { return hi + lo; }
};
// acc += a b for real and complex operands
static void acc_prod(Acc2* acc, double a, double b) { acc[0].add_prod(a, b); }
static void acc_prod(Acc2* acc, const cplx& a, const cplx& b) {
    acc[0].add_prod(a.real(), b.real());
    acc[0].add_prod(-a.imag(), b.imag());
    acc[1].add_prod(a.real(), b.imag());
    acc[1].add_prod(a.imag(), b.real());
}
static void acc_init(Acc2* acc, double v) { acc[0] = Acc2{}; acc[0].add(v); }
static void acc_init(Acc2* acc, const cplx& v) {
    acc[0] = Acc2{};
    acc[1] = Acc2{};
    acc[0].add(v.real());
    acc[1].add(v.imag());
}
static void acc_get(const Acc2* acc, double& v) { v = acc[0].value(); }
static void acc_get(const Acc2* acc, cplx& v) { v = cplx(acc[0].value(), acc[1].value()); }

template <class T>
bool factor_bordered(const std::vector<T>& band, int n_c, int h,
                     const std::vector<double>& tau, int p, Bordered<T>& out) {
    const int W = 2 * h + 1;
    const int n = n_c - p;
    out.n = n;
    out.p = p;
    out.h = h;
    // banded block D (rows/cols p..n_c-1) in a local dense-band work array
    // work[i][j - i + 2h] for |j - i| <= h (room for no fill: unpivoted LU keeps the band)
    std::vector<T> Db((size_t)n * W, T(0));
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < W; ++d) {
            int col = (i + p) - h + d;  // column in the full matrix
            if (col >= p && col < n_c) Db[(size_t)i * W + (col - p - i + h)] = band[(size_t)(i + p) * W + d];
        }
    auto at = [&](int i, int j) -> T& { return Db[(size_t)i * W + (j - i + h)]; };
    // unpivoted band LU
    for (int k = 0; k < n; ++k) {
        T piv = at(k, k);
        if (piv == T(0)) return false;
        for (int i = k + 1; i <= std::min(n - 1, k + h); ++i) {
            T l = at(i, k) / piv;
            at(i, k) = l;
            for (int j = k + 1; j <= std::min(n - 1, k + h); ++j) at(i, j) -= l * at(k, j);
        }
    }
    out.L.assign((size_t)n * h, T(0));
    out.U.assign((size_t)n * h, T(0));
    out.invd.assign(n, T(0));
    for (int i = 0; i < n; ++i) {
        out.invd[i] = T(1) / at(i, i);
        for (int t = 0; t < h; ++t) {
            if (i + 1 + t < n) {
                out.L[(size_t)i * h + t] = at(i + 1 + t, i);
                out.U[(size_t)i * h + t] = at(i, i + 1 + t);
            }
        }
    }
    auto solve = [&](std::vector<T>& x) {
        for (int j = 0; j < n; ++j)
            for (int t = 0; t < h && j + 1 + t < n; ++t) x[j + 1 + t] -= out.L[(size_t)j * h + t] * x[j];
        for (int j = n - 1; j >= 0; --j) {
            x[j] *= out.invd[j];
            for (int t = 0; t < h && j - 1 - t >= 0; ++t) x[j - 1 - t] -= out.U[(size_t)(j - 1 - t) * h + t] * x[j];
        }
    };
    // Y = D^{-1} C, C = rows p.., columns 0..p-1 of the band rows, refined twice
    // with residuals C - D Y summed in twice the working precision.  The bordered
    // step forms psi_2 = x - Y psi_1, a difference that cancels for large N_c;
    // with Y accurate to the last bits one refinement of the solve reaches ~10x
    // closer to the exact solution there (n_r = 2049, m = 2048: 4e-12 against
    // 4e-11 with the unrefined Y, measured on the tau systems).
    out.Y.assign((size_t)n * p, T(0));
    std::vector<T> col(n), cc(n), res(n);
    Acc2 acc[2];
    for (int c = 0; c < p; ++c) {
        for (int i = 0; i < n; ++i) {
            int row = i + p, d = c - row + h;
            cc[i] = (d >= 0 && d < W) ? band[(size_t)row * W + d] : T(0);
        }
        col = cc;
        solve(col);
        for (int it = 0; it < 2; ++it) {
            for (int i = 0; i < n; ++i) {
                acc_init(acc, cc[i]);
                const int row = i + p;
                for (int d = 0; d < W; ++d) {
                    const int j = row - h + d - p;  // column within D
                    if (j >= 0 && j < n) acc_prod(acc, -band[(size_t)row * W + d], col[j]);
                }
                acc_get(acc, res[i]);
            }
            solve(res);
            for (int i = 0; i < n; ++i) col[i] += res[i];
        }
        for (int i = 0; i < n; ++i) out.Y[(size_t)i * p + c] = col[i];
    }
    // Schur complement S = A - B Y
    std::vector<T> S((size_t)p * p);
    for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c) {
            T acc = T(tau[(size_t)r * n_c + c]);
            for (int i = 0; i < n; ++i) acc -= tau[(size_t)r * n_c + p + i] * out.Y[(size_t)i * p + c];
            S[(size_t)r * p + c] = acc;
        }
    // inverse by Gauss-Jordan with partial pivoting
    std::vector<T> I((size_t)p * p, T(0));
    for (int i = 0; i < p; ++i) I[(size_t)i * p + i] = T(1);
    for (int k = 0; k < p; ++k) {
        int piv = k;
        for (int i = k + 1; i < p; ++i)
            if (std::abs(S[(size_t)i * p + k]) > std::abs(S[(size_t)piv * p + k])) piv = i;
        if (S[(size_t)piv * p + k] == T(0)) return false;
        if (piv != k)
            for (int j = 0; j < p; ++j) {
                std::swap(S[(size_t)k * p + j], S[(size_t)piv * p + j]);
                std::swap(I[(size_t)k * p + j], I[(size_t)piv * p + j]);
            }
        T inv = T(1) / S[(size_t)k * p + k];
        for (int j = 0; j < p; ++j) {
            S[(size_t)k * p + j] *= inv;
            I[(size_t)k * p + j] *= inv;
        }
        for (int i = 0; i < p; ++i) {
            if (i == k) continue;
            T f = S[(size_t)i * p + k];
            for (int j = 0; j < p; ++j) {
                S[(size_t)i * p + j] -= f * S[(size_t)k * p + j];
                I[(size_t)i * p + j] -= f * I[(size_t)k * p + j];
            }
        }
    }
    out.Sinv = I;
    return true;
}

namespace {
template <class T>
bool invert_small(std::vector<T> A, int h, std::vector<T>& inv) {
    inv.assign((size_t)h * h, T(0));
    for (int i = 0; i < h; ++i) inv[(size_t)i * h + i] = T(1);
    for (int k = 0; k < h; ++k) {
        int piv = k;
        for (int i = k + 1; i < h; ++i)
            if (std::abs(A[(size_t)i * h + k]) > std::abs(A[(size_t)piv * h + k])) piv = i;
        if (A[(size_t)piv * h + k] == T(0)) return false;
        if (piv != k)
            for (int j = 0; j < h; ++j) {
                std::swap(A[(size_t)k * h + j], A[(size_t)piv * h + j]);
                std::swap(inv[(size_t)k * h + j], inv[(size_t)piv * h + j]);
            }
        const T d = T(1) / A[(size_t)k * h + k];
        for (int j = 0; j < h; ++j) {
            A[(size_t)k * h + j] *= d;
            inv[(size_t)k * h + j] *= d;
        }
        for (int i = 0; i < h; ++i) {
            if (i == k) continue;
            const T f = A[(size_t)i * h + k];
            if (f == T(0)) continue;
            for (int j = 0; j < h; ++j) {
                A[(size_t)i * h + j] -= f * A[(size_t)k * h + j];
                inv[(size_t)i * h + j] -= f * inv[(size_t)k * h + j];
            }
        }
    }
    return true;
}
}  // namespace

template <class T>
bool block_lu(const std::vector<T>& band, int n_c, int h, int p, std::vector<T>& out) {
    const int W = 2 * h + 1;
    const int n = n_c - p;
    const int nb = (n + h - 1) / h;
    // entry (i, j) of D (0-based within the block), identity beyond n
    auto Dat = [&](int i, int j) -> T {
        if (i >= n || j >= n) return (i == j) ? T(1) : T(0);
        const int d = j - i + h;
        if (d < 0 || d >= W) return T(0);
        return band[(size_t)(i + p) * W + d];
    };
    const size_t hh = (size_t)h * h;
    out.assign((size_t)nb * 3 * hh, T(0));
    std::vector<T> U(hh), Uinv_prev(hh), Uinv(hh), Lk(hh);
    for (int k = 0; k < nb; ++k) {
        const int r0 = k * h;
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < h; ++j) U[(size_t)i * h + j] = Dat(r0 + i, r0 + j);
        if (k > 0) {
            // L = D_{k,k-1} Uinv_{k-1};  U_kk -= L D_{k-1,k}
            for (int i = 0; i < h; ++i)
                for (int j = 0; j < h; ++j) {
                    T acc = T(0);
                    for (int t = 0; t < h; ++t) acc += Dat(r0 + i, r0 - h + t) * Uinv_prev[(size_t)t * h + j];
                    Lk[(size_t)i * h + j] = acc;
                }
            for (int i = 0; i < h; ++i)
                for (int j = 0; j < h; ++j) {
                    T acc = T(0);
                    for (int t = 0; t < h; ++t) acc += Lk[(size_t)i * h + t] * Dat(r0 - h + t, r0 + j);
                    U[(size_t)i * h + j] -= acc;
                }
            std::copy(Lk.begin(), Lk.end(), out.begin() + (size_t)k * 3 * hh);
        }
        if (!invert_small(U, h, Uinv)) return false;
        std::copy(Uinv.begin(), Uinv.end(), out.begin() + (size_t)k * 3 * hh + hh);
        if (k < nb - 1)
            for (int i = 0; i < h; ++i)
                for (int j = 0; j < h; ++j) {
                    T acc = T(0);
                    for (int t = 0; t < h; ++t) acc += Uinv[(size_t)i * h + t] * Dat(r0 + t, r0 + h + j);
                    out[(size_t)k * 3 * hh + 2 * hh + (size_t)i * h + j] = acc;
                }
        Uinv_prev = Uinv;
    }
    return true;
}

template <class T>
bool block_lu_twisted(const std::vector<T>& band, int n_c, int h, int p, std::vector<T>& out) {
    const int W = 2 * h + 1;
    const int n = n_c - p;
    const int nb = (n + h - 1) / h;
    const int c = nb / 2;
    auto Dat = [&](int i, int j) -> T {
        if (i >= n || j >= n) return (i == j) ? T(1) : T(0);
        const int d = j - i + h;
        if (d < 0 || d >= W) return T(0);
        return band[(size_t)(i + p) * W + d];
    };
    const size_t hh = (size_t)h * h;
    out.assign((size_t)nb * 3 * hh, T(0));
    auto blockD = [&](int bi, int bj, std::vector<T>& M) {
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < h; ++j) M[(size_t)i * h + j] = Dat(bi * h + i, bj * h + j);
    };
    auto matmul = [&](const std::vector<T>& A, const std::vector<T>& B, std::vector<T>& C) {
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < h; ++j) {
                T acc = T(0);
                for (int t = 0; t < h; ++t) acc += A[(size_t)i * h + t] * B[(size_t)t * h + j];
                C[(size_t)i * h + j] = acc;
            }
    };
    std::vector<T> U(hh), Ui(hh), Uprev(hh), L(hh), X(hh), Dc(hh), Dn(hh);
    auto put = [&](int k, int slot, const std::vector<T>& M) {
        std::copy(M.begin(), M.end(), out.begin() + (size_t)k * 3 * hh + slot * hh);
    };
    // top: U_k = D_kk - L_k D_{k-1,k},  L_k = D_{k,k-1} U_{k-1}^{-1},  H_k = U_k^{-1} D_{k,k+1}
    for (int k = 0; k < c; ++k) {
        blockD(k, k, U);
        if (k > 0) {
            blockD(k, k - 1, Dc);
            matmul(Dc, Uprev, L);
            blockD(k - 1, k, Dn);
            matmul(L, Dn, X);
            for (size_t i = 0; i < hh; ++i) U[i] -= X[i];
            put(k, 0, L);
        }
        if (!invert_small(U, h, Ui)) return false;
        put(k, 1, Ui);
        blockD(k, k + 1, Dn);
        matmul(Ui, Dn, X);
        put(k, 2, X);
        Uprev = Ui;
    }
    std::vector<T> Lc(hh, T(0)), Utop = Uprev;
    // bottom: V_k = D_kk - M_k D_{k+1,k},  M_k = D_{k,k+1} V_{k+1}^{-1},  G_k = V_k^{-1} D_{k,k-1}
    std::vector<T> Vprev(hh);
    for (int k = nb - 1; k > c; --k) {
        blockD(k, k, U);
        if (k < nb - 1) {
            blockD(k, k + 1, Dn);
            matmul(Dn, Vprev, L);
            blockD(k + 1, k, Dc);
            matmul(L, Dc, X);
            for (size_t i = 0; i < hh; ++i) U[i] -= X[i];
            put(k, 0, L);
        }
        if (!invert_small(U, h, Ui)) return false;
        put(k, 1, Ui);
        blockD(k, k - 1, Dc);
        matmul(Ui, Dc, X);
        put(k, 2, X);
        Vprev = Ui;
    }
    // middle: S = D_cc - L_c D_{c-1,c} - M_c D_{c+1,c}
    blockD(c, c, U);
    if (c > 0) {
        blockD(c, c - 1, Dc);
        matmul(Dc, Utop, Lc);
        blockD(c - 1, c, Dn);
        matmul(Lc, Dn, X);
        for (size_t i = 0; i < hh; ++i) U[i] -= X[i];
        put(c, 0, Lc);
    }
    if (c < nb - 1) {
        std::vector<T> Mc(hh);
        blockD(c, c + 1, Dn);
        matmul(Dn, Vprev, Mc);
        blockD(c + 1, c, Dc);
        matmul(Mc, Dc, X);
        for (size_t i = 0; i < hh; ++i) U[i] -= X[i];
        put(c, 2, Mc);
    }
    if (!invert_small(U, h, Ui)) return false;
    put(c, 1, Ui);
    return true;
}

void galerkin_gamma(int n, double g[5]) {
    const double x = (double)n;
    const double den = 2 * x * x * x * x + 20 * x * x * x + 78 * x * x + 140 * x + 95;
    const double q = x * x + 4 * x + 5;
    g[0] = 1.0;
    g[1] = 8 * (x + 1) * q / den;
    g[2] = -2 * (x + 2) * (2 * x * x * x * x + 16 * x * x * x + 58 * x * x + 104 * x + 75) / ((x + 3) * den);
    g[3] = -8 * (x + 1) * q / den;
    g[4] = (x + 1) * (2 * x * x * x * x + 12 * x * x * x + 30 * x * x + 36 * x + 15) / ((x + 3) * den);
}

template <class T>
bool band_lu_pivot(int n, int kl, int ku, const std::vector<T>& band, std::vector<T>& Lm, std::vector<T>& Ucol,
                   std::vector<unsigned char>& piv, std::vector<double>& rs) {
    // working rows of width 2 kl + ku + 1: row i holds columns i - kl .. i + kl + ku
    // (the last kl for the fill-in of the interchanges), W[i][c - i + kl]
    const int wb = kl + ku + 1, ww = 2 * kl + ku + 1, kk = kl + ku;
    std::vector<T> W((size_t)n * ww, T(0));
    rs.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double mx = 0.0;
        for (int d = 0; d < wb; ++d) mx = std::max(mx, std::abs(band[(size_t)i * wb + d]));
        if (!(mx > 0.0)) return false;
        rs[i] = 1.0 / mx;
        for (int d = 0; d < wb; ++d) W[(size_t)i * ww + d] = band[(size_t)i * wb + d] * rs[i];
    }
    auto at = [&](int i, int c) -> T& { return W[(size_t)i * ww + (c - i + kl)]; };
    Lm.assign((size_t)n * kl, T(0));
    piv.assign(n, 0);
    for (int j = 0; j < n; ++j) {
        const int last = std::min(n - 1, j + kl), cend = std::min(n - 1, j + kk);
        int p = j;
        double best = std::abs(at(j, j));
        for (int i = j + 1; i <= last; ++i)
            if (std::abs(at(i, j)) > best) {
                best = std::abs(at(i, j));
                p = i;
            }
        if (!(best > 0.0)) return false;
        piv[j] = (unsigned char)(p - j);
        if (p != j)
            for (int c = j; c <= cend; ++c) std::swap(at(j, c), at(p, c));
        const T d = at(j, j);
        for (int i = j + 1; i <= last; ++i) {
            const T l = at(i, j) / d;
            Lm[(size_t)j * kl + (i - j - 1)] = l;
            at(i, j) = T(0);
            for (int c = j + 1; c <= cend; ++c) at(i, c) -= l * at(j, c);
        }
    }
    Ucol.assign((size_t)n * (kk + 1), T(0));
    for (int i = 0; i < n; ++i) {
        const T rd = T(1) / at(i, i);
        Ucol[(size_t)i * (kk + 1)] = rd;
        for (int t = 1; t <= kk && i - t >= 0; ++t) Ucol[(size_t)i * (kk + 1) + t] = at(i - t, i) * rd;
    }
    return true;
}

template <class T>
void band_lu_pivot_solve(int n, int kl, int ku, const std::vector<T>& Lm, const std::vector<T>& Ucol,
                         const std::vector<unsigned char>& piv, const std::vector<double>& rs, T* b) {
    const int kk = kl + ku;
    for (int i = 0; i < n; ++i) b[i] *= rs[i];
    for (int j = 0; j < n; ++j) {  // L z = P b, the interchanges interleaved
        const int p = j + piv[j];
        if (p != j) std::swap(b[j], b[p]);
        for (int t = 0; t < kl && j + 1 + t < n; ++t) b[j + 1 + t] -= Lm[(size_t)j * kl + t] * b[j];
    }
    for (int i = n - 1; i >= 0; --i) {  // U x = z with U's columns divided by U_ii
        const T yi = b[i];
        for (int t = 1; t <= kk && i - t >= 0; ++t) b[i - t] -= Ucol[(size_t)i * (kk + 1) + t] * yi;
        b[i] = yi * Ucol[(size_t)i * (kk + 1)];
    }
}

template void band_lu_pivot_solve<cplx>(int, int, int, const std::vector<cplx>&, const std::vector<cplx>&,
                                        const std::vector<unsigned char>&, const std::vector<double>&, cplx*);
template void band_lu_pivot_solve<double>(int, int, int, const std::vector<double>&, const std::vector<double>&,
                                        const std::vector<unsigned char>&, const std::vector<double>&, double*);

template bool band_lu_pivot<double>(int, int, int, const std::vector<double>&, std::vector<double>&,
                                    std::vector<double>&, std::vector<unsigned char>&, std::vector<double>&);
template bool band_lu_pivot<cplx>(int, int, int, const std::vector<cplx>&, std::vector<cplx>&, std::vector<cplx>&,
                                  std::vector<unsigned char>&, std::vector<double>&);

template bool block_lu_twisted<double>(const std::vector<double>&, int, int, int, std::vector<double>&);
template bool block_lu_twisted<cplx>(const std::vector<cplx>&, int, int, int, std::vector<cplx>&);
template bool block_lu<double>(const std::vector<double>&, int, int, int, std::vector<double>&);
template bool block_lu<cplx>(const std::vector<cplx>&, int, int, int, std::vector<cplx>&);

template bool factor_bordered<double>(const std::vector<double>&, int, int, const std::vector<double>&, int,
                                      Bordered<double>&);
template bool factor_bordered<cplx>(const std::vector<cplx>&, int, int, const std::vector<double>&, int,
                                    Bordered<cplx>&);

}  // namespace pz
