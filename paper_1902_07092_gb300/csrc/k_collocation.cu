// Chebyshev-collocation formulation (Section 3.1 of Gastine, pizza, GJI 2019):
// explicit terms and implicit solves with every field held as its values on the
// Gauss-Lobatto grid.
//
// Layouts (double2 = complex):
//   state   omega_k, psi_k, theta_k  [M][n_r],  u_bar_k [n_r]  (grid values; psi_0 = 0)
//   rows    e / mass / imp vectors: vorticity rows (field w), temperature rows
//           (field th), zonal-flow rows (field u), [M][n_r]; rows 0 and n_r-1
//           are boundary rows and hold 0
//   G1, G2  as in the integration path: [n_r][4][M] with fields
//           (v, u_phi, omega, theta) and their products
// With v = d psi/d phi (u_s = v/s) the velocities are (Eq. vel_def)
//   u_phi = u_bar - d psi/ds - beta psi,  beta psi -> 0 at s_o where psi has a
//   double zero.
#include <algorithm>

#include "device_common.cuh"

namespace pz {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int g_index(int k, int f, int m, int M) { return (k * 4 + f) * M + m; }

__host__ __device__ inline int coll_batch(int L) { return L <= 1024 ? 2 : 1; }

// Plain Chebyshev coefficients c_n (f = sum_n c_n T_n) of the grid values held in
// the even-extension FFT result Z: c_n = w_n Z_n / K, w = 1/2 at n = 0, K.
__device__ __forceinline__ void plain_from_fft(const double2* Z, double2* c, int K) {
    const double inv = 1.0 / (double)K;
    for (int n = threadIdx.x; n <= K; n += blockDim.x)
        c[n] = cscale(Z[n], (n == 0 || n == K) ? 0.5 * inv : inv);
}

// even extension of plain coefficients for synthesis: values = Z/2
__device__ __forceinline__ void load_plain_for_synthesis(double2* z, const double2* c, int K) {
    for (int j = threadIdx.x; j <= K; j += blockDim.x) {
        double2 v = c[j];
        if (j == 0 || j == K) v = cscale(v, 2.0);
        even_extend_store(z, K, j, v);
    }
}

// ---------------------------------------------------------------------------
// K1c: per m, grid fields -> G1.
//   m >= 1: v = i m psi, u_phi = -psi' - beta psi, omega, theta
//   m = 0:  v = 0, u_phi = u_bar, omega = u_bar' + u_bar/s, theta_0
// psi' (or u_bar') is the derivative of the n_r-point interpolant: Eq. icheb by
// the DCT-I, the derivative recurrence, Eq. cheb.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_coll_spec_to_grid(StepParams P, VecSet y, double2* __restrict__ G1) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, M = P.M;
    double2* bufA = sm;
    double2* bufB = bufA + L;
    double2* cc0 = bufB + L;
    double2* cc1 = cc0 + N;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double2* f = y.psi + (size_t)m * N;

    for (int j = tid; j <= K; j += nth) {
        const double2 v = (m > 0) ? f[j] : make_double2(y.u[j], 0.0);
        even_extend_store(bufA, K, j, v);
    }
    double2* R = radial_dct1(bufA, bufB, P, 1);
    plain_from_fft(R, cc0, K);
    __syncthreads();
    cheb_derivative_scan(cc0, cc1, bufA, N, P.inv_a);
    load_plain_for_synthesis(bufA, cc1, K);
    R = radial_dct1(bufA, bufB, P, 1);
    const double dm = (double)m;
    for (int k = tid; k < N; k += nth) {
        const double2 d = cscale(R[k], 0.5);
        double2* out = G1 + g_index(k, 0, m, M);
        if (m > 0) {
            const double2 p = f[k];
            out[0] = cmul_i(p, dm);
            out[M] = csub(cscale(p, -P.beta[k]), d);
            out[2 * M] = y.w[(size_t)m * N + k];
            out[3 * M] = y.th[(size_t)m * N + k];
        } else {
            const double u = y.u[k];
            out[0] = make_double2(0.0, 0.0);
            out[M] = make_double2(u, 0.0);
            out[2 * M] = make_double2(d.x + u * P.inv_s[k], 0.0);
            out[3 * M] = y.th[k];
        }
    }
}

// ---------------------------------------------------------------------------
// K3c: per m, flux divergences and explicit rows on the grid (interior points):
//   N_omega = (1/s) d[v omega]_m/ds + (i m/s)[u_phi omega]_m
//   N_theta = (1/s) d[v theta]_m/ds + (i m/s)[u_phi theta]_m + (beta/s)[v theta]_m
//   e_omega = -(Ra/Pr)(i m/s_o) theta_m - N_omega                       (m >= 1)
//   e_theta = -(i m/s) dT_c/ds psi_m - N_theta = -(tc/s^2) v_m - N_theta
//   e_u     = -[v omega]_0 / s                                          (m = 0)
// (Eqs. psiomcoll, tempcoll, uphicoll; dT_c/ds = tc/s with tc = alpha/ln eta; the
// conduction term is -u_s dT_c/ds as in Eq. temp.)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_coll_grid_rows(StepParams P, const double2* __restrict__ G1,
                                                       const double2* __restrict__ G2, VecSet e) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, M = P.M;
    const int NB = coll_batch(L);
    double2* bufA = sm;
    double2* bufB = bufA + NB * L;
    double2* cc0 = bufB + NB * L;
    double2* cc1 = cc0 + N;
    double2* cc2 = cc1 + N;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double dm = (double)m;

    // plain coefficients of F0 = [v omega]_m (-> cc0) and F1 = [v theta]_m (-> cc1)
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b) {
            const int f = (b0 + b == 0) ? 0 : 2;
            for (int j = tid; j <= K; j += nth) even_extend_store(bufA + b * L, K, j, G2[g_index(j, f, m, M)]);
        }
        double2* R = radial_dct1(bufA, bufB, P, nb);
        for (int b = 0; b < nb; ++b) plain_from_fft(R + b * L, (b0 + b == 0) ? cc0 : cc1, K);
        __syncthreads();
    }
    cheb_derivative_scan(cc0, cc2, bufA, N, P.inv_a);
    for (int n = tid; n < N; n += nth) cc0[n] = cc2[n];
    __syncthreads();
    cheb_derivative_scan(cc1, cc2, bufA, N, P.inv_a);
    for (int n = tid; n < N; n += nth) cc1[n] = cc2[n];
    __syncthreads();
    // derivative values: d F0 -> cc2, d F1 -> cc0 (cc0 is consumed before it is overwritten)
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b) load_plain_for_synthesis(bufA + b * L, (b0 + b == 0) ? cc0 : cc1, K);
        double2* R = radial_dct1(bufA, bufB, P, nb);
        for (int b = 0; b < nb; ++b) {
            double2* dst = (b0 + b == 0) ? cc2 : cc0;
            for (int k = tid; k < N; k += nth) dst[k] = cscale(R[b * L + k], 0.5);
        }
        __syncthreads();
    }
    const double bfac = P.Ra / P.Pr * dm / P.s_o;
    for (int k = tid; k < N; k += nth) {
        double2 ew = make_double2(0.0, 0.0), et = make_double2(0.0, 0.0);
        double eu = 0.0;
        if (k > 0 && k < N - 1) {
            const double is = P.inv_s[k];
            const double2 vw = G2[g_index(k, 0, m, M)], uw = G2[g_index(k, 1, m, M)];
            const double2 vt = G2[g_index(k, 2, m, M)], ut = G2[g_index(k, 3, m, M)];
            const double2 nt = cscale(cadd(cadd(cc0[k], cmul_i(ut, dm)), cscale(vt, P.beta[k])), is);
            if (m > 0) {
                const double2 nw = cscale(cadd(cc2[k], cmul_i(uw, dm)), is);
                const double2 th = G1[g_index(k, 3, m, M)], v = G1[g_index(k, 0, m, M)];
                ew = P.buoy_imp ? cscale(nw, -1.0) : csub(cmul_i(th, -bfac), nw);
                et = csub(cscale(v, -P.tc * is * is), nt);
            } else {
                et = cscale(nt, -1.0);
                eu = -vw.x * is;
                // self-interaction of the zonal wind with Ekman pumping (Eq. uphicoll)
                if (P.pump)
                    eu -= 0.5 * P.E * P.pump_ups[k] * G1[g_index(k, 1, 0, M)].x * G1[g_index(k, 2, 0, M)].x;
            }
        }
        e.w[(size_t)m * N + k] = ew;
        e.th[(size_t)m * N + k] = et;
        if (m == 0) e.u[k] = eu;
    }
}

// ---------------------------------------------------------------------------
// Implicit solve: right-hand side r = sum_t c_t V_t on the interior rows, then
// the grid values of the solution x = G r with the precomputed inverse columns,
// stored column-major so that one thread owns one output row and a warp reads
// 32 consecutive entries of a column: colW [M][n_r-2][2 n_r] (omega, psi; complex),
// colT [M][n_r-2][n_r] and colU [n_r-2][n_r] (real).  r sits in shared memory and
// is broadcast.  With the mass term equal to the field itself, the implicit term
// of the new state follows from its own equation:  imp = (x - r)/(gamma dt).
// Grid (M, RB): CTA (m, rb) owns rows rb*blockDim .. of mode m; rows of m >= 1
// are omega (n_r), psi (n_r), theta (n_r); of m = 0 theta (n_r), u_bar (n_r).
// No output vector may alias an input term.
// ---------------------------------------------------------------------------
// With implicit buoyancy the solve runs in two launches: phase 1 the temperature
// and zonal-flow rows, phase 2 the vorticity and streamfunction rows, whose
// right-hand side gains g (-(Ra/Pr)(i m/s_o)) theta_new at the interior points
// (the implicit term of the new state still uses the original right-hand side).
// phase 0: all rows at once (explicit buoyancy).
__global__ void __launch_bounds__(NT) k_coll_solve(StepParams P, RhsSpec R, DevFactors F, VecSet yo, VecSet mo,
                                                   VecSet io, int want_mass, int want_imp, int phase) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int N = P.n_r, ni = N - 2;
    double2* rw = sm;       // interior vorticity rows (m >= 1) or zonal rows (m = 0, real part)
    double2* rt = rw + ni;  // interior temperature rows
    double2* rg = rt + ni;  // phase 2: vorticity rows with the new temperature's buoyancy
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int j = tid; j < ni; j += nth) {
        const size_t idx = (size_t)m * N + j + 1;
        double2 aw = make_double2(0.0, 0.0), at = make_double2(0.0, 0.0);
        for (int t = 0; t < R.nterms; ++t) {
            const double c = R.t[t].c;
            const VecSet& v = R.t[t].v;
            if (m > 0) {
                const double2 x = v.w[idx];
                aw.x = fma(c, x.x, aw.x);
                aw.y = fma(c, x.y, aw.y);
            } else {
                aw.x = fma(c, v.u[j + 1], aw.x);
            }
            const double2 x = v.th[idx];
            at.x = fma(c, x.x, at.x);
            at.y = fma(c, x.y, at.y);
        }
        rw[j] = aw;
        rt[j] = at;
        if (phase == 2 && m > 0)
            rg[j] = cadd(aw, cmul_i(yo.th[idx], -F.gdt * P.Ra / P.Pr * (double)m / P.s_o));
    }
    __syncthreads();
    const int row = blockIdx.y * nth + tid;
    const int nrows = (m > 0) ? 3 * N : 2 * N;
    const double igdt = 1.0 / F.gdt;
    if (m == 0 && row < N && phase != 2) {
        yo.w[row] = make_double2(0.0, 0.0);
        yo.psi[row] = make_double2(0.0, 0.0);
        if (want_mass) mo.w[row] = make_double2(0.0, 0.0);
        if (want_imp) io.w[row] = make_double2(0.0, 0.0);
    }
    if (row >= nrows) return;
    // field: 0 omega, 1 psi, 2 theta, 3 u_bar
    int fld, k;
    if (m > 0) {
        fld = row / N;
        k = row - fld * N;
    } else {
        fld = (row < N) ? 2 : 3;
        k = (row < N) ? row : row - N;
    }
    if ((phase == 1 && fld <= 1) || (phase == 2 && fld >= 2)) return;
    const double2* rwg = (phase == 2) ? rg : rw;  // the right-hand side the inverse acts on
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    if (fld <= 1) {
        const int ld = 2 * N;
        const double2* g = F.colW + (size_t)m * ni * ld + row;
        int j = 0;
        for (; j + 1 < ni; j += 2) {
            a0 = cfma(__ldg(&g[(size_t)j * ld]), rwg[j], a0);
            a1 = cfma(__ldg(&g[(size_t)(j + 1) * ld]), rwg[j + 1], a1);
        }
        if (j < ni) a0 = cfma(__ldg(&g[(size_t)j * ld]), rwg[j], a0);
    } else {
        const double* g = (fld == 2) ? F.colT + (size_t)m * ni * N + k : F.colU + k;
        const double2* r = (fld == 2) ? rt : rw;
        int j = 0;
        for (; j + 1 < ni; j += 2) {
            const double b0 = __ldg(&g[(size_t)j * N]), b1 = __ldg(&g[(size_t)(j + 1) * N]);
            a0.x = fma(b0, r[j].x, a0.x);
            a0.y = fma(b0, r[j].y, a0.y);
            a1.x = fma(b1, r[j + 1].x, a1.x);
            a1.y = fma(b1, r[j + 1].y, a1.y);
        }
        if (j < ni) {
            const double b0 = __ldg(&g[(size_t)j * N]);
            a0.x = fma(b0, r[j].x, a0.x);
            a0.y = fma(b0, r[j].y, a0.y);
        }
    }
    const double2 acc = cadd(a0, a1);
    const size_t idx = (size_t)m * N + k;
    const bool interior = (k > 0 && k < N - 1);
    if (fld == 1) {
        yo.psi[idx] = interior ? acc : make_double2(0.0, 0.0);
    } else if (fld == 0) {
        yo.w[idx] = acc;
        if (want_mass) mo.w[idx] = acc;
        if (want_imp) io.w[idx] = interior ? cscale(csub(acc, rw[k - 1]), igdt) : make_double2(0.0, 0.0);
    } else if (fld == 2) {
        yo.th[idx] = acc;
        if (want_mass) mo.th[idx] = acc;
        if (want_imp) io.th[idx] = interior ? cscale(csub(acc, rt[k - 1]), igdt) : make_double2(0.0, 0.0);
    } else {
        yo.u[k] = acc.x;
        if (want_mass) mo.u[k] = acc.x;
        if (want_imp) io.u[k] = interior ? (acc.x - rw[k - 1].x) * igdt : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Implicit terms of a grid state with the dense differentiation matrices (used
// once when a state is set, for the schemes that need I(y_n)):
//   omega rows: D2 omega + D1 omega/s - m^2 omega/s^2 + (2/E)(i m beta/s) psi
//   theta rows: (D2 theta + D1 theta/s - m^2 theta/s^2)/Pr
//   u rows:     D2 u + D1 u/s - u/s^2;   boundary rows 0.
// With Ekman pumping (Eqs. pumping_full, uphicoll) the omega rows gain
//   -U omega - (U beta/2) psi' + U (-beta^2/2 + beta m^2/s + i m c5) psi
// and the u rows -U u  (U = Upsilon, c5 = 5 s_o beta/(2 h s)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_coll_apply(StepParams P, VecSet y, VecSet io) {
    const int m = blockIdx.x, N = P.n_r;
    const double mu = (double)m * m;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const size_t idx = (size_t)m * N + k;
        double2 iw = make_double2(0.0, 0.0), it = make_double2(0.0, 0.0);
        double iu = 0.0;
        if (k > 0 && k < N - 1) {
            const double is = P.inv_s[k];
            const double* d1 = P.cD1 + (size_t)k * N;
            const double* d2 = P.cD2 + (size_t)k * N;
            double2 w1 = make_double2(0.0, 0.0), w2 = w1, t1 = w1, t2 = w1, p1 = w1;
            double u1 = 0.0, u2 = 0.0;
            for (int j = 0; j < N; ++j) {
                const double a = d1[j], b = d2[j];
                const double2 th = y.th[(size_t)m * N + j];
                t1.x = fma(a, th.x, t1.x); t1.y = fma(a, th.y, t1.y);
                t2.x = fma(b, th.x, t2.x); t2.y = fma(b, th.y, t2.y);
                if (m > 0) {
                    const double2 w = y.w[(size_t)m * N + j];
                    w1.x = fma(a, w.x, w1.x); w1.y = fma(a, w.y, w1.y);
                    w2.x = fma(b, w.x, w2.x); w2.y = fma(b, w.y, w2.y);
                    if (P.pump) {
                        const double2 ps = y.psi[(size_t)m * N + j];
                        p1.x = fma(a, ps.x, p1.x); p1.y = fma(a, ps.y, p1.y);
                    }
                } else {
                    u1 = fma(a, y.u[j], u1);
                    u2 = fma(b, y.u[j], u2);
                }
            }
            const double2 th = y.th[idx];
            it = cscale(csub(cadd(t2, cscale(t1, is)), cscale(th, mu * is * is)), 1.0 / P.Pr);
            if (m > 0) {
                const double2 w = y.w[idx];
                iw = csub(cadd(w2, cscale(w1, is)), cscale(w, mu * is * is));
                iw = cadd(iw, cmul_i(y.psi[idx], 2.0 / P.E * (double)m * P.beta[k] * is));
                if (P.buoy_imp)  // -(Ra/Pr)(i m/s_o) theta
                    iw = cadd(iw, cmul_i(y.th[idx], -P.Ra / P.Pr * (double)m / P.s_o));
                if (P.pump) {
                    const double U = P.pump_ups[k], b = P.beta[k];
                    const double2 ps = y.psi[idx];
                    iw = csub(iw, cscale(w, U));
                    iw = csub(iw, cscale(p1, 0.5 * U * b));
                    iw = cadd(iw, cscale(ps, U * (-0.5 * b * b + b * mu * is)));
                    iw = cadd(iw, cmul_i(ps, U * (double)m * P.pump_ci[k]));
                }
            } else {
                iu = u2 + u1 * is - y.u[k] * is * is;
                if (P.pump) iu -= P.pump_ups[k] * y.u[k];
            }
        }
        io.w[idx] = iw;
        io.th[idx] = it;
        if (m == 0) io.u[k] = iu;
    }
}

// ---------------------------------------------------------------------------
// Paper coefficients -> grid state: f_k = sum_n T_kn f_hat_n (Eq. cheb, N_c = n_r)
// and omega = -L_beta psi (Eq. psi) with the limit (5/4) psi'' of L_beta psi at
// s_o, where psi = dpsi/ds = 0.  In: hat.psi, hat.th [M][n_r], hat.u [n_r].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_coll_from_hat(StepParams P, VecSet hat, VecSet y) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x, N = P.n_r;
    double2* pg = sm;  // psi grid values
    const double mu = (double)m * m;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double* t = P.cTm + (size_t)k * N;
        double2 p = make_double2(0.0, 0.0), th = p;
        double u = 0.0;
        for (int n = 0; n < N; ++n) {
            const double a = t[n];
            const double2 h = hat.th[(size_t)m * N + n];
            th.x = fma(a, h.x, th.x);
            th.y = fma(a, h.y, th.y);
            if (m > 0) {
                const double2 q = hat.psi[(size_t)m * N + n];
                p.x = fma(a, q.x, p.x);
                p.y = fma(a, q.y, p.y);
            } else {
                u = fma(a, hat.u[n], u);
            }
        }
        pg[k] = p;
        y.th[(size_t)m * N + k] = th;
        y.psi[(size_t)m * N + k] = p;
        if (m == 0) y.u[k] = u;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double2 w = make_double2(0.0, 0.0);
        if (m > 0) {
            const double* d1 = P.cD1 + (size_t)k * N;
            const double* d2 = P.cD2 + (size_t)k * N;
            double2 p1 = make_double2(0.0, 0.0), p2 = p1;
            for (int j = 0; j < N; ++j) {
                p1.x = fma(d1[j], pg[j].x, p1.x); p1.y = fma(d1[j], pg[j].y, p1.y);
                p2.x = fma(d2[j], pg[j].x, p2.x); p2.y = fma(d2[j], pg[j].y, p2.y);
            }
            if (k == 0) {
                w = cscale(p2, -1.25);
            } else {
                const double is = P.inv_s[k], b = P.beta[k];
                w = cadd(p2, cscale(p1, b + is));
                w = cadd(w, cscale(pg[k], P.dbeta[k] + b * is - mu * is * is));
                w = cscale(w, -1.0);
            }
        }
        y.w[(size_t)m * N + k] = w;
    }
}

// grid state -> paper coefficients (Eq. icheb; with N_c = n_r the synthesis
// matrix T is an involution, f_hat_n = sum_k T_nk f_k):
// out.psi, out.th, out.w [M][n_r], out.u [n_r]
__global__ void __launch_bounds__(NT) k_coll_to_hat(StepParams P, VecSet y, VecSet out) {
    const int m = blockIdx.x, N = P.n_r;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double* t = P.cTm + (size_t)n * N;
        double2 p = make_double2(0.0, 0.0), th = p, w = p;
        double u = 0.0;
        for (int k = 0; k < N; ++k) {
            const double a = t[k];
            const size_t idx = (size_t)m * N + k;
            th.x = fma(a, y.th[idx].x, th.x);
            th.y = fma(a, y.th[idx].y, th.y);
            if (m > 0) {
                p.x = fma(a, y.psi[idx].x, p.x);
                p.y = fma(a, y.psi[idx].y, p.y);
                w.x = fma(a, y.w[idx].x, w.x);
                w.y = fma(a, y.w[idx].y, w.y);
            } else {
                u = fma(a, y.u[k], u);
            }
        }
        out.th[(size_t)m * N + n] = th;
        out.psi[(size_t)m * N + n] = p;
        out.w[(size_t)m * N + n] = w;
        if (m == 0) out.u[n] = u;
    }
}

}  // namespace

size_t smem_coll_spec_to_grid(const StepParams& P) { return sizeof(double2) * (2 * 2 * P.K + 2 * P.n_r); }
size_t smem_coll_grid_rows(const StepParams& P) {
    const int L = 2 * P.K;
    return sizeof(double2) * (2 * coll_batch(L) * L + 3 * P.n_r);
}

cudaError_t launch_coll_spec_to_grid(const StepParams& P, VecSet y, double2* G1, cudaStream_t st) {
    const size_t sm = smem_coll_spec_to_grid(P);
    cudaError_t err = cudaFuncSetAttribute(k_coll_spec_to_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_coll_spec_to_grid<<<P.M, NT, sm, st>>>(P, y, G1);
    return cudaGetLastError();
}

cudaError_t launch_coll_grid_rows(const StepParams& P, const double2* G1, const double2* G2, VecSet e,
                                  cudaStream_t st) {
    const size_t sm = smem_coll_grid_rows(P);
    cudaError_t err = cudaFuncSetAttribute(k_coll_grid_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_coll_grid_rows<<<P.M, NT, sm, st>>>(P, G1, G2, e);
    return cudaGetLastError();
}

cudaError_t launch_coll_solve(const StepParams& P, const RhsSpec& R, const DevFactors& F, VecSet y_out,
                              VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp, cudaStream_t st) {
    const size_t sm = sizeof(double2) * 3 * (P.n_r - 2);
    dim3 grid(P.M, (3 * P.n_r + NT - 1) / NT);
    for (int phase = P.buoy_imp ? 1 : 0; phase <= (P.buoy_imp ? 2 : 0); ++phase) {
        k_coll_solve<<<grid, NT, sm, st>>>(P, R, F, y_out, mass_out, imp_out, want_mass ? 1 : 0, want_imp ? 1 : 0,
                                           phase);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_coll_apply(const StepParams& P, VecSet y, VecSet imp_out, cudaStream_t st) {
    k_coll_apply<<<P.M, NT, 0, st>>>(P, y, imp_out);
    return cudaGetLastError();
}

cudaError_t launch_coll_from_hat(const StepParams& P, VecSet hat, VecSet y, cudaStream_t st) {
    const size_t sm = sizeof(double2) * P.n_r;
    k_coll_from_hat<<<P.M, NT, sm, st>>>(P, hat, y);
    return cudaGetLastError();
}

cudaError_t launch_coll_to_hat(const StepParams& P, VecSet y, VecSet out, cudaStream_t st) {
    k_coll_to_hat<<<P.M, NT, 0, st>>>(P, y, out);
    return cudaGetLastError();
}

}  // namespace pz
