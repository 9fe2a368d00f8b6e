// Discrete adjoint of the Chebyshev-integration time step (Sections 3.2 and 4 of
// Gastine, pizza, GJI 2019): the explicit stage taken backwards, the transposed
// tau solve and the transposed mass/implicit operators, for the reverse sweep of
// a CNAB2 run (the derivation is in include/pizza.h, pizza_adjoint_step).
//
// Inner product: Re sum conj(a) b over the stored arrays.  Each kernel applies
// the adjoint of one forward stage:
//   k_adj_grid_to_spec   adjoint of k_grid_to_spec: C^T, D^T, G^T (conjugated
//                        where complex), zero padding, the transpose of Eq. icheb,
//                        the transposed flux divergences -> adjoints of the
//                        product spectra (G2 layout)
//   k_adj_phi            adjoint of k_phi_products: the forward fields and the
//                        product adjoints on the azimuthal grid, the product
//                        rule, back to spectra -> adjoints of (v, u_phi, omega,
//                        theta) (G1 layout)
//   k_adj_spec_to_grid   adjoint of k_spec_to_grid: transposed Chebyshev synthesis
//                        and derivative recurrences -> adjoint of the state
//   k_adj_solve          rho = P S^{-H} lambda with precomputed dense inverses
//   k_adj_apply          lambda = g + (Mass + (dt/2) Lin)^H rho and the weight
//                        w = dt (c rho_n + c' rho_{n+1}) of the explicit adjoint
// Only the real parts of the m = 0 spectra enter the forward grid fields, and
// the adjoints keep that.
#include "device_common.cuh"

namespace pz {

namespace {

constexpr int NTA = 256;
constexpr int MAXPER_A = 12;  // azimuthal points per thread (n_phi <= 3072)

__device__ __forceinline__ int g_index(int k, int f, int m, int M) { return (k * 4 + f) * M + m; }

// radial transforms per shared-memory pass: the analysis adjoint has pairs, the
// synthesis adjoint four fields (one pass up to n_r = 513)
__host__ __device__ inline int adj_batch(int L) { return L <= 1024 ? 2 : 1; }
__host__ __device__ inline int adj_batch4(int L) { return L <= 1024 ? 4 : 1; }

// (X^T x)_n for a band operator stored transposed (row n of X^T, half width H)
template <int H>
__device__ __forceinline__ double2 bandT_row(const double* __restrict__ bandT, const double2* x, int n, int nc) {
    const double* row = bandT + (size_t)n * (2 * H + 1);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int d = 0; d <= 2 * H; ++d) {
        const int k = n - H + d;
        if (k >= 0 && k < nc) {
            const double c = __ldg(&row[d]);
            acc.x = fma(c, x[k].x, acc.x);
            acc.y = fma(c, x[k].y, acc.y);
        }
    }
    return acc;
}

template <int H>
__device__ __forceinline__ double bandT_row_r(const double* __restrict__ bandT, const double* x, int n, int nc) {
    const double* row = bandT + (size_t)n * (2 * H + 1);
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d <= 2 * H; ++d) {
        const int k = n - H + d;
        if (k >= 0 && k < nc) acc = fma(__ldg(&row[d]), x[k], acc);
    }
    return acc;
}

// sum_k cos(pi n k/K) a_k for n = 0..K of nb vectors a (length K+1 each, in src
// with stride K+1): the DCT-I of the even extension with the end values doubled,
// Z_n = 2 sum''_k z_k cos(...) = 2 sum_k a_k cos(...) (the half-length transform
// where the forward stage uses it).  Results are Z/2 into dst (stride K+1).
// bufA, bufB: nb*2K scratch, nb <= 4.
__device__ void cos_sums(const double2* src, double2* dst, int nb, double2* bufA, double2* bufB, const StepParams& P) {
    const int K = P.K, L = 2 * K;
    for (int b = 0; b < nb; ++b)
        for (int j = threadIdx.x; j <= K; j += blockDim.x) {
            double2 v = src[b * (K + 1) + j];
            if (j == 0 || j == K) v = cscale(v, 2.0);
            even_extend_store(bufA + b * L, K, j, v);
        }
    double2* R = radial_dct1(bufA, bufB, P, nb);
    for (int b = 0; b < nb; ++b)
        for (int n = threadIdx.x; n <= K; n += blockDim.x) dst[b * (K + 1) + n] = cscale(R[b * L + n], 0.5);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// adjoint of k_grid_to_spec, per m.  w: adjoint of (e_psi, e_theta, e_u).
//   q = C^T w_psi;  Nw_hat_bar = q;  lam_theta += conj((Ra/Pr)(i m/s_o)) q
//   Nt_hat_bar = -D^T w_theta;  lam_psi += conj(-tc i m) G^T w_theta
//   Nu_hat_bar = -D^T w_u  (m = 0)
// then the grid adjoints f_bar_k = C w'_k sum_n cos(pi n k/K) f_hat_bar_n (the
// transpose of Eq. icheb; w' halves k = 0, K), and with a = N_bar/s and
// Dg^T = Ana^T Dc^T Syn^T (Dg the radial derivative of the interpolant):
//   [v omega]_bar = h^2 Dg^T a_omega  (m = 0: (h^2/s) Re Nu_bar)
//   [u omega]_bar = -i m a_omega
//   [v theta]_bar = h^2 Dg^T a_theta - Nt_bar,  [u theta]_bar = -i m a_theta
// ra[m] = sum_n Re(conj(q_n) (i m/(Pr s_o)) theta_hat_n)  (dE/dRa term).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTA) k_adj_grid_to_spec(StepParams P, VecSet w, VecSet y, VecSet lam,
                                                          double2* __restrict__ Gb2, double* __restrict__ ra) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, nc = P.nc, M = P.M;
    const int NB = adj_batch(L);
    double2* bufA = sm;
    double2* bufB = bufA + NB * L;
    double2* c0 = bufB + NB * L;  // [2][N]: Nw_hat_bar (or Nu_hat_bar), Nt_hat_bar; then grid adjoints
    double2* c1 = c0 + N;
    double2* c2 = c1 + N;         // [2][N] work
    double2* c3 = c2 + N;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double dm = (double)m;
    const double2* wp = w.psi + (size_t)m * nc;
    const double2* wt = w.th + (size_t)m * nc;
    __shared__ double red[32];
    double rpart = 0.0;
    for (int n = tid; n < N; n += nth) {
        double2 nw = make_double2(0.0, 0.0), nt = make_double2(0.0, 0.0);
        if (n < nc) {
            if (m > 0) {
                const double2 q = bandT_row<8>(P.ops.bandT[OP_C], wp, n, nc);
                nw = q;
                const double2 th = y.th[(size_t)m * nc + n];
                lam.th[(size_t)m * nc + n] = cadd(lam.th[(size_t)m * nc + n], cmul_i(q, -P.Ra / P.Pr * dm / P.s_o));
                rpart += dm / (P.Pr * P.s_o) * (q.y * th.x - q.x * th.y);
                const double2 gt = bandT_row<4>(P.ops.bandT[OP_G], wt, n, nc);
                lam.psi[(size_t)m * nc + n] = cadd(lam.psi[(size_t)m * nc + n], cmul_i(gt, P.tc * dm));
            } else {
                nw = make_double2(-bandT_row_r<4>(P.ops.bandT[OP_D], w.u, n, nc), 0.0);
            }
            nt = cscale(bandT_row<4>(P.ops.bandT[OP_D], wt, n, nc), -1.0);
        }
        c0[n] = nw;
        c1[n] = nt;
    }
    for (int o = 16; o > 0; o >>= 1) rpart += __shfl_xor_sync(0xffffffffu, rpart, o);
    if ((tid & 31) == 0) red[tid >> 5] = rpart;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int i = 0; i < (nth >> 5); ++i) a += red[i];
        ra[m] = a;
    }
    // grid adjoints: f_bar_k = C w'_k sum_n cos(pi n k/K) f_hat_bar_n  -> c0, c1
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        cos_sums(c0 + b0 * N, c0 + b0 * N, nb, bufA, bufB, P);
    }
    for (int k = tid; k < N; k += nth) {
        const double f = P.cnorm * ((k == 0 || k == K) ? 0.5 : 1.0);
        c0[k] = cscale(c0[k], f);
        c1[k] = cscale(c1[k], f);
        // a = N_bar / s into c2, c3
        c2[k] = cscale(c0[k], P.inv_s[k]);
        c3[k] = cscale(c1[k], P.inv_s[k]);
    }
    __syncthreads();
    // Dg^T a = Ana^T Dc^T Syn^T a for a in (c2, c3) (m = 0: only the theta field)
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        cos_sums(c2 + b0 * N, c2 + b0 * N, nb, bufA, bufB, P);  // Syn^T
    }
    // Dc^T of both, then the Ana^T weights 2 w_n/K (the scans side by side, in place)
    cheb_derivative_adjoint_scan2(c2, bufA, c3, bufB, N, P.inv_a, 2.0 / (double)K);
    // Ana^T: sum''_n ... with the ends halved: the even extension already counts
    // the end values once, so load without doubling
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b)
            for (int j = tid; j <= K; j += nth) even_extend_store(bufA + b * L, K, j, c2[(b0 + b) * N + j]);
        double2* R = radial_dct1(bufA, bufB, P, nb);
        for (int b = 0; b < nb; ++b)
            for (int k = tid; k <= K; k += nth) {
                const double wk = (k == 0 || k == K) ? 0.5 : 1.0;
                c2[(b0 + b) * N + k] = cscale(R[b * L + k], 0.5 * wk);
            }
        __syncthreads();
    }
    for (int k = tid; k < N; k += nth) {
        const double h2 = P.h2[k], is = P.inv_s[k];
        double2* out = Gb2 + g_index(k, 0, m, M);
        if (m > 0) {
            out[0] = cscale(c2[k], h2);
            out[M] = cmul_i(cscale(c0[k], is), -dm);
        } else {
            out[0] = make_double2(h2 * is * c0[k].x, 0.0);
            out[M] = make_double2(0.0, 0.0);
        }
        out[2 * M] = csub(cscale(c3[k], h2), c1[k]);
        out[3 * M] = cmul_i(cscale(c1[k], is), -dm);
    }
}

// ---------------------------------------------------------------------------
// adjoint of k_phi_products, per radius.  Forward fields f (v, u_phi, omega,
// theta) on the azimuthal grid from G1; product adjoints
//   p_bar_j = (1/n_phi) Re sum_{m=0}^{N_m} P_bar_m e^{i m phi_j}
// (the transpose of Eq. ifft restricted to m <= N_m); the product rule
//   v_bar = omega p_vw + theta p_vt,  u_bar = omega p_uw + theta p_ut,
//   omega_bar = v p_vw + u p_uw,  theta_bar = v p_vt + u p_ut;
// and the transpose of Eq. fft: F_bar_0 = sum_j f_bar_j, F_bar_m = 2 sum_j
// f_bar_j e^{-i m phi_j} (m >= 1).  smem: two work buffers and the two packed
// forward fields (4 n_phi complex).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_hermitian_pair(double2* Z, const double2* __restrict__ src, int M, int Pn,
                                                    int n_m, double s0, double s1) {
    // z = a + i b from one-sided spectra a = src[0..M), b = src[M..2M): a_0, b_0
    // real parts scaled by s0; m >= 1 scaled by s1 with the conjugate images
    for (int j = threadIdx.x; j < Pn; j += blockDim.x) {
        double2 z = make_double2(0.0, 0.0);
        if (j == 0) {
            z = make_double2(s0 * src[0].x, s0 * src[M].x);
        } else if (j <= n_m) {
            const double2 a = cscale(src[j], s1), b = cscale(src[M + j], s1);
            z = make_double2(a.x - b.y, a.y + b.x);
        } else if (j >= Pn - n_m) {
            const int mm = Pn - j;
            const double2 a = cscale(src[mm], s1), b = cscale(src[M + mm], s1);
            z = make_double2(a.x + b.y, -a.y + b.x);
        }
        Z[j] = z;
    }
}

__device__ __forceinline__ void store_split_adjoint(const double2* Y, double2* __restrict__ dst, int M, int Pn,
                                                    int n_m) {
    // a + i b on the grid -> F_bar_0 = sum_j (real), F_bar_m = 2 sum_j e^{-i m phi_j}
    for (int m = threadIdx.x; m <= n_m; m += blockDim.x) {
        double2 a, b;
        if (m == 0) {
            a = make_double2(Y[0].x, 0.0);
            b = make_double2(Y[0].y, 0.0);
        } else {
            const double2 y1 = Y[m], y2 = Y[Pn - m];
            a = make_double2(y1.x + y2.x, y1.y - y2.y);
            b = make_double2(y1.y + y2.y, -(y1.x - y2.x));
        }
        dst[m] = a;
        dst[M + m] = b;
    }
}

__global__ void __launch_bounds__(NTA, 1) k_adj_phi(StepParams P, const double2* __restrict__ G1,
                                                    const double2* __restrict__ Gb2, double2* __restrict__ Gb1,
                                                    int pair) {
    extern __shared__ double2 sm[];
    const int k = blockIdx.x;
    const int Pn = P.n_phi, M = P.M, n_m = P.n_m;
    double2* X = sm;
    double2* Y = X + Pn;
    double2* F1 = Y + Pn;  // v + i u_phi on the grid
    double2* F2 = F1 + Pn; // omega + i theta
    const int tid = threadIdx.x, nth = blockDim.x;
    if (pair) {
        // the three pairs of independent transforms batched (X, Y hold 2 Pn each):
        // half the barrier-separated passes, the same arithmetic per transform
        Y = X + 2 * Pn;
        F1 = Y + 2 * Pn;
        F2 = F1 + Pn;
        load_hermitian_pair(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, 1.0, 1.0);
        load_hermitian_pair(X + Pn, G1 + g_index(k, 2, 0, M), M, Pn, n_m, 1.0, 1.0);
        double2* R = fft_batched<+1>(X, Y, P.plan_p, 2);
        for (int j = tid; j < Pn; j += nth) {
            F1[j] = R[j];
            F2[j] = R[Pn + j];
        }
        __syncthreads();
        const double ip = 1.0 / (double)Pn;
        load_hermitian_pair(X, Gb2 + g_index(k, 0, 0, M), M, Pn, n_m, ip, 0.5 * ip);
        load_hermitian_pair(X + Pn, Gb2 + g_index(k, 2, 0, M), M, Pn, n_m, ip, 0.5 * ip);
        R = fft_batched<+1>(X, Y, P.plan_p, 2);
        double2* O = (R == X) ? Y : X;
        for (int j = tid; j < Pn; j += nth) {
            const double2 p = R[j], q = R[Pn + j], f1 = F1[j], f2 = F2[j];
            double2 a1 = make_double2(f2.x * p.x, f2.x * p.y);
            a1 = make_double2(fma(f2.y, q.x, a1.x), fma(f2.y, q.y, a1.y));
            O[j] = a1;
            O[Pn + j] = make_double2(fma(f1.x, p.x, f1.y * p.y), fma(f1.x, q.x, f1.y * q.y));
        }
        R = fft_batched<-1>(O, R, P.plan_p, 2);
        store_split_adjoint(R, Gb1 + g_index(k, 0, 0, M), M, Pn, n_m);
        store_split_adjoint(R + Pn, Gb1 + g_index(k, 2, 0, M), M, Pn, n_m);
        return;
    }
    double2 acc1[MAXPER_A], acc2[MAXPER_A];
    // forward fields
    load_hermitian_pair(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, 1.0, 1.0);
    double2* R = fft_batched<+1>(X, Y, P.plan_p, 1);
    for (int j = tid; j < Pn; j += nth) F1[j] = R[j];
    __syncthreads();
    load_hermitian_pair(X, G1 + g_index(k, 2, 0, M), M, Pn, n_m, 1.0, 1.0);
    R = fft_batched<+1>(X, Y, P.plan_p, 1);
    for (int j = tid; j < Pn; j += nth) F2[j] = R[j];
    __syncthreads();
    const double ip = 1.0 / (double)Pn;
    // products with omega: (p_vw, p_uw)
    load_hermitian_pair(X, Gb2 + g_index(k, 0, 0, M), M, Pn, n_m, ip, 0.5 * ip);
    R = fft_batched<+1>(X, Y, P.plan_p, 1);
#pragma unroll
    for (int i = 0; i < MAXPER_A; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) {
            const double2 p = R[j], f1 = F1[j], f2 = F2[j];
            acc1[i] = make_double2(f2.x * p.x, f2.x * p.y);
            acc2[i] = make_double2(fma(f1.x, p.x, f1.y * p.y), 0.0);
        }
    }
    __syncthreads();
    // products with theta: (p_vt, p_ut)
    load_hermitian_pair(X, Gb2 + g_index(k, 2, 0, M), M, Pn, n_m, ip, 0.5 * ip);
    R = fft_batched<+1>(X, Y, P.plan_p, 1);
#pragma unroll
    for (int i = 0; i < MAXPER_A; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) {
            const double2 p = R[j], f1 = F1[j], f2 = F2[j];
            acc1[i] = make_double2(fma(f2.y, p.x, acc1[i].x), fma(f2.y, p.y, acc1[i].y));
            acc2[i].y = fma(f1.x, p.x, f1.y * p.y);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXPER_A; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) X[j] = acc1[i];
    }
    R = fft_batched<-1>(X, Y, P.plan_p, 1);
    store_split_adjoint(R, Gb1 + g_index(k, 0, 0, M), M, Pn, n_m);
    __syncthreads();
    double2* other = (R == X) ? Y : X;
#pragma unroll
    for (int i = 0; i < MAXPER_A; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) other[j] = acc2[i];
    }
    double2* o2 = (other == X) ? Y : X;
    R = fft_batched<-1>(other, o2, P.plan_p, 1);
    store_split_adjoint(R, Gb1 + g_index(k, 2, 0, M), M, Pn, n_m);
}

// ---------------------------------------------------------------------------
// adjoint of k_spec_to_grid, per m; adds into lam.  With the grid adjoints
// (v, u, w, t)_bar of mode m >= 1:
//   a0 = conj(i m) v_bar + 3 s u_bar + (6 + m^2 h^2/s^2) w_bar
//   a1 = -h^2 u_bar - (h^2/s - 5 s) w_bar,   a2 = -h^2 w_bar
//   psi_bar_n += C w_n [Syn^T a0 + Dc^T (Syn^T a1 + Dc^T Syn^T a2)]_n
//   theta_bar_n += C w_n [Syn^T t_bar]_n
// m = 0 (real parts): u_bar_n += C w_n [Syn^T (u_bar + w_bar/s) + Dc^T Syn^T w_bar]_n.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTA) k_adj_spec_to_grid(StepParams P, const double2* __restrict__ Gb1,
                                                          VecSet lam) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, nc = P.nc, M = P.M;
    const int NB = adj_batch4(L);
    double2* bufA = sm;
    double2* bufB = bufA + NB * L;
    double2* a = bufB + NB * L;  // [4][N]: a0, a1, a2, t
    double2* e = a + 4 * N;      // scan output
    const int tid = threadIdx.x, nth = blockDim.x;
    const double dm = (double)m;
    for (int k = tid; k < N; k += nth) {
        const double2* g = Gb1 + g_index(k, 0, m, M);
        const double s = P.s[k], h2 = P.h2[k], is = P.inv_s[k];
        double2 a0, a1, a2, t = g[3 * M];
        if (m > 0) {
            const double2 vb = g[0], ub = g[M], wb = g[2 * M];
            a0 = cadd(cadd(cmul_i(vb, -dm), cscale(ub, 3.0 * s)), cscale(wb, 6.0 + dm * dm * h2 * is * is));
            a1 = csub(cscale(ub, -h2), cscale(wb, h2 * is - 5.0 * s));
            a2 = cscale(wb, -h2);
        } else {
            const double ub = g[M].x, wb = g[2 * M].x;
            a0 = make_double2(ub + wb * is, 0.0);
            a1 = make_double2(wb, 0.0);
            a2 = make_double2(0.0, 0.0);
            t = make_double2(t.x, 0.0);
        }
        a[k] = a0;
        a[N + k] = a1;
        a[2 * N + k] = a2;
        a[3 * N + k] = t;
    }
    __syncthreads();
    for (int b0 = 0; b0 < 4; b0 += NB) {
        const int nb = min(NB, 4 - b0);
        cos_sums(a + b0 * N, a + b0 * N, nb, bufA, bufB, P);  // Syn^T of each
    }
    // Horner: a1 += Dc^T a2 (m > 0); a0 += Dc^T a1
    if (m > 0) {
        cheb_derivative_adjoint_scan(a + 2 * N, e, bufA, N, P.inv_a);
        for (int n = tid; n < N; n += nth) a[N + n] = cadd(a[N + n], e[n]);
        __syncthreads();
    }
    cheb_derivative_adjoint_scan(a + N, e, bufA, N, P.inv_a);
    for (int n = tid; n < nc; n += nth) {
        const double cw = P.cnorm * ((n == 0) ? 0.5 : 1.0);
        const double2 pv = cscale(cadd(a[n], e[n]), cw);
        const double2 tv = cscale(a[3 * N + n], cw);
        const size_t idx = (size_t)m * nc + n;
        if (m > 0)
            lam.psi[idx] = cadd(lam.psi[idx], pv);
        else
            lam.u[n] += pv.x;
        lam.th[idx] = cadd(lam.th[idx], tv);
    }
}

// ---------------------------------------------------------------------------
// rho = P S^{-H} lam with the dense inverses (column-major: Wp [M][nc][nc-4]
// complex, Wt [M][nc][nc-2], Wu [nc][nc-2] real); rows below the tau rows are
// written 0.  The kernel streams the inverses once (HBM-bound): a CTA takes ASR
// consecutive output rows of one kind (Psi, theta or u) of one mode m, its ASS
// warps split the columns j into slices, each warp load reading one column's ASR
// consecutive rows (coalesced), so that every thread has only ~nc/ASS dependent
// iterations; the slices' partial sums are added in a fixed order.
// Grid (M, tp + 2 tt): row tiles [0, tp) Psi, [tp, tp + tt) theta, then u (m = 0).
// ---------------------------------------------------------------------------
constexpr int ASR = 32, ASS = 8;

__global__ void __launch_bounds__(ASR * ASS) k_adj_solve(StepParams P, AdjFactors A, VecSet lam, VecSet rho) {
    extern __shared__ double2 sm[];  // the input vector, nc entries
    __shared__ double2 part[ASS][ASR];
    const int m = blockIdx.x, nc = P.nc, np = nc - 4, nt = nc - 2;
    const int tp = (np + ASR - 1) / ASR, tt = (nt + ASR - 1) / ASR;
    const int tile = blockIdx.y;
    const int kind = (tile < tp) ? 0 : (tile < tp + tt) ? 1 : 2;
    if (kind == 2 && m != 0) return;
    const int r0 = (tile - (kind == 0 ? 0 : (kind == 1 ? tp : tp + tt))) * ASR;
    const int tid = threadIdx.x, lane = tid & 31, sl = tid >> 5;
    for (int j = tid; j < nc; j += blockDim.x) {
        const size_t idx = (size_t)m * nc + j;
        sm[j] = (kind == 0) ? lam.psi[idx] : (kind == 1) ? lam.th[idx] : make_double2(lam.u[j], 0.0);
    }
    __syncthreads();
    const int row = r0 + lane, nrows = (kind == 0) ? np : nt;
    const int j0 = sl * nc / ASS, j1 = (sl + 1) * nc / ASS;
    double2 acc = make_double2(0.0, 0.0), acc1 = acc;
    if (row < nrows) {
        if (kind == 0) {
            if (m > 0) {
                const double2* g = A.Wp + (size_t)m * nc * np + row;
                int j = j0;
#pragma unroll 4
                for (; j + 1 < j1; j += 2) {
                    acc = cfma(__ldg(&g[(size_t)j * np]), sm[j], acc);
                    acc1 = cfma(__ldg(&g[(size_t)(j + 1) * np]), sm[j + 1], acc1);
                }
                if (j < j1) acc = cfma(__ldg(&g[(size_t)j * np]), sm[j], acc);
            }
        } else {
            const double* g = (kind == 1) ? A.Wt + (size_t)m * nc * nt + row : A.Wu + row;
            int j = j0;
#pragma unroll 4
            for (; j + 1 < j1; j += 2) {
                const double c = __ldg(&g[(size_t)j * nt]), c1 = __ldg(&g[(size_t)(j + 1) * nt]);
                acc.x = fma(c, sm[j].x, acc.x);
                acc.y = fma(c, sm[j].y, acc.y);
                acc1.x = fma(c1, sm[j + 1].x, acc1.x);
                acc1.y = fma(c1, sm[j + 1].y, acc1.y);
            }
            if (j < j1) {
                const double c = __ldg(&g[(size_t)j * nt]);
                acc.x = fma(c, sm[j].x, acc.x);
                acc.y = fma(c, sm[j].y, acc.y);
            }
        }
    }
    part[sl][lane] = cadd(acc, acc1);
    __syncthreads();
    if (sl == 0 && row < nrows) {
        double2 t = part[0][lane];
#pragma unroll
        for (int q = 1; q < ASS; ++q) t = cadd(t, part[q][lane]);
        const size_t base = (size_t)m * nc;
        if (kind == 0) {
            rho.psi[base + 4 + row] = t;
            if (row < 4) rho.psi[base + row] = make_double2(0.0, 0.0);
        } else if (kind == 1) {
            rho.th[base + 2 + row] = t;
            if (row < 2) rho.th[base + row] = make_double2(0.0, 0.0);
        } else {
            rho.u[2 + row] = t.x;
            if (row < 2) rho.u[row] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// lam = g + (Mass + (dt/2) Lin)^H rho and w = dt (c rho + c2 rho_next), per m,
// with the operators applied through their transposed bands:
//   psi:   (A0 + mu A2)^T + (dt/2) [(B0 + mu B2 + mu^2 B4)^T - i m (2/E) C^T]
//   theta: D^T + (dt/2)(F0 + mu F2)^T / Pr;   u: D^T + (dt/2) E^T
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTA) k_adj_apply(StepParams P, VecSet g, VecSet rho, VecSet rho_next, VecSet lam,
                                                   VecSet w, double dt, double c, double c2) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x, nc = P.nc;
    double2* rp = sm;
    double2* rt = rp + nc;
    double* ru = reinterpret_cast<double*>(rt + nc);
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        const size_t idx = (size_t)m * nc + j;
        rp[j] = rho.psi[idx];
        rt[j] = rho.th[idx];
        if (m == 0) ru[j] = rho.u[j];
        w.psi[idx] = cscale(cadd(cscale(rho.psi[idx], c), cscale(rho_next.psi[idx], c2)), dt);
        w.th[idx] = cscale(cadd(cscale(rho.th[idx], c), cscale(rho_next.th[idx], c2)), dt);
        if (m == 0) w.u[j] = dt * (c * rho.u[j] + c2 * rho_next.u[j]);
    }
    __syncthreads();
    const double mu = (double)m * m, hd = 0.5 * dt;
    for (int n = threadIdx.x; n < nc; n += blockDim.x) {
        const size_t idx = (size_t)m * nc + n;
        double2 lp = g.psi ? g.psi[idx] : make_double2(0.0, 0.0);
        double2 lt = g.th ? g.th[idx] : make_double2(0.0, 0.0);
        if (m > 0) {
            const double2 a0 = bandT_row<8>(P.ops.bandT[OP_A0], rp, n, nc);
            const double2 a2 = bandT_row<8>(P.ops.bandT[OP_A2], rp, n, nc);
            const double2 b0 = bandT_row<6>(P.ops.bandT[OP_B0], rp, n, nc);
            const double2 b2 = bandT_row<6>(P.ops.bandT[OP_B2], rp, n, nc);
            const double2 b4 = bandT_row<6>(P.ops.bandT[OP_B4], rp, n, nc);
            const double2 cc = bandT_row<8>(P.ops.bandT[OP_C], rp, n, nc);
            double2 v = make_double2(a0.x + mu * a2.x, a0.y + mu * a2.y);
            double2 b = make_double2(b0.x + mu * (b2.x + mu * b4.x), b0.y + mu * (b2.y + mu * b4.y));
            b = cadd(b, cmul_i(cc, -2.0 * (double)m / P.E));
            v = cadd(v, cscale(b, hd));
            lp = cadd(lp, v);
        } else {
            lp = make_double2(0.0, 0.0);
        }
        const double2 d = bandT_row<4>(P.ops.bandT[OP_D], rt, n, nc);
        const double2 f0 = bandT_row<2>(P.ops.bandT[OP_F0], rt, n, nc);
        const double2 f2 = bandT_row<2>(P.ops.bandT[OP_F2], rt, n, nc);
        const double fp = hd / P.Pr;
        lt = cadd(lt, make_double2(d.x + fp * (f0.x + mu * f2.x), d.y + fp * (f0.y + mu * f2.y)));
        lam.psi[idx] = lp;
        lam.th[idx] = lt;
        if (m == 0) {
            double lu = g.u ? g.u[n] : 0.0;
            lu += bandT_row_r<4>(P.ops.bandT[OP_D], ru, n, nc) + hd * bandT_row_r<2>(P.ops.bandT[OP_EZ], ru, n, nc);
            lam.u[n] = lu;
        }
    }
}

// a += b over the three fields (b's null fields are skipped)
__global__ void k_vec_add(int M, int nc, VecSet a, VecSet b) {
    const size_t n = (size_t)M * nc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (b.psi) a.psi[i] = cadd(a.psi[i], b.psi[i]);
        if (b.th) a.th[i] = cadd(a.th[i], b.th[i]);
        if (b.u && i < (size_t)nc) a.u[i] += b.u[i];
    }
}

__global__ void k_ra_accumulate(const double* __restrict__ ra, int M, double* __restrict__ acc) {
    double t = 0.0;
    for (int m = threadIdx.x; m < M; m += 32) t += ra[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *acc += t;
}

}  // namespace

cudaError_t launch_ra_accumulate(const double* ra, int M, double* acc, cudaStream_t st) {
    k_ra_accumulate<<<1, 32, 0, st>>>(ra, M, acc);
    return cudaGetLastError();
}

cudaError_t launch_vec_add(const StepParams& P, VecSet a, VecSet b, cudaStream_t st) {
    k_vec_add<<<P.M, NTA, 0, st>>>(P.M, P.nc, a, b);
    return cudaGetLastError();
}

size_t smem_adj_grid_to_spec(const StepParams& P) {
    const int L = 2 * P.K;
    return sizeof(double2) * (2 * adj_batch(L) * L + 4 * P.n_r);
}
size_t smem_adj_spec_to_grid(const StepParams& P) {
    const int L = 2 * P.K;
    return sizeof(double2) * (2 * adj_batch4(L) * L + 5 * P.n_r);
}

cudaError_t launch_adj_explicit(const StepParams& P, VecSet w, VecSet y, VecSet lam, const double2* G1, double2* Gb2,
                                double2* Gb1, double* ra, cudaStream_t st) {
    if (P.n_phi > NTA * MAXPER_A) return cudaErrorInvalidValue;
    size_t sm = smem_adj_grid_to_spec(P);
    cudaError_t err = cudaFuncSetAttribute(k_adj_grid_to_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_adj_grid_to_spec<<<P.M, NTA, sm, st>>>(P, w, y, lam, Gb2, ra);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // the batched pairs need 6 n_phi entries (n_phi <= 2048), else 4 n_phi
    int dev = 0, smax = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    const int pair = sizeof(double2) * 6 * P.n_phi <= (size_t)smax ? 1 : 0;
    sm = sizeof(double2) * (pair ? 6 : 4) * P.n_phi;
    err = cudaFuncSetAttribute(k_adj_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_adj_phi<<<P.n_r, NTA, sm, st>>>(P, G1, Gb2, Gb1, pair);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    sm = smem_adj_spec_to_grid(P);
    err = cudaFuncSetAttribute(k_adj_spec_to_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_adj_spec_to_grid<<<P.M, NTA, sm, st>>>(P, Gb1, lam);
    return cudaGetLastError();
}

cudaError_t launch_adj_solve(const StepParams& P, const AdjFactors& A, VecSet lam, VecSet rho, cudaStream_t st) {
    const size_t sm = sizeof(double2) * P.nc;
    const int tp = (P.nc - 4 + ASR - 1) / ASR, tt = (P.nc - 2 + ASR - 1) / ASR;
    dim3 grid(P.M, tp + 2 * tt);
    k_adj_solve<<<grid, ASR * ASS, sm, st>>>(P, A, lam, rho);
    return cudaGetLastError();
}

cudaError_t launch_adj_apply(const StepParams& P, VecSet g, VecSet rho, VecSet rho_next, VecSet lam, VecSet w,
                             double dt, double c, double c2, cudaStream_t st) {
    const size_t sm = sizeof(double2) * 2 * P.nc + sizeof(double) * P.nc;
    k_adj_apply<<<P.M, NTA, sm, st>>>(P, g, rho, rho_next, lam, w, dt, c, c2);
    return cudaGetLastError();
}

}  // namespace pz
