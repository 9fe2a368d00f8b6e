// Explicit stage of one IMEX step (Sections 2, 3 and 3.2 of Gastine, pizza,
// GJI 2019): spectral -> radial grid per azimuthal mode m, grid products per
// radius, radial grid -> integrated right-hand sides per m.
//
// Layouts (double2 = complex):
//   state   Psi_hat, theta_hat  [M][nc]  (paper f_hat convention, Eq. cheb)
//   G1      [n_r][4][M]  radial-grid Fourier coefficients of
//           v = dPsi/dphi, u_phi, omega, theta            (radius-major)
//   G2      [n_r][4][M]  Fourier coefficients of the products
//           v*omega, u_phi*omega, v*theta, u_phi*theta     (radius-major)
//   e       [M][nc] integrated explicit right-hand sides
// The change from mode-major to radius-major order (the paper's MPI transpose)
// is folded into the stores of spec_to_grid and the loads of grid_to_spec.
#include "device_common.cuh"

namespace pz {

namespace {

constexpr int NTHREADS_R = 256;  // radial kernels
constexpr int MAXPER = 12;       // azimuthal points per thread held in registers

__device__ __forceinline__ int g_index(int k, int f, int m, int M) { return (k * 4 + f) * M + m; }

// number of radial transforms batched together in shared memory (the
// autotuner's choice, else up to n_r = 513 four in FP64 -- all four synthesised
// fields of a mode in one pass -- and two in FP32, measured fastest at n_r = 257)
__host__ __device__ inline int radial_batch(const StepParams& P) {
    if (P.nb_r > 0) return P.nb_r;
    if (2 * P.K > 1024) return 1;
    return P.fp32 ? 2 : 4;
}
// threads of the per-radius azimuthal kernels
inline int phi_threads(const StepParams& P) {
    if (P.phi_threads > 0) return P.phi_threads;
    return P.n_phi > 256 * MAXPER ? 512 : 256;
}

// ---------------------------------------------------------------------------
// K1: per m, Chebyshev coefficients -> values on the Gauss-Lobatto grid.
//   v = i m Psi,  u_phi = -h^2 Psi' + 3 s Psi,
//   omega = -[h^2 Psi'' + (h^2/s - 5 s) Psi' - (6 + m^2 h^2/s^2) Psi]   (m >= 1)
//   m = 0:  v = 0, u_phi = u_bar, omega = u_bar' + u_bar/s
// (Section 3.2: u_s = (h^2/s) dPsi/dphi, u_phi = u_bar - h^2 dPsi/ds + 3 s Psi,
//  omega = (1/s) d(s u_bar)/ds - L_I Psi.)
// With Ekman pumping it also writes P.pump_F[m][k]: for m >= 1 the approximate
// pumping of Eq. approx_pump,
//   F_eps = Ups_eps [ -omega + (s/2) Psi' - (3 s^2/(2 h_eps^2) + m^2 + i m 5 s_o/(2 h_eps)) Psi ]
// (L_I Psi = -omega), built up over the passes of Psi, Psi' and omega; for m = 0
// the zonal-flow terms Ups_eps u_bar (1 + (E/2) omega_0) of Eqs. uphi_int and
// uphicoll.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(NTHREADS_R) k_spec_to_grid(StepParams P, VecSet y, T* __restrict__ G1) {
    using RT = typename Cx<T>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, nc = P.nc, M = P.M;
    const int NB = radial_batch(P);
    T* bufA = sm;
    T* bufB = bufA + NB * L;
    T* cc0 = bufB + NB * L;  // Psi (or u_bar) plain coefficients, length N
    T* cc1 = cc0 + N;        // first derivative
    T* cc2 = cc1 + N;        // second derivative
    const int tid = threadIdx.x, nth = blockDim.x;
    // C w_n of Eq. cheb in the working precision (the state is converted first)
    const RT Cw = (RT)P.cnorm, Cw0 = (RT)(0.5 * P.cnorm);

    for (int n = tid; n < N; n += nth) {
        T a = Cx<T>::make(0.0, 0.0);
        if (n < nc) {
            const RT w = (n == 0) ? Cw0 : Cw;
            if (m > 0)
                a = cscale(Cx<T>::from(y.psi[(size_t)m * nc + n]), w);
            else
                a = Cx<T>::make((RT)y.u[n] * w, 0.0);
        }
        cc0[n] = a;
    }
    __syncthreads();
    cheb_derivative_scan(cc0, cc1, bufA, N, P.inv_a);
    if (m > 0) cheb_derivative_scan(cc1, cc2, bufA, N, P.inv_a);

    // field list: 0 Psi, 1 Psi', 2 Psi'', 3 theta, 4 packed u_bar + i lam u_bar'
    // (lam a power of two balancing the two parts).  The reduction's 16 doubles
    // live in bufB (at least 128 bytes: n_r >= 9), unused until the first
    // transform: without static shared memory two FP32 CTAs fit an SM at
    // n_r = 2049.
    RT lam = 1;
    if (m == 0) {
        double* red = reinterpret_cast<double*>(bufB);  // [warp][2]
        double a0 = 0.0, a1 = 0.0;
        for (int i = tid; i < N; i += nth) {
            a0 = fmax(a0, (double)(fabs(cc0[i].x) + fabs(cc0[i].y)));
            a1 = fmax(a1, (double)(fabs(cc1[i].x) + fabs(cc1[i].y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 = fmax(a0, __shfl_xor_sync(0xffffffffu, a0, o));
            a1 = fmax(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        }
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            red[2 * w] = a0;
            red[2 * w + 1] = a1;
        }
        __syncthreads();
        double r0 = 0.0, r1 = 0.0;
        for (int q = 0; q < (nth >> 5); ++q) {
            r0 = fmax(r0, red[2 * q]);
            r1 = fmax(r1, red[2 * q + 1]);
        }
        lam = (RT)pow2_ratio(r0, r1);
    }
    int fields[4];
    int nf;
    if (m > 0) {
        fields[0] = 0; fields[1] = 1; fields[2] = 2; fields[3] = 3; nf = 4;
    } else {
        fields[0] = 4; fields[1] = 3; nf = 2;
    }
    const RT dm = (RT)m;
    T* PF = P.pump ? reinterpret_cast<T*>(P.pump_F) + (size_t)m * N : nullptr;
    for (int f0 = 0; f0 < nf; f0 += NB) {
        const int nb = min(NB, nf - f0);
        for (int b = 0; b < nb; ++b) {
            const int fid = fields[f0 + b];
            T* z = bufA + b * L;
            for (int j = tid; j <= K; j += nth) {
                T v;
                if (fid == 0) v = cc0[j];
                else if (fid == 1) v = cc1[j];
                else if (fid == 2) v = cc2[j];
                else if (fid == 3)
                    v = (j < nc) ? cscale(Cx<T>::from(y.th[(size_t)m * nc + j]), (j == 0) ? Cw0 : Cw)
                                 : Cx<T>::make(0.0, 0.0);
                else {
                    v.x = cc0[j].x;
                    v.y = lam * cc1[j].x;
                }
                if (j == 0 || j == K) v = cscale(v, (RT)2);
                even_extend_store(z, K, j, v);
            }
        }
        T* R = radial_dct1(bufA, bufB, P, nb);
        for (int b = 0; b < nb; ++b) {
            const int fid = fields[f0 + b];
            const T* Z = R + b * L;
            for (int k = tid; k < N; k += nth) {
                const T g = cscale(Z[k], (RT)0.5);  // value of the series at x_k
                const RT s = Tab<T>::s(P, k), h2 = Tab<T>::h2(P, k), is = Tab<T>::is(P, k);
                T* out = G1 + g_index(k, 0, m, M);
                // out[0] = v, out[M] = u_phi, out[2M] = omega, out[3M] = theta
                if (fid == 0) {
                    out[0] = cmul_i(g, dm);
                    out[M] = cscale(g, (RT)3 * s);
                    out[2 * M] = cscale(g, (RT)6 + dm * dm * h2 * is * is);
                    if (PF) {
                        const RT U = (RT)P.pump_ups[k];
                        PF[k] = cadd(cscale(g, -U * ((RT)P.pump_cr[k] + dm * dm)), cmul_i(g, -U * dm * (RT)P.pump_ci[k]));
                    }
                } else if (fid == 1) {
                    out[M] = csub(out[M], cscale(g, h2));
                    out[2 * M] = csub(out[2 * M], cscale(g, h2 * is - (RT)5 * s));
                    if (PF) PF[k] = cadd(PF[k], cscale(g, (RT)P.pump_ups[k] * (RT)0.5 * s));
                } else if (fid == 2) {
                    out[2 * M] = csub(out[2 * M], cscale(g, h2));
                    if (PF) PF[k] = csub(PF[k], cscale(out[2 * M], (RT)P.pump_ups[k]));
                } else if (fid == 3) {
                    out[3 * M] = g;
                } else {
                    out[0] = Cx<T>::make(0.0, 0.0);
                    out[M] = Cx<T>::make(g.x, 0.0);
                    out[2 * M] = Cx<T>::make(g.y / lam + g.x * is, 0.0);
                    if (PF) {
                        const RT w0 = g.y / lam + g.x * is;
                        PF[k] = Cx<T>::make((RT)P.pump_ups[k] * g.x * ((RT)1 + (RT)(0.5 * P.E) * w0), 0.0);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K2: per radius, Eq. fft to the N_phi-point azimuthal grid, the four products,
// Eq. ifft back (modes m <= N_m kept).  Two real fields travel in one complex
// transform: g1 = v + i u_phi, g2 = omega + i theta; then
//   g1 * Re(g2) = v omega + i u_phi omega,  g1 * Im(g2) = v theta + i u_phi theta.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void load_packed_spectrum(T* Z, const T* __restrict__ src, int M, int Pn, int n_m,
                                                     typename Cx<T>::R sa, typename Cx<T>::R sb) {
    // src points at G1/G2 row (k, f): field a = src[0..M), field b = src[M..2M);
    // packed as sa a + i sb b
    for (int j = threadIdx.x; j < Pn; j += blockDim.x) {
        T z = Cx<T>::make(0.0, 0.0);
        if (j == 0) {
            z.x = sa * src[0].x;
            z.y = sb * src[M].x;
        } else if (j <= n_m) {
            const T a = cscale(src[j], sa), b = cscale(src[M + j], sb);
            z.x = a.x - b.y;  // a + i b
            z.y = a.y + b.x;
        } else if (j >= Pn - n_m) {
            const int mm = Pn - j;
            const T a = cscale(src[mm], sa), b = cscale(src[M + mm], sb);
            z.x = a.x + b.y;  // conj(a) + i conj(b)
            z.y = -a.y + b.x;
        }
        Z[j] = z;
    }
}

// Split the transform Y of a + i b (a, b real fields) into the spectra of a and
// b, scaled by ia and ib (1/Pn times the inverse packing weights).
template <class T>
__device__ __forceinline__ void store_split_spectrum(const T* Y, T* __restrict__ dst, int M, int Pn, int n_m,
                                                     typename Cx<T>::R ia, typename Cx<T>::R ib) {
    using RT = typename Cx<T>::R;
    const RT h = (RT)0.5;
    for (int m = threadIdx.x; m <= n_m; m += blockDim.x) {
        T a, b;
        if (m == 0) {
            a = Cx<T>::make(Y[0].x * ia, 0.0);
            b = Cx<T>::make(Y[0].y * ib, 0.0);
        } else {
            const T y1 = Y[m], y2 = Y[Pn - m];
            // a = (y1 + conj(y2))/2,  b = (y1 - conj(y2))/(2i)
            a.x = h * (y1.x + y2.x) * ia;
            a.y = h * (y1.y - y2.y) * ia;
            b.x = h * (y1.y + y2.y) * ib;
            b.y = -h * (y1.x - y2.x) * ib;
        }
        dst[m] = a;
        dst[M + m] = b;
    }
}

// exact powers of two in the working precision; balancing exponents are
// limited further in FP32 (exponent range of float)
template <class T>
struct P2;
template <>
struct P2<double2> {
    static constexpr int lim = 400;
    __device__ static double v(int e) { return pow2d(e); }
};
template <>
struct P2<float2> {
    static constexpr int lim = 40;
    __device__ static float v(int e) { return pow2f(e); }
};

// Courant rates of Eq. cfl at radius k from the synthesised packed pair
// g1 = v + i l1 u_phi on the n_phi points (v = d Psi/d phi, u_s = (h^2/s) v in
// the integration formulation, v/s in collocation): max |u_s|/ds_k and
// max |u_phi|/(s_k dphi), folded into P.cfl_max[0..1] as atomic maxima of their
// bit patterns (non-negative doubles order like their bits).  Called by every
// thread of the block; uses red[0 .. 2 * warps).
__device__ __forceinline__ double re_abs(float2 z) { return fabs((double)z.x); }
__device__ __forceinline__ double im_abs(float2 z) { return fabs((double)z.y); }
__device__ __forceinline__ double re_abs(double2 z) { return fabs(z.x); }
__device__ __forceinline__ double im_abs(double2 z) { return fabs(z.y); }
__device__ __forceinline__ double re_abs(ddc z) { return fabs(dd_to(z.x)); }
__device__ __forceinline__ double im_abs(ddc z) { return fabs(dd_to(z.y)); }

template <class T>
__device__ void cfl_rates(const StepParams& P, const T* R, int Pn, double l1, int k, double* red) {
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < Pn; j += blockDim.x) {
        a = fmax(a, re_abs(R[j]));
        b = fmax(b, im_abs(R[j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) {
            a = fmax(a, red[2 * i]);
            b = fmax(b, red[2 * i + 1]);
        }
        const double s = P.s[k];
        const double fs = P.coll ? 1.0 / s : P.h2[k] / s;
        const double rs = fs * a / P.cfl_ds[k];
        const double rp = b / l1 / (s * P.cfl_dphi);
        atomicMax(reinterpret_cast<unsigned long long*>(P.cfl_max), (unsigned long long)__double_as_longlong(rs));
        atomicMax(reinterpret_cast<unsigned long long*>(P.cfl_max + 1),
                  (unsigned long long)__double_as_longlong(rp));
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(512, 1) k_phi_products(StepParams P, const T* __restrict__ G1,
                                                         T* __restrict__ G2, int pair) {
    using RT = typename Cx<T>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int k = P.k_lo + blockIdx.x;
    const int Pn = P.n_phi, M = P.M, n_m = P.n_m;
    T* X = sm;
    T* Y = sm + Pn;
    const int tid = threadIdx.x, nth = blockDim.x;
    T reg[MAXPER];
    // exact power-of-two weights that balance the packed pairs:
    // g1 = v + i l1 u_phi, g2 = omega + i l2 theta
    __shared__ double red[4 * 32], mx[4];
    block_max_abs(G1 + g_index(k, 0, 0, M), M, 4, n_m + 1, mx, red);
    const int e1 = pow2_exponent(mx[0], mx[1], P2<T>::lim), e2 = pow2_exponent(mx[2], mx[3], P2<T>::lim);
    const RT l1 = P2<T>::v(e1), l2 = P2<T>::v(e2);
    const RT iP = (RT)P.inv_nphi;  // 1/n_phi, a power of two divided by 3

    if (pair) {
        // both packed pairs in one batched transform each way (X, Y hold 2 Pn)
        Y = X + 2 * Pn;
        load_packed_spectrum(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, (RT)1, l1);
        load_packed_spectrum(X + Pn, G1 + g_index(k, 2, 0, M), M, Pn, n_m, (RT)1, l2);
        T* R = fft_batched<+1>(X, Y, P.plan_p, 2);
        if (P.cfl_max) cfl_rates(P, R, Pn, (double)l1, k, red);
        T* O = (R == X) ? Y : X;
        for (int j = tid; j < Pn; j += nth) {
            const T g1 = R[j], g2 = R[Pn + j];
            O[j] = cscale(g1, g2.x);
            O[Pn + j] = cscale(g1, g2.y);
        }
        T* S = fft_batched<-1>(O, R, P.plan_p, 2);
        store_split_spectrum(S, G2 + g_index(k, 0, 0, M), M, Pn, n_m, iP, iP * P2<T>::v(-e1));
        store_split_spectrum(S + Pn, G2 + g_index(k, 2, 0, M), M, Pn, n_m, iP * P2<T>::v(-e2),
                             iP * P2<T>::v(-e1 - e2));
        return;
    }
    load_packed_spectrum(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, (RT)1, l1);
    T* R = fft_batched<+1>(X, Y, P.plan_p, 1);
    if (P.cfl_max) cfl_rates(P, R, Pn, (double)l1, k, red);
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) reg[i] = R[j];
    }
    __syncthreads();
    load_packed_spectrum(X, G1 + g_index(k, 2, 0, M), M, Pn, n_m, (RT)1, l2);
    R = fft_batched<+1>(X, Y, P.plan_p, 1);
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) {
            const T g2 = R[j], g1 = reg[i];
            R[j] = cscale(g1, g2.x);
            reg[i] = cscale(g1, g2.y);
        }
    }
    T* other = (R == X) ? Y : X;
    T* S = fft_batched<-1>(R, other, P.plan_p, 1);
    // g1 Re(g2) = v omega + i l1 u_phi omega
    store_split_spectrum(S, G2 + g_index(k, 0, 0, M), M, Pn, n_m, iP, iP * P2<T>::v(-e1));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) X[j] = reg[i];
    }
    S = fft_batched<-1>(X, Y, P.plan_p, 1);
    // g1 Im(g2) = l2 (v theta + i l1 u_phi theta)
    store_split_spectrum(S, G2 + g_index(k, 2, 0, M), M, Pn, n_m, iP * P2<T>::v(-e2), iP * P2<T>::v(-e1 - e2));
}

// ---------------------------------------------------------------------------
// K2 of the FP64 stage in double-float arithmetic (ddfloat.cuh): the FP64
// spectra are split into float pairs on load, the transforms and products run
// on the FP32 pipe with ~48-bit significands, and the product spectra are
// rounded back to FP64 on store.  The same steps as k_phi_products; the packed
// pairs are balanced within float range (|exponent difference| <= 40).
// The m = 0 modes of the products are taken in FP64 from the input spectra
// instead: with band-limited fields (2 n_m < n_phi, no aliasing) the mean of
// a b is a_0 b_0 + 2 sum_{m >= 1} Re(a_m conj(b_m)).  These means (the zonal
// forcing [v omega]_0 above all) cancel to ~1e-4 of their terms, which would
// magnify the double-float rounding beyond FP64 accuracy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_packed_spectrum_dd(ddc* Z, const double2* __restrict__ src, int M, int Pn,
                                                        int n_m, float sb) {
    // each spectral value converted once, written to m and to its mirror Pn - m
    for (int m = threadIdx.x; m <= n_m; m += blockDim.x) {
        if (m == 0) {
            Z[0] = ddc{dd_from_bits(src[0].x), dd_scale2(dd_from_bits(src[M].x), sb)};
            continue;
        }
        const ddc a = dd_from_bits(src[m]);
        ddc b = dd_from_bits(src[M + m]);
        b.x = dd_scale2(b.x, sb);
        b.y = dd_scale2(b.y, sb);
        Z[m] = ddc{a.x - b.y, a.y + b.x};        // a + i b
        Z[Pn - m] = ddc{a.x + b.y, b.x - a.y};   // conj(a) + i conj(b)
    }
    for (int j = n_m + 1 + threadIdx.x; j < Pn - n_m; j += blockDim.x) Z[j] = ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}};
}

__device__ __forceinline__ void store_split_spectrum_dd(const ddc* Y, double2* __restrict__ dst, int M, int Pn,
                                                        int n_m, ddf ia, ddf ib) {
    for (int m = threadIdx.x; m <= n_m; m += blockDim.x) {
        ddc a, b;
        if (m == 0) {
            a = ddc{Y[0].x * ia, ddf{0.f, 0.f}};
            b = ddc{Y[0].y * ib, ddf{0.f, 0.f}};
        } else {
            const ddc y1 = Y[m], y2 = Y[Pn - m];
            // a = (y1 + conj(y2))/2,  b = (y1 - conj(y2))/(2i)
            a.x = dd_scale2(y1.x + y2.x, 0.5f) * ia;
            a.y = dd_scale2(y1.y - y2.y, 0.5f) * ia;
            b.x = dd_scale2(y1.y + y2.y, 0.5f) * ib;
            b.y = -(dd_scale2(y1.x - y2.x, 0.5f) * ib);
        }
        dst[m] = dd_compose(a);
        dst[M + m] = dd_compose(b);
    }
}

// |x| as the high word of its bits (monotone in |x|: its biased exponent and
// leading fraction bits), on the integer pipe
__device__ __forceinline__ unsigned hi_word_abs(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
// the power of two a / b rounded down to exponents, from the high words of a and b,
// clamped to [-lim, lim]; 0 where either is zero or subnormal
__device__ __forceinline__ int pow2_exponent_words(unsigned wa, unsigned wb, int lim) {
    const int ea = (int)(wa >> 20), eb = (int)(wb >> 20);
    if (ea == 0 || eb == 0) return 0;
    return max(-lim, min(lim, ea - eb));
}

__global__ void __launch_bounds__(512, 1) k_phi_products_dd(StepParams P, const double2* __restrict__ G1,
                                                            double2* __restrict__ G2, int pair) {
    extern __shared__ __align__(16) unsigned char smraw[];
    ddc* sm = reinterpret_cast<ddc*>(smraw);
    const int k = P.k_lo + blockIdx.x;
    const int Pn = P.n_phi, M = P.M, n_m = P.n_m;
    ddc* X = sm;
    ddc* Y = sm + Pn;
    const int tid = threadIdx.x, nth = blockDim.x;
    ddc reg[MAXPER];
    __shared__ double red[4 * 32];
    const ddf iP = dd_from(P.inv_nphi);  // 1/n_phi
    // One pass over the four fields (v, u_phi, omega, theta):
    // * the FP64 means of the four products, pairs (v, omega), (u_phi, omega),
    //   (v, theta), (u_phi, theta): a_0 b_0 + 2 sum_{m >= 1} Re(a_m conj(b_m)), with
    //   the real parts only at m = 0 (the transforms read no more of mode 0);
    // * the largest biased exponent of |Re|, |Im| of each field, from the high
    //   words on the integer pipe: the powers of two that balance the packed pairs.
    __shared__ double msum[4][16];
    __shared__ unsigned wmx[4][16];
    {
        double acc[4] = {0.0, 0.0, 0.0, 0.0}, a0[4] = {0.0, 0.0, 0.0, 0.0};
        unsigned hx[4] = {0u, 0u, 0u, 0u};
        const double2* f = G1 + g_index(k, 0, 0, M);  // f[q * M + m]: v, u_phi, omega, theta
        for (int m = tid; m <= n_m; m += nth) {
            const double2 v = f[m], up = f[M + m], om = f[2 * M + m], th = f[3 * M + m];
            hx[0] = max(hx[0], max(hi_word_abs(v.x), hi_word_abs(v.y)));
            hx[1] = max(hx[1], max(hi_word_abs(up.x), hi_word_abs(up.y)));
            hx[2] = max(hx[2], max(hi_word_abs(om.x), hi_word_abs(om.y)));
            hx[3] = max(hx[3], max(hi_word_abs(th.x), hi_word_abs(th.y)));
            if (m == 0) {
                a0[0] = v.x * om.x;
                a0[1] = up.x * om.x;
                a0[2] = v.x * th.x;
                a0[3] = up.x * th.x;
            } else {
                acc[0] = fma(v.x, om.x, fma(v.y, om.y, acc[0]));
                acc[1] = fma(up.x, om.x, fma(up.y, om.y, acc[1]));
                acc[2] = fma(v.x, th.x, fma(v.y, th.y, acc[2]));
                acc[3] = fma(up.x, th.x, fma(up.y, th.y, acc[3]));
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[q] = fma(2.0, acc[q], a0[q]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            hx[q] = __reduce_max_sync(0xffffffffu, hx[q]);
        }
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                msum[q][tid >> 5] = acc[q];
                wmx[q][tid >> 5] = hx[q];
            }
    }
    __syncthreads();
    int e1, e2;
    {
        unsigned w[4] = {0u, 0u, 0u, 0u};
        for (int i = 0; i < (nth >> 5); ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = max(w[q], wmx[q][i]);
        e1 = pow2_exponent_words(w[0], w[1], 40);
        e2 = pow2_exponent_words(w[2], w[3], 40);
    }

    if (pair) {
        // both packed pairs in one batched transform each way (X, Y hold 2 Pn):
        // half the barrier-separated passes, the same arithmetic per transform
        Y = X + 2 * Pn;
        load_packed_spectrum_dd(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, pow2f(e1));
        load_packed_spectrum_dd(X + Pn, G1 + g_index(k, 2, 0, M), M, Pn, n_m, pow2f(e2));
        ddc* R = fft_batched<+1, ddc, true>(X, Y, P.plan_p, 2);
        if (P.cfl_max) cfl_rates(P, R, Pn, (double)pow2f(e1), k, red);
        ddc* O = (R == X) ? Y : X;
        for (int j = tid; j < Pn; j += nth) {
            const ddc g1 = R[j], g2 = R[Pn + j];
            O[j] = cscale(g1, g2.x);
            O[Pn + j] = cscale(g1, g2.y);
        }
        ddc* S = fft_batched<-1, ddc, true>(O, R, P.plan_p, 2);
        store_split_spectrum_dd(S, G2 + g_index(k, 0, 0, M), M, Pn, n_m, iP, dd_scale2(iP, pow2f(-e1)));
        store_split_spectrum_dd(S + Pn, G2 + g_index(k, 2, 0, M), M, Pn, n_m, dd_scale2(iP, pow2f(-e2)),
                                dd_scale2(dd_scale2(iP, pow2f(-e1)), pow2f(-e2)));
        __syncthreads();  // the stores above are done (thread 0 wrote the m = 0 entries replaced here)
        if (tid < 4) {
            double t = 0.0;
            for (int w = 0; w < (nth >> 5); ++w) t += msum[tid][w];
            G2[g_index(k, tid, 0, M)] = make_double2(t, 0.0);
        }
        return;
    }
    load_packed_spectrum_dd(X, G1 + g_index(k, 0, 0, M), M, Pn, n_m, pow2f(e1));
    ddc* R = fft_batched<+1, ddc, true>(X, Y, P.plan_p, 1);
    if (P.cfl_max) cfl_rates(P, R, Pn, (double)pow2f(e1), k, red);
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) reg[i] = R[j];
    }
    __syncthreads();
    load_packed_spectrum_dd(X, G1 + g_index(k, 2, 0, M), M, Pn, n_m, pow2f(e2));
    R = fft_batched<+1, ddc, true>(X, Y, P.plan_p, 1);
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) {
            const ddc g2 = R[j], g1 = reg[i];
            R[j] = cscale(g1, g2.x);
            reg[i] = cscale(g1, g2.y);
        }
    }
    ddc* other = (R == X) ? Y : X;
    ddc* S = fft_batched<-1, ddc, true>(R, other, P.plan_p, 1);
    // g1 Re(g2) = v omega + i l1 u_phi omega
    store_split_spectrum_dd(S, G2 + g_index(k, 0, 0, M), M, Pn, n_m, iP, dd_scale2(iP, pow2f(-e1)));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXPER; ++i) {
        const int j = tid + i * nth;
        if (j < Pn) X[j] = reg[i];
    }
    S = fft_batched<-1, ddc, true>(X, Y, P.plan_p, 1);
    // g1 Im(g2) = l2 (v theta + i l1 u_phi theta)
    store_split_spectrum_dd(S, G2 + g_index(k, 2, 0, M), M, Pn, n_m, dd_scale2(iP, pow2f(-e2)),
                            dd_scale2(dd_scale2(iP, pow2f(-e1)), pow2f(-e2)));
    __syncthreads();  // the stores above are done (thread 0 wrote the m = 0 entries replaced here)
    if (tid < 4) {
        double t = 0.0;
        for (int w = 0; w < (nth >> 5); ++w) t += msum[tid][w];
        G2[g_index(k, tid, 0, M)] = make_double2(t, 0.0);  // G2 fields follow the pair order
    }
}

// ---------------------------------------------------------------------------
// K3: per m, radial divergences of the fluxes, Eq. icheb, truncation to n < N_c
// (dealiasing), and the integrated right-hand sides
//   N_omega = (1/s) d/ds(h^2 [v omega]_m) + (i m/s) [u_phi omega]_m
//   N_theta = (1/s) d/ds(h^2 [v theta]_m) + (i m/s) [u_phi theta]_m - [v theta]_m
//   N_u     = (h^2/s) [v omega]_0
//   e_psi   = C^I [ (Ra/Pr)(i m/s_o) theta_hat_m + N_omega_hat ]        (m >= 1)
//   e_theta = -D^I N_theta_hat - (alpha/ln eta) i m G^I Psi_hat_m
//   e_u     = -D^I N_u_hat
// (Eqs. vort, temp, uphi; psi_int, temp_int, uphi_int; u_s = (h^2/s) v and
//  beta u_s = -v.)  The radial derivative is that of the n_r-point interpolant.
// ---------------------------------------------------------------------------
template <int H, class V>
__device__ __forceinline__ double2 band_row(const double* __restrict__ band, const V* x, int k, int nc) {
    const double* row = band + (size_t)k * (2 * H + 1);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int d = 0; d <= 2 * H; ++d) {
        const int n = k - H + d;
        if (n >= 0 && n < nc) {
            const double c = __ldg(&row[d]);
            const double2 v = to_d2(x[n]);
            acc.x = fma(c, v.x, acc.x);
            acc.y = fma(c, v.y, acc.y);
        }
    }
    return acc;
}

template <class T>
__global__ void __launch_bounds__(NTHREADS_R) k_grid_to_spec(StepParams P, const T* __restrict__ G2, VecSet y,
                                                             VecSet e) {
    using RT = typename Cx<T>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, L = 2 * K, N = P.n_r, nc = P.nc, M = P.M;
    const int NB = radial_batch(P);
    T* bufA = sm;
    T* bufB = bufA + NB * L;
    T* cc0 = bufB + NB * L;
    T* cc1 = cc0 + N;
    T* cc2 = cc1 + N;
    const int tid = threadIdx.x, nth = blockDim.x;
    const RT dm = (RT)m;

    // pass A: plain Chebyshev coefficients of F1 = h^2 [v omega]_m, F2 = h^2 [v theta]_m
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b) {
            const int f = (b0 + b == 0) ? 0 : 2;
            T* z = bufA + b * L;
            for (int j = tid; j <= K; j += nth)
                even_extend_store(z, K, j, cscale(G2[g_index(j, f, m, M)], Tab<T>::h2(P, j)));
        }
        T* R = radial_dct1(bufA, bufB, P, nb);
        const RT iK = (RT)(1.0 / (double)K), hK = (RT)(0.5 / (double)K);
        for (int b = 0; b < nb; ++b) {
            T* dst = (b0 + b == 0) ? cc0 : cc1;
            const T* Z = R + b * L;
            for (int n = tid; n <= K; n += nth) dst[n] = cscale(Z[n], (n == 0 || n == K) ? hK : iK);
        }
        __syncthreads();
    }
    // d/ds of both, in place, the two scans side by side (bufA, bufB: scratch)
    cheb_derivative_scan2(cc0, bufA, cc1, bufB, N, P.inv_a);

    // pass B: derivative values on the grid, then N_omega (or N_u) and N_theta;
    // with Ekman pumping N_omega - F_eps and N_u + Ups_eps u_bar (1 + (E/2) omega_0)
    const T* PF = P.pump ? reinterpret_cast<const T*>(P.pump_F) + (size_t)m * N : nullptr;
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b) {
            const T* c = (b0 + b == 0) ? cc0 : cc1;
            T* z = bufA + b * L;
            for (int j = tid; j <= K; j += nth) {
                T v = c[j];
                if (j == 0 || j == K) v = cscale(v, (RT)2);
                even_extend_store(z, K, j, v);
            }
        }
        T* R = radial_dct1(bufA, bufB, P, nb);
        // the grid values of N go to cc2 (omega) and cc0 (theta): cc0 was consumed
        // by the loads above (for NB == 1 the theta pass runs after the omega one)
        for (int b = 0; b < nb; ++b) {
            const int fld = b0 + b;  // 0: omega, 1: theta
            const T* Z = R + b * L;
            T* dst = (fld == 0) ? cc2 : cc0;
            for (int k = tid; k <= K; k += nth) {
                const T dF = cscale(Z[k], (RT)0.5);
                const RT is = Tab<T>::is(P, k);
                T val;
                if (fld == 0) {
                    if (m > 0) {
                        const T uw = G2[g_index(k, 1, m, M)];
                        val = cscale(cadd(dF, cmul_i(uw, dm)), is);
                        if (PF) val = csub(val, PF[k]);
                    } else {
                        const T vw = G2[g_index(k, 0, m, M)];
                        val = cscale(vw, Tab<T>::h2(P, k) * is);
                        if (PF) val = cadd(val, PF[k]);
                    }
                } else {
                    const T ut = G2[g_index(k, 3, m, M)];
                    const T vt = G2[g_index(k, 2, m, M)];
                    val = csub(cscale(cadd(dF, cmul_i(ut, dm)), is), vt);
                }
                dst[k] = val;
            }
        }
        __syncthreads();
    }
    // pass C: Eq. icheb of N_omega (cc2) and N_theta (cc0), truncated to n < nc
    for (int b0 = 0; b0 < 2; b0 += NB) {
        const int nb = min(NB, 2 - b0);
        for (int b = 0; b < nb; ++b) {
            const T* src = (b0 + b == 0) ? cc2 : cc0;
            T* z = bufA + b * L;
            for (int j = tid; j <= K; j += nth) even_extend_store(z, K, j, src[j]);
        }
        T* R = radial_dct1(bufA, bufB, P, nb);
        for (int b = 0; b < nb; ++b) {
            T* dst = (b0 + b == 0) ? cc1 : cc2;  // N_omega_hat -> cc1, N_theta_hat -> cc2
            const T* Z = R + b * L;
            // for NB == 1 the theta pass reads cc0 and writes cc2, which holds
            // nothing needed any more (N_omega_hat went to cc1)
            const RT hc = (RT)(0.5 * P.cnorm);
            for (int n = tid; n < nc; n += nth) dst[n] = cscale(Z[n], hc);
        }
        __syncthreads();
    }
    // integrated right-hand sides; the linear couplings read the FP64 state
    //   e_psi = C^I N_omega_hat + (Ra/Pr)(i m/s_o) C^I theta_hat
    //   e_theta = -D^I N_theta_hat - (alpha/ln eta) i m G^I Psi_hat,  e_u = -D^I N_u_hat
    const double bfac = P.Ra / P.Pr * (double)m / P.s_o;
    const double2* th_m = y.th + (size_t)m * nc;
    const double2* ps_m = y.psi + (size_t)m * nc;
    for (int k = tid; k < nc; k += nth) {
        double2 ep = make_double2(0.0, 0.0), et = make_double2(0.0, 0.0);
        if (k >= 4 && m > 0) {
            ep = band_row<8>(P.ops.band[OP_C], cc1, k, nc);
            if (!P.buoy_imp) ep = cadd(ep, cmul_i(band_row<8>(P.ops.band[OP_C], th_m, k, nc), bfac));
        }
        if (k >= 2) {
            const double2 dn = band_row<4>(P.ops.band[OP_D], cc2, k, nc);
            if (m > 0) {
                const double2 gp = band_row<4>(P.ops.band[OP_G], ps_m, k, nc);
                et = csub(cmul_i(gp, -P.tc * (double)m), dn);
            } else {
                et = cscale(dn, -1.0);
            }
        }
        e.psi[(size_t)m * nc + k] = ep;
        e.th[(size_t)m * nc + k] = et;
        if (m == 0) {
            double eu = 0.0;
            if (k >= 2) eu = -band_row<4>(P.ops.band[OP_D], cc1, k, nc).x;
            e.u[k] = eu;
        }
    }
}

// ---------------------------------------------------------------------------
// Diagnostics from G1 (radial-grid Fourier coefficients written by K1):
// per mode, sums over the Gauss-Lobatto points with quadrature weights q_k
// (int f s ds ~ sum_k q_k f_k) of |u_s|^2 + |u_phi|^2 and |omega|^2;
// u_s = (h^2/s) v.  out[m*2 + 0], out[m*2 + 1].
// ---------------------------------------------------------------------------
__global__ void k_diag_modes(StepParams P, const double2* __restrict__ G1, const double* __restrict__ q,
                             double* __restrict__ out) {
    const int m = blockIdx.x, M = P.M;
    double e = 0.0, z = 0.0;
    for (int k = threadIdx.x; k < P.n_r; k += blockDim.x) {
        const double f = P.coll ? P.inv_s[k] : P.h2[k] * P.inv_s[k];
        const double2 v = G1[g_index(k, 0, m, M)], up = G1[g_index(k, 1, m, M)], w = G1[g_index(k, 2, m, M)];
        const double us2 = f * f * (v.x * v.x + v.y * v.y);
        e += q[k] * (us2 + up.x * up.x + up.y * up.y);
        z += q[k] * (w.x * w.x + w.y * w.y);
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e;
        red[1][threadIdx.x >> 5] = z;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        out[2 * m] = a;
        out[2 * m + 1] = b;
    }
}

// per radius: max |u_s| and max |u_phi| over the azimuthal grid (Eq. fft of
// g = u_s + i l u_phi, l a balancing power of two); out[k*2 + 0], out[k*2 + 1].
__global__ void __launch_bounds__(512) k_phi_cfl(StepParams P, const double2* __restrict__ G1,
                                                 double* __restrict__ out) {
    extern __shared__ double2 sm[];
    const int k = blockIdx.x;
    const int Pn = P.n_phi, M = P.M, n_m = P.n_m;
    double2* X = sm;
    double2* Y = sm + Pn;
    const double f = P.coll ? P.inv_s[k] : P.h2[k] * P.inv_s[k];
    const double2* src = G1 + g_index(k, 0, 0, M);
    __shared__ double red4[4 * 32], mx[4];
    block_max_abs(src, M, 2, n_m + 1, mx, red4);
    const double l = pow2_ratio(f * mx[0], mx[1]);
    load_packed_spectrum(X, src, M, Pn, n_m, f, l);
    double2* R = fft_batched<+1>(X, Y, P.plan_p, 1);
    double ms = 0.0, mp = 0.0;
    for (int j = threadIdx.x; j < Pn; j += blockDim.x) {
        ms = fmax(ms, fabs(R[j].x));
        mp = fmax(mp, fabs(R[j].y));
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        ms = fmax(ms, __shfl_xor_sync(0xffffffffu, ms, o));
        mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ms;
        red[1][threadIdx.x >> 5] = mp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a = fmax(a, red[0][i]);
            b = fmax(b, red[1][i]);
        }
        out[2 * k] = a;
        out[2 * k + 1] = b / l;
    }
}

// per radius: the physical-grid values (Eq. fft) of u_s, u_phi, omega and theta,
// out[k * n_phi + j]; u_s = (h^2/s) v (integration) or v/s (collocation).  The
// pairs (u_s, u_phi) and (omega, theta) travel in one complex transform each,
// balanced by powers of two.
__global__ void __launch_bounds__(512) k_phi_fields(StepParams P, const double2* __restrict__ G1,
                                                    double* __restrict__ us, double* __restrict__ uphi,
                                                    double* __restrict__ omega, double* __restrict__ theta) {
    extern __shared__ double2 sm[];
    const int k = blockIdx.x;
    const int Pn = P.n_phi, M = P.M, n_m = P.n_m;
    double2* X = sm;
    double2* Y = sm + Pn;
    const double f = P.coll ? P.inv_s[k] : P.h2[k] * P.inv_s[k];
    __shared__ double red4[4 * 32], mx[4];
    block_max_abs(G1 + g_index(k, 0, 0, M), M, 4, n_m + 1, mx, red4);
    for (int pass = 0; pass < 2; ++pass) {
        const double2* src = G1 + g_index(k, 2 * pass, 0, M);
        const double fa = (pass == 0) ? f : 1.0;
        const double l = pow2_ratio(fa * mx[2 * pass], mx[2 * pass + 1]);
        load_packed_spectrum(X, src, M, Pn, n_m, fa, l);
        double2* R = fft_batched<+1>(X, Y, P.plan_p, 1);
        double* oa = (pass == 0) ? us : omega;
        double* ob = (pass == 0) ? uphi : theta;
        const double il = 1.0 / l;
        for (int j = threadIdx.x; j < Pn; j += blockDim.x) {
            oa[(size_t)k * Pn + j] = R[j].x;
            ob[(size_t)k * Pn + j] = R[j].y * il;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_diagnostics(const StepParams& P, const double2* G1, const double* q, double* mode_sums,
                               double* radius_max, cudaStream_t st) {
    k_diag_modes<<<P.M, 128, 0, st>>>(P, G1, q, mode_sums);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const size_t sm = smem_phi_products(P);
    const int nth = P.n_phi > 256 * MAXPER ? 512 : 256;
    err = cudaFuncSetAttribute(k_phi_cfl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_phi_cfl<<<P.n_r, nth, sm, st>>>(P, G1, radius_max);
    return cudaGetLastError();
}

cudaError_t launch_phi_fields(const StepParams& P, const double2* G1, double* us, double* uphi, double* omega,
                              double* theta, cudaStream_t st) {
    const size_t sm = smem_phi_products(P);
    cudaError_t err = cudaFuncSetAttribute(k_phi_fields, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_phi_fields<<<P.n_r, 256, sm, st>>>(P, G1, us, uphi, omega, theta);
    return cudaGetLastError();
}

size_t smem_spec_to_grid(const StepParams& P) {
    const int L = 2 * P.K;
    const size_t c = P.fp32 ? sizeof(float2) : sizeof(double2);
    return c * (2 * radial_batch(P) * L + 3 * P.n_r);
}
size_t smem_phi_products(const StepParams& P) {
    return (P.fp32 ? sizeof(float2) : sizeof(double2)) * 2 * P.n_phi;
}
size_t smem_grid_to_spec(const StepParams& P) { return smem_spec_to_grid(P); }

// The explicit stage runs on double2 (FP64) or float2 (option "precision" =
// mixed) grid arrays; G1, G2 hold either type.
// ---------------------------------------------------------------------------
// Large radial grids in FP64 (K = n_r - 1 >= LEAN_K, the half-length DCT-I;
// measured faster than the batched layout from n_r = 513, slower at 257):
// a1 and a3 with three shared arrays of K + 1 entries, X, C, Y (98 KB at
// n_r = 2049), instead of the batched layout's 2 x 2K + 3 n_r entries (229 KB),
// so that two CTAs share an SM and hide each other's barrier and shared-memory
// latency (one CTA left the FP64 pipe ~50 % idle).  The fields of a mode go
// through the transform one after another; the derivative scans run in place on
// C with X as scratch; the DCT-I works in place on the pair (X, Y).  The same
// equations, in the same precision, as k_spec_to_grid / k_grid_to_spec.
// ---------------------------------------------------------------------------
constexpr int LEAN_K = 512;

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// The mixed-precision (FP32) stage takes the lean layout only when asked
// (radial_lean = 1): at n_r = 2049 it ran the mixed step 5.99 against 6.53 ms,
// but the half-length DCT-I builds its odd outputs from a prefix sum over the
// FP32 transform's outputs, which accumulates their rounding: 2.2e-7 from the
// FP64 path after 20 steps against 1.1e-8 with the batched layout's
// even-extension transform.
__host__ __device__ inline bool lean_radial(const StepParams& P) {
    if (P.plan_h.L != P.K || P.K < 128 || P.radial_lean == 0) return false;
    if (P.fp32) return P.radial_lean > 0;
    return P.radial_lean > 0 || P.K >= LEAN_K;
}

// double-float radial transforms in the lean kernels (option "radial_dd"):
// 1 always, 0 never, -1 (default) as the lean layout's own default
__host__ __device__ inline bool radial_dd(const StepParams& P) {
    if (!P.plan_r.twdd || !P.s_dd || P.radial_dd == 0) return false;
    return P.radial_dd > 0 || P.K >= LEAN_K;
}

// The FP64 accumulators of dct1_pair: exact widening of FP32 values by their
// bits (no FP64-unit conversion), the nearest float on the way back
__device__ __forceinline__ double acc_of(double v) { return v; }
__device__ __forceinline__ double acc_of(float v) { return f2d_bits(v); }
__device__ __forceinline__ double2 acc_of(double2 v) { return v; }
__device__ __forceinline__ double2 acc_of(float2 v) { return make_double2(f2d_bits(v.x), f2d_bits(v.y)); }
template <class T>
__device__ __forceinline__ T from_acc(double2 v);
template <>
__device__ __forceinline__ double2 from_acc<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 from_acc<float2>(double2 v) { return make_float2(f32_from_bits(v.x), f32_from_bits(v.y)); }

// DCT-I of x_0..x_K in X (K + 1 entries):
//   C_k = x_0 + (-1)^k x_K + 2 sum_{j=1}^{K-1} x_j cos(pi j k / K),  k = 0..K,
// by one complex FFT of length K, as dct1_batched: y_j = (x_j + x_{K-j})/2
// - sin(pi j/K)(x_j - x_{K-j}) formed in place pair by pair (j, K - j),
// F = FFT(y), C_{2k} = F_k + F_{K-k}, and the odd outputs from
// C_1 = sum_j (x_j - x_{K-j}) cos(pi j/K) by C_{2k+1} = C_{2k-1} - i(F_k - F_{K-k}),
// the prefix sum taken by the whole CTA in FP64 (also for FP32 data, whose
// transform and pair arithmetic stay FP32).  The FFT ping-pongs between X and Y;
// the outputs go to the buffer that does not hold F, which is returned.
// Starts and ends with __syncthreads().
template <class T>
__device__ T* dct1_pair(T* X, T* Y, const StepParams& P) {
    using RT = typename Cx<T>::R;
    const int K = P.plan_h.L, H = K / 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    const T* tw = Cx<T>::tw(P.plan_r);  // tw[j] = (cos(pi j/K), -sin(pi j/K))
    __shared__ double2 wsum[NTHREADS_R / 32];
    __shared__ double2 c1;
    __syncthreads();
    double2 acc = make_double2(0.0, 0.0);
    for (int j = tid; j < H; j += nth) {
        if (j == 0) {
            const T a = X[0], b = X[K];
            T h = a;
            h.x = (RT)0.5 * (a.x + b.x);
            h.y = (RT)0.5 * (a.y + b.y);
            X[0] = h;
            acc = acc_of(csub(a, b));
        } else {
            const T a = X[j], b = X[K - j];
            const RT sn = -tw[j].y, cs = tw[j].x;
            const T sum = cadd(a, b), dif = csub(a, b);
            T lo = sum, hi = sum;
            lo.x = fmat(-sn, dif.x, (RT)0.5 * sum.x);
            lo.y = fmat(-sn, dif.y, (RT)0.5 * sum.y);
            hi.x = fmat(sn, dif.x, (RT)0.5 * sum.x);
            hi.y = fmat(sn, dif.y, (RT)0.5 * sum.y);
            X[j] = lo;
            X[K - j] = hi;
            const double2 dd = acc_of(dif);
            const double c2 = 2.0 * acc_of(cs);
            acc.x = fma(c2, dd.x, acc.x);
            acc.y = fma(c2, dd.y, acc.y);
        }
    }
    // (j = H: y_H = x_H, and its term of C_1 vanishes)
    acc = warp_sum(acc);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        double2 t = wsum[0];
        for (int w = 1; w < nw; ++w) t = cadd(t, wsum[w]);
        c1 = t;
    }
    T* F = fft_batched<+1>(X, Y, P.plan_h, 1);  // begins with a barrier
    T* O = (F == X) ? Y : X;
    for (int k = tid; k <= H; k += nth) O[2 * k] = cadd(F[k], F[k == 0 ? 0 : K - k]);
    // odd outputs: each thread a contiguous chunk of k in [0, H), its sum of
    // d_k = -i (F_k - F_{K-k}) (d_0 = 0), a block-wide exclusive scan, then the chunk
    const int chunk = (H + nth - 1) / nth;
    const int lo = min(tid * chunk, H), hi = min(lo + chunk, H);
    double2 tot = make_double2(0.0, 0.0);
    for (int k = max(lo, 1); k < hi; ++k) {
        const double2 df = acc_of(csub(F[k], F[K - k]));
        tot.x += df.y;
        tot.y -= df.x;
    }
    double2 inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double ux = __shfl_up_sync(0xffffffffu, inc.x, o);
        const double uy = __shfl_up_sync(0xffffffffu, inc.y, o);
        if (lane >= o) {
            inc.x += ux;
            inc.y += uy;
        }
    }
    __syncthreads();  // c1 and the even outputs are published; wsum is free again
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    double2 run = c1;
    for (int w = 0; w < warp; ++w) run = cadd(run, wsum[w]);
    run.x += inc.x - tot.x;
    run.y += inc.y - tot.y;
    for (int k = lo; k < hi; ++k) {
        if (k > 0) {
            const double2 df = acc_of(csub(F[k], F[K - k]));
            run.x += df.y;
            run.y -= df.x;
        }
        O[2 * k + 1] = from_acc<T>(run);
    }
    __syncthreads();
    return O;
}

// ---------------------------------------------------------------------------
// Double-float radial transforms (option "radial_dd", lean layout).  The same
// DCT-I and derivative scan as dct1_pair and cheb_derivative_scan with complex
// double-floats (ddfloat.cuh: about 48 significant bits) on the FP32 pipe, which
// issues 64 times the FP64 rate on GB300; grid and coefficient values cross to
// and from FP64 at the kernels' loads and stores only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ddf dd_shfl_xor(ddf v, int o) {
    return ddf{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ ddf dd_shfl_up(ddf v, int o) {
    return ddf{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ ddf dd_shfl_down(ddf v, int o) {
    return ddf{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ ddc dd_warp_sum(ddc v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x = v.x + dd_shfl_xor(v.x, o);
        v.y = v.y + dd_shfl_xor(v.y, o);
    }
    return v;
}
// an integer |k| < 2^24 as a double-float (exact)
__device__ __forceinline__ ddf dd_int(int k) { return ddf{(float)k, 0.f}; }
__device__ __forceinline__ ddc dd_scale2c(ddc a, float s) { return ddc{dd_scale2(a.x, s), dd_scale2(a.y, s)}; }

// dct1_pair in double-float: X, Y hold K + 1 (resp. the FFT's K) complex
// double-floats; the same steps, the C_1 sum and the prefix sums in double-float.
__device__ ddc* dct1_pair_dd(ddc* X, ddc* Y, const StepParams& P) {
    const int K = P.plan_h.L, H = K / 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    const ddc* tw = reinterpret_cast<const ddc*>(P.plan_r.twdd);  // (cos(pi j/K), -sin(pi j/K))
    __shared__ ddc wsum[NTHREADS_R / 32];
    __shared__ ddc c1;
    __syncthreads();
    ddc acc = ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}};
    for (int j = tid; j < H; j += nth) {
        if (j == 0) {
            const ddc a = X[0], b = X[K];
            X[0] = dd_scale2c(cadd(a, b), 0.5f);
            acc = csub(a, b);
        } else {
            const ddc a = X[j], b = X[K - j];
            const ddc t = ldg_tw(tw + j);
            const ddf sn = -t.y, cs2 = dd_scale2(t.x, 2.f);
            const ddc hs = dd_scale2c(cadd(a, b), 0.5f), dif = csub(a, b);
            X[j] = ddc{hs.x - sn * dif.x, hs.y - sn * dif.y};
            X[K - j] = ddc{hs.x + sn * dif.x, hs.y + sn * dif.y};
            acc = ddc{acc.x + cs2 * dif.x, acc.y + cs2 * dif.y};
        }
    }
    acc = dd_warp_sum(acc);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        ddc t = wsum[0];
        for (int w = 1; w < nw; ++w) t = cadd(t, wsum[w]);
        c1 = t;
    }
    ddc* F = fft_batched<+1, ddc, true>(X, Y, P.plan_h, 1);  // begins with a barrier
    ddc* O = (F == X) ? Y : X;
    for (int k = tid; k <= H; k += nth) O[2 * k] = cadd(F[k], F[k == 0 ? 0 : K - k]);
    const int chunk = (H + nth - 1) / nth;
    const int lo = min(tid * chunk, H), hi = min(lo + chunk, H);
    ddc tot = ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}};
    for (int k = max(lo, 1); k < hi; ++k) {
        const ddc df = csub(F[k], F[K - k]);
        tot = ddc{tot.x + df.y, tot.y - df.x};
    }
    ddc inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const ddf ux = dd_shfl_up(inc.x, o), uy = dd_shfl_up(inc.y, o);
        if (lane >= o) inc = ddc{inc.x + ux, inc.y + uy};
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    ddc run = c1;
    for (int w = 0; w < warp; ++w) run = cadd(run, wsum[w]);
    run = cadd(run, csub(inc, tot));
    for (int k = lo; k < hi; ++k) {
        if (k > 0) {
            const ddc df = csub(F[k], F[K - k]);
            run = ddc{run.x + df.y, run.y - df.x};
        }
        O[2 * k + 1] = run;
    }
    __syncthreads();
    return O;
}

// cheb_derivative_scan in double-float (scale: the x -> s factor, rounded to
// double-float once)
__device__ void cheb_derivative_scan_dd(const ddc* c, ddc* d, ddc* tmp, int n, double scale) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ddc zero = ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}};
    if (warp < 2) {
        const int q = warp;
        const int len = (n - q + 1) / 2;
        const int per = (len + 31) / 32;
        const int i0 = lane * per, i1 = min(i0 + per, len);
        ddc acc = zero;
        for (int i = i1 - 1; i >= i0; --i) {
            const int k = 2 * i + q;
            if (k > 0) {
                const ddf f = dd_int(2 * k);
                acc = ddc{acc.x + f * c[k].x, acc.y + f * c[k].y};
            }
            tmp[k] = acc;
        }
        ddc sfx = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const ddf x = dd_shfl_down(sfx.x, o), y = dd_shfl_down(sfx.y, o);
            if (lane + o < 32) sfx = ddc{sfx.x + x, sfx.y + y};
        }
        const ddc off = csub(sfx, acc);
        for (int i = i0; i < i1; ++i) {
            const int k = 2 * i + q;
            tmp[k] = cadd(tmp[k], off);
        }
    }
    __syncthreads();
    const ddf fs = dd_from(scale), f0 = dd_from(0.5 * scale);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const ddf f = (j == 0) ? f0 : fs;
        d[j] = (j + 1 < n) ? cscale(tmp[j + 1], f) : zero;
    }
    __syncthreads();
}

// The FP64 coefficients as the lean kernels' element type: unchanged in FP64,
// the nearest float in FP32 (bit-level, off the FP64 unit)
template <class T>
__device__ __forceinline__ T to_elem(double2 v);
template <>
__device__ __forceinline__ double2 to_elem<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 to_elem<float2>(double2 v) { return make_float2(f32_from_bits(v.x), f32_from_bits(v.y)); }

// CTAs per SM of the lean kernels: two in FP64 (98 KB of shared memory at
// n_r = 2049), three in FP32 (the FP32 arrays and the FP64 coefficients of a3)
template <class T>
constexpr int lean_ctas() { return sizeof(T) == sizeof(double2) ? 2 : 3; }

// T = double2: the FP64 stage; T = float2: the mixed-precision stage (FP32
// transforms and field arithmetic, grid arrays in FP32, the FP64 state read and
// the analysed coefficients widened to FP64 for the banded applies).
template <class T>
__global__ void __launch_bounds__(NTHREADS_R, lean_ctas<T>()) k_spec_to_grid_lean(StepParams P, VecSet y,
                                                                                  T* __restrict__ G1) {
    using RT = typename Cx<T>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, N = P.n_r, nc = P.nc, M = P.M;
    T* X = reinterpret_cast<T*>(smraw);
    T* C = X + N;   // plain coefficients (Psi, then its derivatives; u_bar)
    T* Y = C + N;   // second DCT buffer (u_bar' for m = 0)
    const int tid = threadIdx.x, nth = blockDim.x;
    const double Cw = P.cnorm, Cw0 = 0.5 * P.cnorm;
    const RT dm = (RT)m;
    const T zero = Cx<T>::make(0.0, 0.0);

    for (int n = tid; n < N; n += nth) {
        double2 a = make_double2(0.0, 0.0);
        if (n < nc) {
            const double w = (n == 0) ? Cw0 : Cw;
            a = (m > 0) ? cscale(y.psi[(size_t)m * nc + n], w) : make_double2(y.u[n] * w, 0.0);
        }
        C[n] = to_elem<T>(a);
    }
    __syncthreads();
    T* PF = P.pump ? reinterpret_cast<T*>(P.pump_F) + (size_t)m * N : nullptr;
    __shared__ double red[4 * 32], mx[4];
    RT lam = (RT)1;
    if (m == 0) {  // u_bar and lam u_bar' packed into one transform (lam a power of two)
        cheb_derivative_scan(C, Y, X, N, P.inv_a);
        block_max_abs(C, N, 2, N, mx, red);
        lam = (RT)pow2_ratio(mx[0], mx[1]);
    }
    // fields: 0 Psi, 1 Psi', 2 Psi'', 3 theta (m >= 1); 4 packed u_bar, 3 theta (m = 0)
    const int nf = (m > 0) ? 4 : 2;
    for (int i = 0; i < nf; ++i) {
        const int fid = (m > 0) ? i : (i == 0 ? 4 : 3);
        if (m > 0 && (fid == 1 || fid == 2)) cheb_derivative_scan(C, C, X, N, P.inv_a);  // C <- dC/ds
        for (int j = tid; j <= K; j += nth) {
            T v;
            if (fid <= 2) {
                v = C[j];
            } else if (fid == 3) {
                v = (j < nc) ? to_elem<T>(cscale(y.th[(size_t)m * nc + j], (j == 0) ? Cw0 : Cw)) : zero;
            } else {
                v = C[j];
                v.y = lam * Y[j].x;
            }
            X[j] = (j == 0 || j == K) ? cscale(v, (RT)2) : v;
        }
        T* Z = dct1_pair(X, Y, P);
        for (int k = tid; k < N; k += nth) {
            const T g = cscale(Z[k], (RT)0.5);  // value of the series at x_k
            const RT s = Tab<T>::s(P, k), h2 = Tab<T>::h2(P, k), is = Tab<T>::is(P, k);
            T* out = G1 + g_index(k, 0, m, M);
            if (fid == 0) {
                out[0] = cmul_i(g, dm);
                out[M] = cscale(g, (RT)3 * s);
                out[2 * M] = cscale(g, (RT)6 + dm * dm * h2 * is * is);
                if (PF) {
                    const RT U = (RT)P.pump_ups[k];
                    PF[k] = cadd(cscale(g, -U * ((RT)P.pump_cr[k] + dm * dm)), cmul_i(g, -U * dm * (RT)P.pump_ci[k]));
                }
            } else if (fid == 1) {
                out[M] = csub(out[M], cscale(g, h2));
                out[2 * M] = csub(out[2 * M], cscale(g, h2 * is - (RT)5 * s));
                if (PF) PF[k] = cadd(PF[k], cscale(g, (RT)P.pump_ups[k] * (RT)0.5 * s));
            } else if (fid == 2) {
                out[2 * M] = csub(out[2 * M], cscale(g, h2));
                if (PF) PF[k] = csub(PF[k], cscale(out[2 * M], (RT)P.pump_ups[k]));
            } else if (fid == 3) {
                out[3 * M] = g;
            } else {
                T o = zero;
                out[0] = o;
                o.x = g.x;
                out[M] = o;
                o.x = g.y / lam + g.x * is;
                out[2 * M] = o;
                if (PF) {
                    const RT w0 = g.y / lam + g.x * is;
                    T pf = zero;
                    pf.x = (RT)P.pump_ups[k] * g.x * ((RT)1 + (RT)(0.5 * P.E) * w0);
                    PF[k] = pf;
                }
            }
        }
        __syncthreads();
    }
}

// byte offset of a3's FP64 coefficient array behind the three T arrays (16-byte
// aligned); in FP64 the coefficients overwrite C instead
template <class T>
__host__ __device__ inline size_t lean_cd_offset(int n_r) {
    return sizeof(T) == sizeof(double2) ? sizeof(T) * (size_t)n_r : (sizeof(T) * 3 * (size_t)n_r + 15) / 16 * 16;
}

template <class T>
__global__ void __launch_bounds__(NTHREADS_R, lean_ctas<T>()) k_grid_to_spec_lean(StepParams P, const T* __restrict__ G2,
                                                                                  VecSet y, VecSet e) {
    using RT = typename Cx<T>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, N = P.n_r, nc = P.nc, M = P.M;
    T* X = reinterpret_cast<T*>(smraw);
    T* C = X + N;
    T* Y = C + N;
    double2* Cd = reinterpret_cast<double2*>(smraw + lean_cd_offset<T>(N));  // FP64 coefficients
    const int tid = threadIdx.x, nth = blockDim.x;
    const RT dm = (RT)m, iK = (RT)(1.0 / (double)K), hK = (RT)(0.5 / (double)K);
    const double dmd = (double)m, hc = 0.5 * P.cnorm;
    const T* PF = P.pump ? reinterpret_cast<const T*>(P.pump_F) + (size_t)m * N : nullptr;
    const double bfac = P.Ra / P.Pr * (double)m / P.s_o;
    // field 0: N_omega (m >= 1) or N_u (m = 0); field 1: N_theta
    for (int fld = 0; fld < 2; ++fld) {
        T* W = X;  // the buffer holding the grid values to analyse
        if (fld == 1 || m > 0) {
            // plain coefficients of F = h^2 [v omega]_m (or h^2 [v theta]_m), d/ds of them
            const int f = (fld == 0) ? 0 : 2;
            for (int j = tid; j <= K; j += nth) X[j] = cscale(G2[g_index(j, f, m, M)], Tab<T>::h2(P, j));
            const T* Z = dct1_pair(X, Y, P);
            for (int n = tid; n <= K; n += nth) C[n] = cscale(Z[n], (n == 0 || n == K) ? hK : iK);
            __syncthreads();
            cheb_derivative_scan(C, C, X, N, P.inv_a);
            for (int j = tid; j <= K; j += nth) X[j] = (j == 0 || j == K) ? cscale(C[j], (RT)2) : C[j];
            const T* D = dct1_pair(X, Y, P);
            W = (D == X) ? Y : X;
            for (int k = tid; k <= K; k += nth) {
                const T dF = cscale(D[k], (RT)0.5);
                const RT is = Tab<T>::is(P, k);
                T val;
                if (fld == 0) {
                    val = cscale(cadd(dF, cmul_i(G2[g_index(k, 1, m, M)], dm)), is);
                    if (PF) val = csub(val, PF[k]);
                } else {
                    val = csub(cscale(cadd(dF, cmul_i(G2[g_index(k, 3, m, M)], dm)), is), G2[g_index(k, 2, m, M)]);
                }
                W[k] = val;
            }
        } else {  // N_u = (h^2/s) [v omega]_0 (+ pumping)
            for (int k = tid; k <= K; k += nth) {
                T val = cscale(G2[g_index(k, 0, m, M)], Tab<T>::h2(P, k) * Tab<T>::is(P, k));
                if (PF) val = cadd(val, PF[k]);
                W[k] = val;
            }
        }
        // Eq. icheb of the grid values, truncated to n < nc
        const T* Z = dct1_pair(W, (W == X) ? Y : X, P);
        // N_omega_hat, with the buoyancy (Ra/Pr)(i m/s_o) theta_hat added before the
        // one C^I apply (Eq. psi_int applies C^I to their sum); Z lives in X or Y,
        // never where the FP64 coefficients go
        const bool buoy = (fld == 0 && m > 0 && !P.buoy_imp);
        for (int n = tid; n < nc; n += nth) {
            const double2 v = cscale(acc_of(Z[n]), hc);
            Cd[n] = buoy ? cadd(v, cmul_i(y.th[(size_t)m * nc + n], bfac)) : v;
        }
        __syncthreads();
        // integrated right-hand sides; the linear couplings read the FP64 state
        for (int k = tid; k < nc; k += nth) {
            if (fld == 0) {
                if (m > 0) {
                    double2 ep = make_double2(0.0, 0.0);
                    if (k >= 4) ep = band_row<8>(P.ops.band[OP_C], Cd, k, nc);
                    e.psi[(size_t)m * nc + k] = ep;
                } else {
                    e.psi[k] = make_double2(0.0, 0.0);
                    e.u[k] = (k >= 2) ? -band_row<4>(P.ops.band[OP_D], Cd, k, nc).x : 0.0;
                }
            } else {
                double2 et = make_double2(0.0, 0.0);
                if (k >= 2) {
                    const double2 dn = band_row<4>(P.ops.band[OP_D], Cd, k, nc);
                    if (m > 0) {
                        const double2 gp = band_row<4>(P.ops.band[OP_G], y.psi + (size_t)m * nc, k, nc);
                        et = csub(cmul_i(gp, -P.tc * dmd), dn);
                    } else {
                        et = cscale(dn, -1.0);
                    }
                }
                e.th[(size_t)m * nc + k] = et;
            }
        }
        __syncthreads();
    }
}

// k_spec_to_grid_lean with double-float transforms: the coefficients become
// double-floats when loaded (the Chebyshev weights applied in double-float), the
// field arithmetic at each radius runs in double-float with double-float tables
// of s, h^2 and 1/s, and each grid value becomes FP64 once, when it is final.
// Between the passes over psi, dpsi/ds and d2psi/ds2 the partial sums of the
// u_phi and omega columns wait in the grid array in double-float form (each CTA
// owns its column m); the pumping flux and the m = 0 column stay FP64.
__global__ void __launch_bounds__(NTHREADS_R, 2) k_spec_to_grid_lean_dd(StepParams P, VecSet y,
                                                                         double2* __restrict__ G1) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, N = P.n_r, nc = P.nc, M = P.M;
    ddc* X = reinterpret_cast<ddc*>(smraw);
    ddc* C = X + N;
    ddc* Y = C + N;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double dm = (double)m;
    const ddf Cw = dd_from(P.cnorm), Cw0 = dd_scale2(Cw, 0.5f);
    const float fm = (float)m;  // exact: m < 2^24
    const ddf fm2 = dd_from(dm * dm);
    const ddf* s_dd = reinterpret_cast<const ddf*>(P.s_dd);
    const ddf* h2_dd = reinterpret_cast<const ddf*>(P.h2_dd);
    const ddf* is_dd = reinterpret_cast<const ddf*>(P.inv_s_dd);
    const ddc zero = ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}};
    for (int n = tid; n < N; n += nth) {
        ddc a = zero;
        if (n < nc) {
            const ddf w = (n == 0) ? Cw0 : Cw;
            a = (m > 0) ? cscale(dd_from_bits(y.psi[(size_t)m * nc + n]), w)
                        : ddc{dd_from_bits(y.u[n]) * w, ddf{0.f, 0.f}};
        }
        C[n] = a;
    }
    __syncthreads();
    double2* PF = P.pump ? P.pump_F + (size_t)m * N : nullptr;
    __shared__ double red[4 * 32], mx[4];
    float lam = 1.f;
    if (m == 0) {  // u_bar and lam u_bar' packed into one transform (lam a power of two)
        cheb_derivative_scan_dd(C, Y, X, N, P.inv_a);
        double a0 = 0.0, a1 = 0.0;  // max |u_bar|, max |u_bar'| (leading parts)
        for (int i = tid; i < N; i += nth) {
            a0 = fmax(a0, fabs((double)C[i].x.hi) + fabs((double)C[i].y.hi));
            a1 = fmax(a1, fabs((double)Y[i].x.hi) + fabs((double)Y[i].y.hi));
        }
        const int warp = tid >> 5, lane = tid & 31;
        for (int o = 16; o > 0; o >>= 1) {
            a0 = fmax(a0, __shfl_xor_sync(0xffffffffu, a0, o));
            a1 = fmax(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        }
        if (lane == 0) {
            red[warp] = a0;
            red[32 + warp] = a1;
        }
        __syncthreads();
        if (tid < 2) {
            double r = 0.0;
            for (int w = 0; w < (nth >> 5); ++w) r = fmax(r, red[tid * 32 + w]);
            mx[tid] = r;
        }
        __syncthreads();
        lam = (float)pow2_ratio(mx[0], mx[1]);
    }
    const int nf = (m > 0) ? 4 : 2;
    for (int i = 0; i < nf; ++i) {
        const int fid = (m > 0) ? i : (i == 0 ? 4 : 3);
        if (m > 0 && (fid == 1 || fid == 2)) cheb_derivative_scan_dd(C, C, X, N, P.inv_a);  // C <- dC/ds
        for (int j = tid; j <= K; j += nth) {
            ddc v;
            if (fid <= 2)
                v = C[j];
            else if (fid == 3)
                v = (j < nc) ? cscale(dd_from_bits(y.th[(size_t)m * nc + j]), (j == 0) ? Cw0 : Cw) : zero;
            else
                v = ddc{C[j].x, dd_scale2(Y[j].x, lam)};
            X[j] = (j == 0 || j == K) ? dd_scale2c(v, 2.f) : v;
        }
        const ddc* Z = dct1_pair_dd(X, Y, P);
        for (int k = tid; k < N; k += nth) {
            const ddc gd = dd_scale2c(Z[k], 0.5f);  // value of the series at x_k
            double2* out = G1 + g_index(k, 0, m, M);
            ddc* outd = reinterpret_cast<ddc*>(out);  // the partial sums, double-float
            if (fid == 0) {
                const ddf h2 = h2_dd[k], is = is_dd[k];
                out[0] = dd_compose(cmul_if(gd, fm));
                outd[M] = cscale(gd, dd_mulf(s_dd[k], 3.f));
                outd[2 * M] = cscale(gd, h2 * (is * is) * fm2 + ddf{6.f, 0.f});
                if (PF) {
                    const double2 g = dd_compose(gd);
                    const double U = P.pump_ups[k];
                    PF[k] = cadd(cscale(g, -U * (P.pump_cr[k] + dm * dm)), cmul_i(g, -U * dm * P.pump_ci[k]));
                }
            } else if (fid == 1) {
                const ddf s_ = s_dd[k], h2 = h2_dd[k];
                out[M] = dd_compose(csub(outd[M], cscale(gd, h2)));
                outd[2 * M] = csub(outd[2 * M], cscale(gd, h2 * is_dd[k] - dd_mulf(s_, 5.f)));
                if (PF) PF[k] = cadd(PF[k], cscale(dd_compose(gd), P.pump_ups[k] * 0.5 * P.s[k]));
            } else if (fid == 2) {
                const double2 o2 = dd_compose(csub(outd[2 * M], cscale(gd, h2_dd[k])));
                out[2 * M] = o2;
                if (PF) PF[k] = csub(PF[k], cscale(o2, P.pump_ups[k]));
            } else if (fid == 3) {
                out[3 * M] = dd_compose(gd);
            } else {
                const double2 g = dd_compose(gd);
                const double is = P.inv_s[k];
                out[0] = make_double2(0.0, 0.0);
                out[M] = make_double2(g.x, 0.0);
                out[2 * M] = make_double2(g.y / (double)lam + g.x * is, 0.0);
                if (PF) {
                    const double w0 = g.y / (double)lam + g.x * is;
                    PF[k] = make_double2(P.pump_ups[k] * g.x * (1.0 + 0.5 * P.E * w0), 0.0);
                }
            }
        }
        __syncthreads();
    }
}

// k_grid_to_spec_lean with double-float transforms: grid values become
// double-floats when loaded, the flux divergence is formed in double-float at
// each radius from the double-float derivative (double-float tables of h^2 and
// 1/s), and the analysed coefficients, with the explicit buoyancy added in
// double-float, are FP64 again (in C, over the double-float data) before the
// FP64 banded applies.  The pumping flux is read in FP64.
__global__ void __launch_bounds__(NTHREADS_R, 2) k_grid_to_spec_lean_dd(StepParams P, const double2* __restrict__ G2,
                                                                         VecSet y, VecSet e) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = P.m_lo + blockIdx.x;
    const int K = P.K, N = P.n_r, nc = P.nc, M = P.M;
    ddc* X = reinterpret_cast<ddc*>(smraw);
    ddc* C = X + N;
    ddc* Y = C + N;
    double2* Cd = reinterpret_cast<double2*>(C);  // the analysed coefficients, FP64
    const int tid = threadIdx.x, nth = blockDim.x;
    const double dm = (double)m;
    const ddf hc = dd_from(0.5 * P.cnorm);
    const float iK = 1.f / (float)K, hK = 0.5f / (float)K;  // K a power of two: exact
    const float fm = (float)m;                               // exact: m < 2^24
    const double2* PF = P.pump ? P.pump_F + (size_t)m * N : nullptr;
    const ddf bfac = dd_from(P.Ra / P.Pr * (double)m / P.s_o);
    const ddf* h2_dd = reinterpret_cast<const ddf*>(P.h2_dd);
    const ddf* is_dd = reinterpret_cast<const ddf*>(P.inv_s_dd);
    for (int fld = 0; fld < 2; ++fld) {
        ddc* W = X;
        if (fld == 1 || m > 0) {
            const int f = (fld == 0) ? 0 : 2;
            for (int j = tid; j <= K; j += nth) X[j] = cscale(dd_from_bits(G2[g_index(j, f, m, M)]), h2_dd[j]);
            const ddc* Z = dct1_pair_dd(X, Y, P);
            for (int n = tid; n <= K; n += nth) C[n] = dd_scale2c(Z[n], (n == 0 || n == K) ? hK : iK);
            __syncthreads();
            cheb_derivative_scan_dd(C, C, X, N, P.inv_a);
            for (int j = tid; j <= K; j += nth) X[j] = (j == 0 || j == K) ? dd_scale2c(C[j], 2.f) : C[j];
            const ddc* D = dct1_pair_dd(X, Y, P);
            W = (D == X) ? Y : X;
            for (int k = tid; k <= K; k += nth) {
                const ddc dF = dd_scale2c(D[k], 0.5f);
                const ddf is = is_dd[k];
                ddc val;
                if (fld == 0) {
                    val = cscale(cadd(dF, cmul_if(dd_from_bits(G2[g_index(k, 1, m, M)]), fm)), is);
                    if (PF) val = csub(val, dd_from_bits(PF[k]));
                } else {
                    val = csub(cscale(cadd(dF, cmul_if(dd_from_bits(G2[g_index(k, 3, m, M)]), fm)), is),
                               dd_from_bits(G2[g_index(k, 2, m, M)]));
                }
                W[k] = val;
            }
        } else {  // N_u = (h^2/s) [v omega]_0 (+ pumping)
            for (int k = tid; k <= K; k += nth) {
                ddc val = cscale(dd_from_bits(G2[g_index(k, 0, m, M)]), h2_dd[k] * is_dd[k]);
                if (PF) val = cadd(val, dd_from_bits(PF[k]));
                W[k] = val;
            }
        }
        const ddc* Z = dct1_pair_dd(W, (W == X) ? Y : X, P);
        const bool buoy = (fld == 0 && m > 0 && !P.buoy_imp);
        // Z lives in X or Y, never in C: the FP64 coefficients overwrite C
        for (int n = tid; n < nc; n += nth) {
            const ddc v = cscale(Z[n], hc);
            if (buoy) {
                const ddc t = dd_from_bits(y.th[(size_t)m * nc + n]);
                Cd[n] = dd_compose(ddc{v.x - t.y * bfac, v.y + t.x * bfac});  // + i bfac theta
            } else {
                Cd[n] = dd_compose(v);
            }
        }
        __syncthreads();
        for (int k = tid; k < nc; k += nth) {
            if (fld == 0) {
                if (m > 0) {
                    double2 ep = make_double2(0.0, 0.0);
                    if (k >= 4) ep = band_row<8>(P.ops.band[OP_C], Cd, k, nc);
                    e.psi[(size_t)m * nc + k] = ep;
                } else {
                    e.psi[k] = make_double2(0.0, 0.0);
                    e.u[k] = (k >= 2) ? -band_row<4>(P.ops.band[OP_D], Cd, k, nc).x : 0.0;
                }
            } else {
                double2 et = make_double2(0.0, 0.0);
                if (k >= 2) {
                    const double2 dn = band_row<4>(P.ops.band[OP_D], Cd, k, nc);
                    if (m > 0) {
                        const double2 gp = band_row<4>(P.ops.band[OP_G], y.psi + (size_t)m * nc, k, nc);
                        et = csub(cmul_i(gp, -P.tc * dm), dn);
                    } else {
                        et = cscale(dn, -1.0);
                    }
                }
                e.th[(size_t)m * nc + k] = et;
            }
        }
        __syncthreads();
    }
}

size_t smem_radial_lean(const StepParams& P) { return sizeof(double2) * 3 * (size_t)P.n_r; }
// the FP32 lean kernels: three float2 arrays; a3 also the FP64 coefficients
static size_t smem_radial_lean32(const StepParams& P, bool analysis) {
    return analysis ? lean_cd_offset<float2>(P.n_r) + sizeof(double2) * (size_t)P.nc : sizeof(float2) * 3 * (size_t)P.n_r;
}

template <class T>
static cudaError_t spec_to_grid_t(const StepParams& P, VecSet y, void* G1, cudaStream_t st) {
    const size_t sm = smem_spec_to_grid(P);
    cudaError_t err = cudaFuncSetAttribute(k_spec_to_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_spec_to_grid<T><<<slab_modes(P), NTHREADS_R, sm, st>>>(P, y, static_cast<T*>(G1));
    return cudaGetLastError();
}

// 1 when the azimuthal kernels can hold both packed pairs at once (twice
// smem_phi_products: n_phi <= 3072 in FP64), else 0
static int phi_pair(const StepParams& P, cudaError_t& err) {
    int dev = 0, smax = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (err == cudaSuccess && 2 * smem_phi_products(P) <= (size_t)smax) ? 1 : 0;
}

template <class T>
static cudaError_t phi_products_t(const StepParams& P, const void* G1, void* G2, cudaStream_t st) {
    const int nth = phi_threads(P);
    if (P.n_phi > nth * MAXPER || nth > 512) return cudaErrorInvalidValue;
    cudaError_t err;
    const int pair = phi_pair(P, err);
    if (err != cudaSuccess) return err;
    const size_t sm = (pair ? 2 : 1) * smem_phi_products(P);
    err = cudaFuncSetAttribute(k_phi_products<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_phi_products<T><<<slab_radii(P), nth, sm, st>>>(P, static_cast<const T*>(G1), static_cast<T*>(G2), pair);
    return cudaGetLastError();
}

template <class T>
static cudaError_t grid_to_spec_t(const StepParams& P, const void* G2, VecSet y, VecSet e, cudaStream_t st) {
    const size_t sm = smem_grid_to_spec(P);
    cudaError_t err = cudaFuncSetAttribute(k_grid_to_spec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_grid_to_spec<T><<<slab_modes(P), NTHREADS_R, sm, st>>>(P, static_cast<const T*>(G2), y, e);
    return cudaGetLastError();
}

cudaError_t launch_spec_to_grid(const StepParams& P, VecSet y, double2* G1, cudaStream_t st) {
    if (lean_radial(P) && P.fp32) {
        const size_t sm = smem_radial_lean32(P, false);
        cudaError_t err =
            cudaFuncSetAttribute(k_spec_to_grid_lean<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_spec_to_grid_lean<float2><<<slab_modes(P), NTHREADS_R, sm, st>>>(P, y, reinterpret_cast<float2*>(G1));
        return cudaGetLastError();
    }
    if (lean_radial(P)) {
        const size_t sm = smem_radial_lean(P);
        auto kern = radial_dd(P) ? k_spec_to_grid_lean_dd : k_spec_to_grid_lean<double2>;
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        kern<<<slab_modes(P), NTHREADS_R, sm, st>>>(P, y, G1);
        return cudaGetLastError();
    }
    return P.fp32 ? spec_to_grid_t<float2>(P, y, G1, st) : spec_to_grid_t<double2>(P, y, G1, st);
}

cudaError_t launch_phi_products(const StepParams& P, const double2* G1, double2* G2, cudaStream_t st) {
    if (P.fp32) return phi_products_t<float2>(P, G1, G2, st);
    if (P.phi_dd && P.plan_p.twdd) {
        const int nth = phi_threads(P);
        if (P.n_phi > nth * MAXPER || nth > 512) return cudaErrorInvalidValue;
        // the batched pair of transforms needs twice the buffers (n_phi <= 3072)
        cudaError_t err;
        const int pair = phi_pair(P, err);
        if (err != cudaSuccess) return err;
        const size_t sm = (pair ? 2 : 1) * smem_phi_products(P);
        err = cudaFuncSetAttribute(k_phi_products_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_phi_products_dd<<<slab_radii(P), nth, sm, st>>>(P, G1, G2, pair);
        return cudaGetLastError();
    }
    return phi_products_t<double2>(P, G1, G2, st);
}

cudaError_t launch_grid_to_spec(const StepParams& P, const double2* G2, VecSet y, VecSet e, cudaStream_t st) {
    if (lean_radial(P) && P.fp32) {
        const size_t sm = smem_radial_lean32(P, true);
        cudaError_t err =
            cudaFuncSetAttribute(k_grid_to_spec_lean<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_grid_to_spec_lean<float2><<<slab_modes(P), NTHREADS_R, sm, st>>>(P, reinterpret_cast<const float2*>(G2), y, e);
        return cudaGetLastError();
    }
    if (lean_radial(P)) {
        const size_t sm = smem_radial_lean(P);
        auto kern = radial_dd(P) ? k_grid_to_spec_lean_dd : k_grid_to_spec_lean<double2>;
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        kern<<<slab_modes(P), NTHREADS_R, sm, st>>>(P, G2, y, e);
        return cudaGetLastError();
    }
    return P.fp32 ? grid_to_spec_t<float2>(P, G2, y, e, st) : grid_to_spec_t<double2>(P, G2, y, e, st);
}

}  // namespace pz
