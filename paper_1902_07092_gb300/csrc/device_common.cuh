// Device helpers: complex arithmetic, CTA-cooperative mixed-radix Stockham FFT in
// shared memory, the DCT-I of the Gauss-Lobatto grid (Eqs. cheb and icheb of
// Section 3) through an FFT of the even extension, and the Chebyshev derivative
// of plain coefficients by a parity-split suffix scan.
#pragma once
#include <cuda_runtime.h>

#include "ddfloat.cuh"
#include "pizza_internal.h"

namespace pz {

// complex arithmetic on double2 (FP64) and float2 (FP32)
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// multiply by i*t (t real)
__device__ __forceinline__ double2 cmul_i(double2 a, double t) { return make_double2(-a.y * t, a.x * t); }

// a + w*b and 2a - (a + w*b) = a - w*b with fused multiply-adds
__device__ __forceinline__ double2 cfma(double2 w, double2 b, double2 a) {
    return make_double2(fma(w.x, b.x, fma(-w.y, b.y, a.x)), fma(w.x, b.y, fma(w.y, b.x, a.y)));
}
__device__ __forceinline__ double2 creflect(double2 a, double2 s) {  // 2a - s
    return make_double2(fma(2.0, a.x, -s.x), fma(2.0, a.y, -s.y));
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_i(float2 a, float t) { return make_float2(-a.y * t, a.x * t); }
__device__ __forceinline__ float2 cfma(float2 w, float2 b, float2 a) {
    return make_float2(fmaf(w.x, b.x, fmaf(-w.y, b.y, a.x)), fmaf(w.x, b.y, fmaf(w.y, b.x, a.y)));
}
__device__ __forceinline__ float2 creflect(float2 a, float2 s) {
    return make_float2(fmaf(2.0f, a.x, -s.x), fmaf(2.0f, a.y, -s.y));
}

// fused multiply-add in the precision of its arguments (never promoted to FP64)
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

// Real type, constructor and conversions of the two complex types.
template <class T>
struct Cx;
template <>
struct Cx<double2> {
    using R = double;
    __device__ static double2 make(double a, double b) { return make_double2(a, b); }
    __device__ static double2 from(double2 a) { return a; }
    __device__ static const double2* tw(const FftPlan& p) { return p.tw; }
};
template <>
struct Cx<float2> {
    using R = float;
    __device__ static float2 make(double a, double b) { return make_float2((float)a, (float)b); }
    __device__ static float2 from(double2 a) { return make_float2((float)a.x, (float)a.y); }
    __device__ static const float2* tw(const FftPlan& p) { return p.twf; }
};
template <>
struct Cx<ddc> {
    using R = ddf;
    __device__ static ddc make(double a, double b) { return ddc{dd_from(a), dd_from(b)}; }
    __device__ static ddc from(double2 a) { return dd_from(a); }
    __device__ static const ddc* tw(const FftPlan& p) { return reinterpret_cast<const ddc*>(p.twdd); }
};
// a real constant in the real type of a complex type
template <class RT>
__device__ __forceinline__ RT rconst(double c) {
    return (RT)c;
}
template <>
__device__ __forceinline__ ddf rconst<ddf>(double c) {
    return dd_from(c);
}
// twiddle load through the read-only cache
template <class T>
__device__ __forceinline__ T ldg_tw(const T* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ ddc ldg_tw<ddc>(const ddc* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return ddc{ddf{v.x, v.y}, ddf{v.z, v.w}};
}
// radial tables in the precision of the complex type
template <class T>
struct Tab;
template <>
struct Tab<double2> {
    __device__ static double s(const StepParams& P, int k) { return P.s[k]; }
    __device__ static double h2(const StepParams& P, int k) { return P.h2[k]; }
    __device__ static double is(const StepParams& P, int k) { return P.inv_s[k]; }
};
template <>
struct Tab<float2> {
    __device__ static float s(const StepParams& P, int k) { return P.s_f[k]; }
    __device__ static float h2(const StepParams& P, int k) { return P.h2_f[k]; }
    __device__ static float is(const StepParams& P, int k) { return P.inv_s_f[k]; }
};
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2((double)a.x, (double)a.y); }

// 4-point DFT y_k = sum_n a_n e^(SIGN 2 pi i nk/4) (SIGN = -1 forward, +1 backward)
template <int SIGN, class T>
__device__ __forceinline__ void dft4(T a0, T a1, T a2, T a3, T* y) {
    const T t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
    T rt;  // forward: -i t3, backward: +i t3
    if (SIGN < 0) {
        rt.x = t3.y;
        rt.y = -t3.x;
    } else {
        rt.x = -t3.y;
        rt.y = t3.x;
    }
    y[0] = cadd(t0, t2);
    y[2] = csub(t0, t2);
    y[1] = cadd(t1, rt);
    y[3] = csub(t1, rt);
}

// One Stockham pass of radix R over a batch of nb transforms of length L, on
// complex type T (double2 or float2).
// SIGN = -1: forward  sum_j x_j exp(-2 pi i jk/L);  SIGN = +1: backward (unscaled).
// In the first pass (Ns = 1) every twiddle factor is 1 and the multiplies are
// skipped; otherwise the twiddle products are fused into the butterfly adds.
template <int SIGN, int R, bool FIRST, class T>
__device__ __forceinline__ void stockham_pass(const T* __restrict__ src, T* __restrict__ dst, int L, int Ns,
                                              const T* __restrict__ tw, int tws, int nb, int tid, int nth) {
    using RT = typename Cx<T>::R;
    const int nbf = L / R;
    const int twmul = L / (Ns * R) * tws;
    constexpr bool first = FIRST;
    for (int t = tid; t < nb * nbf; t += nth) {
        const int bt = t / nbf;
        const int j = t - bt * nbf;
        const T* s = src + (size_t)bt * L;
        T* d = dst + (size_t)bt * L;
        const int k = j % Ns;
        T v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[j + r * nbf];
        T w[R];
        w[0] = Cx<T>::make(1.0, 0.0);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            w[r] = first ? Cx<T>::make(1.0, 0.0) : ldg_tw(&tw[r * k * twmul]);
            if (SIGN > 0) w[r].y = -w[r].y;
        }
        if (R == 2) {
            T y0 = first ? cadd(v[0], v[1]) : cfma(w[1], v[1], v[0]);
            v[1] = first ? csub(v[0], v[1]) : creflect(v[0], y0);
            v[0] = y0;
        } else if (R == 4) {
            T t0, t1, t2, t3;
            if (first) {
                t0 = cadd(v[0], v[2]);
                t1 = csub(v[0], v[2]);
                t2 = cadd(v[1], v[3]);
                t3 = csub(v[1], v[3]);
            } else {
                t0 = cfma(w[2], v[2], v[0]);          // v0 + w2 v2
                t1 = creflect(v[0], t0);              // v0 - w2 v2
                const T b1 = cmul(w[1], v[1]);
                t2 = cfma(w[3], v[3], b1);            // w1 v1 + w3 v3
                t3 = creflect(b1, t2);                // w1 v1 - w3 v3
            }
            // forward: -i*t3 ; backward: +i*t3
            T rt;
            if (SIGN < 0) {
                rt.x = t3.y;
                rt.y = -t3.x;
            } else {
                rt.x = -t3.y;
                rt.y = t3.x;
            }
            v[0] = cadd(t0, t2);
            v[2] = csub(t0, t2);
            v[1] = cadd(t1, rt);
            v[3] = csub(t1, rt);
        } else if (R == 3) {
            const RT h3 = rconst<RT>(0.86602540378443864676);  // sqrt(3)/2
            T t1, t2;
            if (first) {
                t1 = cadd(v[1], v[2]);
                t2 = csub(v[1], v[2]);
            } else {
                const T b1 = cmul(w[1], v[1]);
                t1 = cfma(w[2], v[2], b1);            // w1 v1 + w2 v2
                t2 = creflect(b1, t1);                // w1 v1 - w2 v2
            }
            T m1;
            m1.x = fmat(rconst<RT>(-0.5), t1.x, v[0].x);
            m1.y = fmat(rconst<RT>(-0.5), t1.y, v[0].y);
            // forward: -i*h3*t2 ; backward: +i*h3*t2
            T rt;
            if (SIGN < 0) {
                rt.x = t2.y;
                rt.y = -t2.x;
            } else {
                rt.x = -t2.y;
                rt.y = t2.x;
            }
            v[0] = cadd(v[0], t1);
            v[1].x = fmat(h3, rt.x, m1.x);
            v[1].y = fmat(h3, rt.y, m1.y);
            v[2].x = fmat(-h3, rt.x, m1.x);
            v[2].y = fmat(-h3, rt.y, m1.y);        } else if (R == 8) {
            // 8-point DFT of x_r = w_r v_r: 4-point DFTs of the even and of the odd
            // samples, the odd ones times e^(-/+ 2 pi i k/8), then one radix-2 level
            T x[8];
            x[0] = v[0];
#pragma unroll
            for (int r = 1; r < 8; ++r) x[r] = first ? v[r] : cmul(w[r], v[r]);
            T e[4], o[4];
            dft4<SIGN>(x[0], x[2], x[4], x[6], e);
            dft4<SIGN>(x[1], x[3], x[5], x[7], o);
            const RT c = rconst<RT>(0.70710678118654752440);  // 1/sqrt(2)
            T o1, o2, o3;
            if (SIGN < 0) {  // (1 - i)/sqrt2, -i, (-1 - i)/sqrt2
                o1.x = (o[1].x + o[1].y) * c;
                o1.y = (o[1].y - o[1].x) * c;
                o2.x = o[2].y;
                o2.y = -o[2].x;
                o3.x = (o[3].y - o[3].x) * c;
                o3.y = -((o[3].x + o[3].y) * c);
            } else {         // (1 + i)/sqrt2, +i, (-1 + i)/sqrt2
                o1.x = (o[1].x - o[1].y) * c;
                o1.y = (o[1].x + o[1].y) * c;
                o2.x = -o[2].y;
                o2.y = o[2].x;
                o3.x = -((o[3].x + o[3].y) * c);
                o3.y = (o[3].x - o[3].y) * c;
            }
            v[0] = cadd(e[0], o[0]);
            v[4] = csub(e[0], o[0]);
            v[1] = cadd(e[1], o1);
            v[5] = csub(e[1], o1);
            v[2] = cadd(e[2], o2);
            v[6] = csub(e[2], o2);
            v[3] = cadd(e[3], o3);
            v[7] = csub(e[3], o3);
        }
        const int idx = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[idx + r * Ns] = v[r];
    }
}

// Batched FFT of nb transforms stored contiguously in buf0 (each length pl.L);
// buf1 is scratch of the same size.  Ends with __syncthreads(); returns the buffer
// holding the result.
template <int SIGN, class T, bool R8 = false>
__device__ __forceinline__ T* fft_batched(T* buf0, T* buf1, const FftPlan& pl, int nb) {
    T* a = buf0;
    T* b = buf1;
    int Ns = 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const T* tw = Cx<T>::tw(pl);
    // FP32 (and R8 callers): the radix-8 factorisation, fewer passes
    constexpr bool f32 = R8 || sizeof(typename Cx<T>::R) == sizeof(float);
    const int npass = f32 ? pl.npass8 : pl.npass;
    __syncthreads();
    for (int p = 0; p < npass; ++p) {
        const int R = f32 ? pl.radix8[p] : pl.radix[p];
        if (p == 0) {  // Ns == 1: unit twiddles
            if (R == 8)
                stockham_pass<SIGN, 8, true>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else if (R == 4)
                stockham_pass<SIGN, 4, true>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else if (R == 2)
                stockham_pass<SIGN, 2, true>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else
                stockham_pass<SIGN, 3, true>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
        } else {
            if (R == 8)
                stockham_pass<SIGN, 8, false>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else if (R == 4)
                stockham_pass<SIGN, 4, false>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else if (R == 2)
                stockham_pass<SIGN, 2, false>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
            else
                stockham_pass<SIGN, 3, false>(a, b, pl.L, Ns, tw, pl.tws, nb, tid, nth);
        }
        __syncthreads();
        T* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// DCT-I of nb complex vectors by one complex FFT of length K each (half the
// length of the even-extension transform).  Input x_b[j], j = 0..K (K a power of
// two), at buf0[b * 2K + j]; output at the same places:
//   C_k = x_0 + (-1)^k x_K + 2 sum_{j=1}^{K-1} x_j cos(pi j k / K),  k = 0..K,
// i.e. the transform of the even extension of x.  With
//   y_j = (x_j + x_{K-j})/2 - sin(pi j/K) (x_j - x_{K-j}),  j = 0..K-1,
//   F_k = sum_j y_j exp(+2 pi i j k/K),
// the even outputs are C_{2k} = F_k + F_{K-k} (F_K = F_0) and the odd ones follow
// from C_1 = sum_j (x_j - x_{K-j}) cos(pi j/K) by C_{2k+1} = C_{2k-1} - i (F_k - F_{K-k})
// (the cosine-sum recurrence of the real-data case, applied to the real and
// imaginary parts at once), a prefix sum taken by one warp per vector.
// plan_h: length K; plan_r: length 2K, whose twiddles give cos and sin(pi j/K).
// The sum for C_1 and the prefix sum are accumulated in FP64.
// buf1: scratch of 2 nb K entries.  nb <= 4.  Starts and ends with __syncthreads().
template <class T>
__device__ T* dct1_batched(T* buf0, T* buf1, const FftPlan& plan_h, const FftPlan& plan_r, int nb) {
    using RT = typename Cx<T>::R;
    const int K = plan_h.L, L = 2 * K, H = K / 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const T* tw = Cx<T>::tw(plan_r);  // tw[j] = (cos(pi j/K), -sin(pi j/K))
    __shared__ double2 c1s[4];
    __syncthreads();
    for (int t = tid; t < nb * K; t += nth) {
        const int b = t / K, j = t - b * K;
        const T* x = buf0 + (size_t)b * L;
        const T xa = x[j], xb = x[K - j];
        const RT s = -tw[j].y;
        const T sum = cadd(xa, xb), dif = csub(xa, xb);
        T y;
        y.x = fmat(-s, dif.x, (RT)0.5 * sum.x);
        y.y = fmat(-s, dif.y, (RT)0.5 * sum.y);
        buf1[(size_t)b * K + j] = y;
    }
    if (warp < nb) {
        const T* x = buf0 + (size_t)warp * L;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = lane; j < K; j += 32) {
            const T dif = csub(x[j], x[K - j]);
            const double c = (double)tw[j].x;
            acc.x = fma(c, (double)dif.x, acc.x);
            acc.y = fma(c, (double)dif.y, acc.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) c1s[warp] = acc;
    }
    T* F = fft_batched<+1>(buf1, buf1 + (size_t)nb * K, plan_h, nb);
    // even outputs
    for (int t = tid; t < nb * (H + 1); t += nth) {
        const int b = t / (H + 1), k = t - b * (H + 1);
        const T* f = F + (size_t)b * K;
        buf0[(size_t)b * L + 2 * k] = cadd(f[k], f[k == 0 ? 0 : K - k]);
    }
    // odd outputs: prefix sum of d_k = -i (F_k - F_{K-k}), d_0 = 0, one warp per vector
    if (warp < nb) {
        const T* f = F + (size_t)warp * K;
        T* out = buf0 + (size_t)warp * L;
        const int chunk = (H + 31) / 32;
        const int lo = min(lane * chunk, H), hi = min(lo + chunk, H);
        double2 tot = make_double2(0.0, 0.0);
        for (int k = lo; k < hi; ++k) {
            if (k == 0) continue;
            const T df = csub(f[k], f[K - k]);
            tot.x += (double)df.y;
            tot.y -= (double)df.x;
        }
        // exclusive scan of the chunk totals across the warp
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
        double2 run = c1s[warp];
        run.x += inc.x - tot.x;
        run.y += inc.y - tot.y;
        for (int k = lo; k < hi; ++k) {
            if (k > 0) {
                const T df = csub(f[k], f[K - k]);
                run.x += (double)df.y;
                run.y -= (double)df.x;
            }
            out[2 * k + 1] = Cx<T>::from(run);
        }
    }
    __syncthreads();
    return buf0;
}

// The radial DCT-I of nb even-extended vectors in buf0 (stride 2K): in FP64 by
// the half-length transform when the plan is set and K >= 128, else by the FFT
// of the even extension.  At small K the extra reduction and scan phases cost
// more latency than the shorter transform saves; in FP32 the odd outputs'
// differences F_k - F_{K-k} cancel to a few ulps of F each and their sum loses
// more than the FP32 transform's own rounding (measured: 50x the state error of
// the mixed path after 50 steps at n_r = 2049), so FP32 keeps the long transform.
// Result at the returned pointer, vector b at [b * 2K + k], k <= K.
template <class T>
__device__ __forceinline__ T* radial_dct1(T* buf0, T* buf1, const StepParams& P, int nb) {
    constexpr bool fp64 = sizeof(typename Cx<T>::R) == sizeof(double);
    if (fp64 && P.plan_h.L == P.K && P.K >= 128) return dct1_batched(buf0, buf1, P.plan_h, P.plan_r, nb);
    return fft_batched<-1>(buf0, buf1, P.plan_r, nb);
}

// 2^e with e the difference of the binary exponents of a and b (1 when either
// is zero), clamped to |e| <= 400.  Two real fields packed into one complex
// transform as a + i (scale) b are given comparable magnitudes this way: the
// scaling is exact, and the rounding of the transform then stays relative to
// each field instead of to the larger one.
__device__ __forceinline__ double pow2_ratio(double a, double b) {
    if (!(a > 0.0) || !(b > 0.0)) return 1.0;
    const int e = max(-400, min(400, ilogb(a) - ilogb(b)));
    return ldexp(1.0, e);
}
// the exponent e of pow2_ratio, clamped to |e| <= lim
__device__ __forceinline__ int pow2_exponent(double a, double b, int lim) {
    if (!(a > 0.0) || !(b > 0.0)) return 0;
    return max(-lim, min(lim, ilogb(a) - ilogb(b)));
}
__device__ __forceinline__ float pow2f(int e) { return ldexpf(1.0f, e); }
__device__ __forceinline__ double pow2d(int e) { return ldexp(1.0, e); }

// CTA-wide max over m < n of |re| + |im| of the nf <= 4 rows src + f*stride,
// into out[f] (shared).  red: shared scratch of 4*32 doubles.  Whole CTA.
template <class T>
__device__ __forceinline__ void block_max_abs(const T* src, int stride, int nf, int n, double* out, double* red) {
    using RT = typename Cx<T>::R;
    RT mx[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (f < nf) {
                const T v = src[(size_t)f * stride + i];
                mx[f] = max(mx[f], abs(v.x) + abs(v.y));
            }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        for (int o = 16; o > 0; o >>= 1) mx[f] = max(mx[f], __shfl_xor_sync(0xffffffffu, mx[f], o));
        if (lane == 0) red[f * 32 + warp] = (double)mx[f];
    }
    __syncthreads();
    if (threadIdx.x < nf) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[threadIdx.x * 32 + w]);
        out[threadIdx.x] = r;
    }
    __syncthreads();
}

// Load the even extension of coefficients a_0..a_K (complex) into z (length 2K):
// z_j = a_j (j <= K), z_{2K-j} = a_j.  The FFT of z then gives
// Z_n = 2 sum''_{j=0..K} a_j cos(pi n j/K),  n = 0..K (the DCT-I core).
template <class T>
__device__ __forceinline__ void even_extend_store(T* z, int K, int j, T aj) {
    z[j] = aj;
    if (j > 0 && j < K) z[2 * K - j] = aj;
}

// Chebyshev derivative in x of plain coefficients c[0..n-1] -> d[0..n-1]
// (d[n-1] = 0):  d_j = (2/c_j) sum_{k>j, k+j odd} k c_k  (c_0 = 2, c_j = 1),
// i.e. suffix sums of t_k = 2 k c_k over each index parity.  Work-efficient:
// warp q (q = 0, 1) owns the indices k = 2i + q; each lane sums a contiguous
// chunk sequentially, a shuffle scan adds the totals of the chunks above it.
// ``tmp`` is scratch of n entries.  Must be called by the whole CTA (>= 64 threads).
template <class T>
__device__ __forceinline__ void cheb_derivative_scan(const T* c, T* d, T* tmp, int n, double scale) {
    using RT = typename Cx<T>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2) {
        const int q = warp;
        const int len = (n - q + 1) / 2;  // number of k = 2i + q below n
        const int per = (len + 31) / 32;
        const int i0 = lane * per, i1 = min(i0 + per, len);
        T acc = Cx<T>::make(0.0, 0.0);
        for (int i = i1 - 1; i >= i0; --i) {
            const int k = 2 * i + q;
            if (k > 0) {
                const RT f = (RT)(2 * k);
                acc.x = fmat(f, c[k].x, acc.x);
                acc.y = fmat(f, c[k].y, acc.y);
            }
            tmp[k] = acc;
        }
        // inclusive suffix scan of the chunk totals over the lanes
        T sfx = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const RT x = __shfl_down_sync(0xffffffffu, sfx.x, o);
            const RT y = __shfl_down_sync(0xffffffffu, sfx.y, o);
            if (lane + o < 32) {
                sfx.x += x;
                sfx.y += y;
            }
        }
        const T off = csub(sfx, acc);  // totals of the chunks above this one
        for (int i = i0; i < i1; ++i) {
            const int k = 2 * i + q;
            tmp[k] = cadd(tmp[k], off);
        }
    }
    __syncthreads();
    const RT fs = (RT)scale, f0 = (RT)(0.5 * scale);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const RT f = (j == 0) ? f0 : fs;
        d[j] = (j + 1 < n) ? cscale(tmp[j + 1], f) : Cx<T>::make(0.0, 0.0);
    }
    __syncthreads();
}

// Two independent derivatives at once, in place: c0 <- D c0 (warps 0-1, scratch
// t0) and c1 <- D c1 (warps 2-3, scratch t1), the same arithmetic as
// cheb_derivative_scan (whose second phase reads only the scratch, so the result
// may overwrite the input).  Whole CTA (>= 128 threads).
template <class T>
__device__ __forceinline__ void cheb_derivative_scan2(T* c0, T* t0, T* c1, T* t1, int n, double scale) {
    using RT = typename Cx<T>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const int q = warp & 1;
        const T* c = (warp < 2) ? c0 : c1;
        T* tmp = (warp < 2) ? t0 : t1;
        const int len = (n - q + 1) / 2;
        const int per = (len + 31) / 32;
        const int i0 = lane * per, i1 = min(i0 + per, len);
        T acc = Cx<T>::make(0.0, 0.0);
        for (int i = i1 - 1; i >= i0; --i) {
            const int k = 2 * i + q;
            if (k > 0) {
                const RT f = (RT)(2 * k);
                acc.x = fmat(f, c[k].x, acc.x);
                acc.y = fmat(f, c[k].y, acc.y);
            }
            tmp[k] = acc;
        }
        T sfx = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const RT x = __shfl_down_sync(0xffffffffu, sfx.x, o);
            const RT y = __shfl_down_sync(0xffffffffu, sfx.y, o);
            if (lane + o < 32) {
                sfx.x += x;
                sfx.y += y;
            }
        }
        const T off = csub(sfx, acc);
        for (int i = i0; i < i1; ++i) {
            const int k = 2 * i + q;
            tmp[k] = cadd(tmp[k], off);
        }
    }
    __syncthreads();
    const RT fs = (RT)scale, f0 = (RT)(0.5 * scale);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const RT f = (j == 0) ? f0 : fs;
        c0[j] = (j + 1 < n) ? cscale(t0[j + 1], f) : Cx<T>::make(0.0, 0.0);
        c1[j] = (j + 1 < n) ? cscale(t1[j + 1], f) : Cx<T>::make(0.0, 0.0);
    }
    __syncthreads();
}

// Transpose of cheb_derivative_scan: with d = D c, d_j = (2/c_j) sum_{k>j, k+j odd}
// k c_k (times scale), returns out = D^T e:
//   out_k = 2 k scale sum_{j<k, j+k odd} e_j / c_j   (c_0 = 2, c_j = 1),
// i.e. prefix sums of e_j/c_j over each index parity.  Warp q (q = 0, 1) owns the
// indices j = 2i + q; each lane sums a contiguous chunk, a shuffle scan adds the
// totals of the chunks below it.  ``tmp`` is scratch of n entries.  Whole CTA
// (>= 64 threads).
template <class T>
__device__ __forceinline__ void cheb_derivative_adjoint_scan(const T* e, T* out, T* tmp, int n, double scale) {
    using RT = typename Cx<T>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2) {
        const int q = warp;
        const int len = (n - q + 1) / 2;
        const int per = (len + 31) / 32;
        const int i0 = lane * per, i1 = min(i0 + per, len);
        T acc = Cx<T>::make(0.0, 0.0);
        for (int i = i0; i < i1; ++i) {
            const int j = 2 * i + q;
            const RT f = (j == 0) ? (RT)0.5 : (RT)1;
            acc.x = fmat(f, e[j].x, acc.x);
            acc.y = fmat(f, e[j].y, acc.y);
            tmp[j] = acc;  // inclusive prefix within the chunk
        }
        // exclusive scan of the chunk totals over the lanes
        T pfx = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const RT x = __shfl_up_sync(0xffffffffu, pfx.x, o);
            const RT y = __shfl_up_sync(0xffffffffu, pfx.y, o);
            if (lane >= o) {
                pfx.x += x;
                pfx.y += y;
            }
        }
        const T off = csub(pfx, acc);
        for (int i = i0; i < i1; ++i) {
            const int j = 2 * i + q;
            tmp[j] = cadd(tmp[j], off);
        }
    }
    __syncthreads();
    // out_k needs the inclusive prefix of the other parity up to k - 1
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        T v = Cx<T>::make(0.0, 0.0);
        if (k > 0) v = cscale(tmp[k - 1], (RT)(2.0 * k * scale));
        out[k] = v;
    }
    __syncthreads();
}

// Two independent transposed derivatives at once, in place: e0 <- post D^T e0
// (warps 0-1, scratch t0) and e1 <- post D^T e1 (warps 2-3, scratch t1), the same
// arithmetic as cheb_derivative_adjoint_scan followed by a multiplication by post.
// Whole CTA (>= 128 threads).
template <class T>
__device__ __forceinline__ void cheb_derivative_adjoint_scan2(T* e0, T* t0, T* e1, T* t1, int n, double scale,
                                                              double post) {
    using RT = typename Cx<T>::R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const int q = warp & 1;
        const T* e = (warp < 2) ? e0 : e1;
        T* tmp = (warp < 2) ? t0 : t1;
        const int len = (n - q + 1) / 2;
        const int per = (len + 31) / 32;
        const int i0 = lane * per, i1 = min(i0 + per, len);
        T acc = Cx<T>::make(0.0, 0.0);
        for (int i = i0; i < i1; ++i) {
            const int j = 2 * i + q;
            const RT f = (j == 0) ? (RT)0.5 : (RT)1;
            acc.x = fmat(f, e[j].x, acc.x);
            acc.y = fmat(f, e[j].y, acc.y);
            tmp[j] = acc;
        }
        T pfx = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const RT x = __shfl_up_sync(0xffffffffu, pfx.x, o);
            const RT y = __shfl_up_sync(0xffffffffu, pfx.y, o);
            if (lane >= o) {
                pfx.x += x;
                pfx.y += y;
            }
        }
        const T off = csub(pfx, acc);
        for (int i = i0; i < i1; ++i) {
            const int j = 2 * i + q;
            tmp[j] = cadd(tmp[j], off);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        T v0 = Cx<T>::make(0.0, 0.0), v1 = v0;
        if (k > 0) {
            v0 = cscale(t0[k - 1], (RT)(2.0 * k * scale));
            v1 = cscale(t1[k - 1], (RT)(2.0 * k * scale));
        }
        e0[k] = cscale(v0, (RT)post);
        e1[k] = cscale(v1, (RT)post);
    }
    __syncthreads();
}

}  // namespace pz
