// Implicit stage of one IMEX step: right-hand-side assembly (Eqs. multistep1
// and dirks of Section 4) and the bordered banded solve of Appendix A of
// Gastine, pizza, GJI 2019.
//
// For each mode the tau system  [tau rows; Mass - gamma dt Lin] y = [0; r]  is
//   (A B; C D)(y1; y2) = (g; h),   D banded (half width 8 for Psi, 4 for theta
//   and u_bar), factored at set-up without pivoting,
//   x = D^{-1} h,  y1 = S^{-1}(g - B x) with S = A - B D^{-1} C,  y2 = x - Y y1,
//   Y = D^{-1} C precomputed.
// The unpivoted factorisation of the streamfunction block loses digits as n_r
// grows, so its solution is refined once: the residual of the assembled system
// is formed in FP64 and solved again with the same factors.
//
// The banded block is solved through its two-sided block-tridiagonal
// factorisation (blocks of 8 rows; the temperature and zonal-flow bands, half
// width 4, are padded to that: twice the block size halves their chains and keeps
// all 32 lanes busy; host_ops.h, block_lu_twisted): a pair of warps walks the top and
// the bottom half towards the middle block and back, each step one lane-parallel
// H x H mat-vec forward and a fused pair of them backward.  On GB300 a dependent
// FP64 FMA costs ~64 cycles, so the sequential chain, not the flop count, sets
// the time of a solve; two half-length chains halve it.  Lane (r, c) =
// (lane/4, lane%4) owns row r of a block and columns c, c+4.  A CTA handles one
// mode: warps 0-1 the streamfunction, 2-3 the temperature, 4-5 the zonal flow
// (m = 0); the right-hand side, Schur updates, residual and the banded mass
// applies for later stages use the whole CTA.
#include "device_common.cuh"

namespace pz {

namespace {

constexpr int NTHREADS_S = 256;

template <class T>
__device__ __forceinline__ T zero();
template <>
__device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ double zero<double>() { return 0.0; }

// x - a*z in fused form
__device__ __forceinline__ double2 fms(double2 x, double2 a, double2 z) {
    return make_double2(fma(-a.x, z.x, fma(a.y, z.y, x.x)), fma(-a.x, z.y, fma(-a.y, z.x, x.y)));
}
__device__ __forceinline__ double2 fms(double2 x, double a, double2 z) {
    return make_double2(fma(-a, z.x, x.x), fma(-a, z.y, x.y));
}
__device__ __forceinline__ double2 mul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 mul(double a, double2 b) { return cscale(b, a); }

template <class TX>
__device__ __forceinline__ TX shfl_idx(TX v, int src);
template <>
__device__ __forceinline__ double shfl_idx<double>(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <>
__device__ __forceinline__ double2 shfl_idx<double2>(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
// sum over the four lanes of a row (lanes 4r .. 4r+3); every lane gets the sum
__device__ __forceinline__ double reduce4(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
}
__device__ __forceinline__ double2 reduce4(double2 v) { return make_double2(reduce4(v.x), reduce4(v.y)); }
// acc + a*b
__device__ __forceinline__ double2 fma_x(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 fma_x(double a, double2 b, double2 acc) {
    return make_double2(fma(a, b.x, acc.x), fma(a, b.y, acc.y));
}
__device__ __forceinline__ double fma_x(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ double2 sub_x(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ double sub_x(double a, double b) { return a - b; }

__device__ __forceinline__ double2 fms_x(double2 a, double2 b, double2 acc) {
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 fms_x(double a, double2 b, double2 acc) {
    return make_double2(fma(-a, b.x, acc.x), fma(-a, b.y, acc.y));
}
__device__ __forceinline__ double fms_x(double a, double b, double acc) { return fma(-a, b, acc); }

// FP32 counterparts for the refined FP32 temperature solves
template <>
__device__ __forceinline__ float2 zero<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ float zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 shfl_idx<float2>(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float reduce4(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
}
__device__ __forceinline__ float2 reduce4(float2 v) { return make_float2(reduce4(v.x), reduce4(v.y)); }
__device__ __forceinline__ float2 fma_x(float a, float2 b, float2 acc) {
    return make_float2(fmaf(a, b.x, acc.x), fmaf(a, b.y, acc.y));
}
__device__ __forceinline__ float2 sub_x(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// conversions between the FP32 chains and FP64 on the integer and FP32 pipes
// (GB300 issues float <-> double conversions on its FP64 unit)
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2(f32_from_bits(v.x), f32_from_bits(v.y)); }
__device__ __forceinline__ double2 to_d2_bits(float2 v) { return make_double2(f2d_bits(v.x), f2d_bits(v.y)); }

// Accumulator, conversions and finalisation of a chain value: for FP64 and FP32
// chains the accumulator is the value type itself and these are identities.
__device__ __forceinline__ double2 sub_acc(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ float2 sub_acc(float2 a, float2 b) { return sub_x(a, b); }
__device__ __forceinline__ double sub_acc(double a, double b) { return a - b; }
__device__ __forceinline__ double2 fin(double2 v) { return v; }
__device__ __forceinline__ float2 fin(float2 v) { return v; }
__device__ __forceinline__ double fin(double v) { return v; }
__device__ __forceinline__ double2 cvt_to(double2 v, const double2*) { return v; }
__device__ __forceinline__ float2 cvt_to(float2 v, const float2*) { return v; }
__device__ __forceinline__ double cvt_to(double v, const double*) { return v; }

// Double-float chains of the streamfunction solve.  The block chains of the
// Appendix A solve need about 44 significant bits: with the Schur step, the
// residual and the refinement in FP64, chains in 44- to 48-bit arithmetic leave
// the refined solution as close to the oracle's as FP64 chains do (measured on the
// tau systems at n_r = 257, 1025 and 2049), while FP32 chains need two and more
// corrections at n_r = 1025 and do not converge at 2049.  A double-float value
// (ddfloat.cuh) carries 48 bits on the FP32 pipe, which issues 64 times the FP64
// rate on GB300.
//
// Factors and chain values are complex double-floats (ddc, 16 bytes like a
// double2).  A row sum runs in an accumulator dacc of leading sums s and trailing
// sums e per component: every product a b of double-floats adds its leading part
// p = a.hi b.hi to s by a two-sum and its trailing parts (the two-product error
// fma(a.hi, b.hi, -p), a.hi b.lo + a.lo b.hi, and the two-sum's error) to e; the
// value is s + e, renormalised once at the end of the row (Ogita, Rump and
// Oishi's compensated dot product, applied to double-float inputs).
struct __align__(16) dacc {
    float xs, xe, ys, ye;
};
template <>
__device__ __forceinline__ dacc zero<dacc>() { return dacc{0.f, 0.f, 0.f, 0.f}; }
template <>
__device__ __forceinline__ ddc zero<ddc>() { return ddc{ddf{0.f, 0.f}, ddf{0.f, 0.f}}; }

// s + p = s' + t exactly (Knuth's two-sum)
__device__ __forceinline__ float two_sum(float s, float p, float& t) {
    const float r = __fadd_rn(s, p);
    const float bb = __fsub_rn(r, s);
    t = __fadd_rn(__fsub_rn(s, __fsub_rn(r, bb)), __fsub_rn(p, bb));
    return r;
}
// (s, e) += (ah + al)(bh + bl)
__device__ __forceinline__ void dd_acc(float& s, float& e, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    const float cr = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
    float t;
    s = two_sum(s, p, t);
    e = __fadd_rn(e, __fadd_rn(t, __fadd_rn(pe, cr)));
}
// acc + a b, complex
__device__ __forceinline__ dacc fma_x(ddc a, ddc b, dacc acc) {
    dd_acc(acc.xs, acc.xe, a.x.hi, a.x.lo, b.x.hi, b.x.lo);
    dd_acc(acc.xs, acc.xe, -a.y.hi, -a.y.lo, b.y.hi, b.y.lo);
    dd_acc(acc.ys, acc.ye, a.x.hi, a.x.lo, b.y.hi, b.y.lo);
    dd_acc(acc.ys, acc.ye, a.y.hi, a.y.lo, b.x.hi, b.x.lo);
    return acc;
}
// sum over the four lanes of a row; the two-sum's result and error do not depend
// on the order of its operands, so every lane gets the same bits
__device__ __forceinline__ void dd_pair_sum(float& s, float& e, int o) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
    float t;
    s = two_sum(s, s2, t);
    e = __fadd_rn(__fadd_rn(e, e2), t);
}
__device__ __forceinline__ dacc reduce4(dacc v) {
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        dd_pair_sum(v.xs, v.xe, o);
        dd_pair_sum(v.ys, v.ye, o);
    }
    return v;
}
// (s + e) as a normalised double-float: two-sum, since e may exceed a cancelled s
__device__ __forceinline__ ddf dd_norm(float s, float e) {
    float t;
    const float h = two_sum(s, e, t);
    return ddf{h, t};
}
__device__ __forceinline__ ddc fin(dacc v) { return ddc{dd_norm(v.xs, v.xe), dd_norm(v.ys, v.ye)}; }
// b - p
__device__ __forceinline__ ddf dd_sub1(ddf b, float s, float e) {
    float t;
    const float h = two_sum(b.hi, -s, t);
    return dd_norm(h, __fadd_rn(__fsub_rn(b.lo, e), t));
}
__device__ __forceinline__ ddc sub_x(ddc b, dacc p) { return ddc{dd_sub1(b.x, p.xs, p.xe), dd_sub1(b.y, p.ys, p.ye)}; }
__device__ __forceinline__ dacc sub_acc(dacc a, dacc b) {
    float t, u;
    const float xs = two_sum(a.xs, -b.xs, t);
    const float ys = two_sum(a.ys, -b.ys, u);
    return dacc{xs, __fadd_rn(__fsub_rn(a.xe, b.xe), t), ys, __fadd_rn(__fsub_rn(a.ye, b.ye), u)};
}
template <>
__device__ __forceinline__ ddc shfl_idx<ddc>(ddc v, int src) {
    return ddc{ddf{__shfl_sync(0xffffffffu, v.x.hi, src), __shfl_sync(0xffffffffu, v.x.lo, src)},
               ddf{__shfl_sync(0xffffffffu, v.y.hi, src), __shfl_sync(0xffffffffu, v.y.lo, src)}};
}
__device__ __forceinline__ ddc cvt_to(ddc v, const ddc*) { return v; }

// Asynchronous 16-byte copies global -> shared (cp.async), committed in groups;
// cp_async_wait<N> returns when at most N of the calling thread's groups are
// still in flight.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait1() { cp_async_wait<1>(); }

// Blocks of coefficients prefetched ahead in the chains.  With a few CTAs per SM
// (N_c up to ~600) two blocks cover the L2 latency at little register cost; the
// large systems run one CTA per SM (shared memory) with their factors streamed
// from HBM, where the chains wait on that latency unless loads go further ahead:
// there the streamfunction chains (FP64 complex coefficients) prefetch 4 blocks
// and the FP32 temperature chains 8.
constexpr int PFB = 2;
constexpr int PFB_DEEP_P = 4;
constexpr int PFB_DEEP_T = 8;

// Barrier of the two warps (64 threads) of a solver pair.
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Solve D x = b with the two-sided block factorisation (host_ops.h,
// block_lu_twisted) by a pair of warps: half 0 walks the top blocks down, half 1
// the bottom blocks up, both compute the middle block, then each substitutes
// back through its half.  Lane (r, c) = (lane/4, lane%4) owns row r of a block
// and columns c + 4q.  Z holds the forward values (nb*H entries), x the solution
// (n entries); rows of b at or beyond n read as zero.  Both warps of the pair
// must call it (bar: named barrier id); act = false skips all memory accesses.
// On return the whole of x is visible to both warps.
template <int H, int PF, class TF, class TX, class TA = TX, class TB = TX>
__device__ void pair_block_solve(const TB* b, TX* Z, TB* x, int n, const TF* __restrict__ blk, bool act, int half,
                                 int bar) {
    constexpr int CPL = H / 4;
    constexpr int HH = H * H;
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const bool ra = act && r < H;
    const int nb = (n + H - 1) / H;
    const int cm = nb / 2;
    const int dir = half ? -1 : 1;
    const int len = half ? (nb - 1 - cm) : cm;  // blocks of this half
    const int k_fw = half ? nb - 1 : 0;         // first block of the forward walk
    const int k_bw = half ? cm + 1 : cm - 1;    // first block of the backward walk
    auto coef = [&](int k, int which, int q) -> TF {
        return (ra && k >= 0 && k < nb) ? blk[(size_t)k * 3 * HH + which * HH + r * H + c + 4 * q] : zero<TF>();
    };
    // forward: Z_k = b_k - [0]_k Z_prev
    {
        TX prev[CPL];
        TF cur[PF][CPL], nxt[PF][CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) prev[q] = zero<TX>();
#pragma unroll
        for (int i = 0; i < PF; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) cur[i][q] = (i < len) ? coef(k_fw + dir * i, 0, q) : zero<TF>();
        for (int i0 = 0; i0 < len; i0 += PF) {
#pragma unroll
            for (int i = 0; i < PF; ++i)
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    nxt[i][q] = (i0 + PF + i < len) ? coef(k_fw + dir * (i0 + PF + i), 0, q) : zero<TF>();
#pragma unroll
            for (int i = 0; i < PF; ++i) {
                if (i0 + i < len) {
                    const int k = k_fw + dir * (i0 + i);
                    const int row = k * H + r;
                    const TX bv = (ra && row < n) ? cvt_to(b[row], (const TX*)nullptr) : zero<TX>();
                    TA p = zero<TA>();
#pragma unroll
                    for (int q = 0; q < CPL; ++q) p = fma_x(cur[i][q], prev[q], p);
                    p = reduce4(p);
                    const TX zv = sub_x(bv, p);
                    if (ra && c == 0) Z[row] = zv;
#pragma unroll
                    for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(zv, 4 * (c + 4 * q));
                }
            }
#pragma unroll
            for (int i = 0; i < PF; ++i)
#pragma unroll
                for (int q = 0; q < CPL; ++q) cur[i][q] = nxt[i][q];
        }
    }
    pair_sync(bar);
    // middle block, by both warps: x_c = S^{-1}(b_c - L_c z_{c-1} - M_c w_{c+1})
    TX prev[CPL];
    {
        TA t = zero<TA>();
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int col = c + 4 * q;
            if (ra && cm > 0) t = fma_x(coef(cm, 0, q), Z[(cm - 1) * H + col], t);
            if (ra && cm < nb - 1) t = fma_x(coef(cm, 2, q), Z[(cm + 1) * H + col], t);
        }
        t = reduce4(t);
        const int row = cm * H + r;
        const TX bv = (ra && row < n) ? cvt_to(b[row], (const TX*)nullptr) : zero<TX>();
        const TX rv = sub_x(bv, t);
        TX rr[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) rr[q] = shfl_idx(rv, 4 * (c + 4 * q));
        TA xa = zero<TA>();
#pragma unroll
        for (int q = 0; q < CPL; ++q) xa = fma_x(coef(cm, 1, q), rr[q], xa);
        const TX xv = fin(reduce4(xa));
        if (half == 0 && ra && c == 0 && row < n) x[row] = cvt_to(xv, (const TB*)nullptr);
#pragma unroll
        for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(xv, 4 * (c + 4 * q));
    }
    // backward: x_k = [1]_k Z_k - [2]_k x_prev, walking away from the middle
    {
        TF cu[PF][CPL], ch[PF][CPL], nu[PF][CPL], nh[PF][CPL];
        const int bdir = half ? 1 : -1;
#pragma unroll
        for (int i = 0; i < PF; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                cu[i][q] = (i < len) ? coef(k_bw + bdir * i, 1, q) : zero<TF>();
                ch[i][q] = (i < len) ? coef(k_bw + bdir * i, 2, q) : zero<TF>();
            }
        for (int i0 = 0; i0 < len; i0 += PF) {
#pragma unroll
            for (int i = 0; i < PF; ++i)
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const bool in = i0 + PF + i < len;
                    nu[i][q] = in ? coef(k_bw + bdir * (i0 + PF + i), 1, q) : zero<TF>();
                    nh[i][q] = in ? coef(k_bw + bdir * (i0 + PF + i), 2, q) : zero<TF>();
                }
#pragma unroll
            for (int i = 0; i < PF; ++i) {
                if (i0 + i < len) {
                    const int k = k_bw + bdir * (i0 + i);
                    TA pz = zero<TA>(), ph = zero<TA>();
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const TX zq = ra ? Z[k * H + c + 4 * q] : zero<TX>();
                        pz = fma_x(cu[i][q], zq, pz);
                        ph = fma_x(ch[i][q], prev[q], ph);
                    }
                    const TX p = fin(reduce4(sub_acc(pz, ph)));
                    const int row = k * H + r;
                    if (ra && c == 0 && row < n) x[row] = cvt_to(p, (const TB*)nullptr);
#pragma unroll
                    for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(p, 4 * (c + 4 * q));
                }
            }
#pragma unroll
            for (int i = 0; i < PF; ++i)
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    cu[i][q] = nu[i][q];
                    ch[i][q] = nh[i][q];
                }
        }
    }
    // both halves of x written before either warp goes on (a Schur step of the
    // caller reads all of it)
    pair_sync(bar);
}

// The same two-sided solve split into phases for a CTA whose other warps can
// help (the kernel with one CTA per system).  The pair's walks each read one
// matrix per block -- [0] forward, [2] backward -- so the same registers prefetch
// PF blocks ahead with PF twice as large; the products W_k = [1]_k Z_k, which no
// chain depends on, are formed between the walks by every warp of the CTA:
//   chain_forward (pair)  -> barrier -> chain_middle (pair) -> barrier ->
//   chain_diag (CTA, Z_k := W_k in place for k != c) -> barrier ->
//   chain_backward (pair), x_k = W_k - [2]_k x_prev.
// Geometry as in pair_block_solve: blocks of H rows, middle block c = nb/2,
// half 0 walks 0..c-1, half 1 nb-1..c+1.  b, Z and x hold the chain type (no
// conversions on the dependent path).
template <int H>
struct ChainGeom {
    int nb, cm, dir, len, k_fw, k_bw;
    __device__ ChainGeom(int n, int half) {
        nb = (n + H - 1) / H;
        cm = nb / 2;
        dir = half ? -1 : 1;
        len = half ? (nb - 1 - cm) : cm;
        k_fw = half ? nb - 1 : 0;
        k_bw = half ? cm + 1 : cm - 1;
    }
};

// Coefficients of a walk come through a ring of D matrices in shared memory
// (ring: D * H * H entries per warp), filled by asynchronous copies D blocks
// ahead: a copy in flight holds no register and no scoreboard, so the walk keeps
// D loads outstanding whatever its own latency.  Step i waits for its block's
// group, reads the lane's coefficients, and refills the slot with block i + D
// once every lane has read it.
template <int H, int D, class TF>
__device__ __forceinline__ void ring_issue(const TF* __restrict__ blk, TF* ring, int k, int which, int slot,
                                           bool valid) {
    constexpr int HH = H * H;
    constexpr int CH = HH * (int)sizeof(TF) / 16;  // 16-byte chunks of one matrix
    const int lane = threadIdx.x & 31;
    if (valid) {
        const char* src = reinterpret_cast<const char*>(blk + (size_t)k * 3 * HH + which * HH);
        char* dst = reinterpret_cast<char*>(ring + slot * HH);
        for (int j = lane; j < CH; j += 32) cp_async16(dst + 16 * j, src + 16 * j);
    }
    cp_async_commit();
}

template <int H, int D, class TF, class TX, class TA>
__device__ void chain_forward(const TX* b, TX* Z, int n, const TF* __restrict__ blk, int half, TF* ring) {
    constexpr int CPL = H / 4;
    constexpr int HH = H * H;
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const ChainGeom<H> g(n, half);
#pragma unroll
    for (int i = 0; i < D; ++i) ring_issue<H, D>(blk, ring, g.k_fw + g.dir * i, 0, i, i < g.len);
    TX prev[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) prev[q] = zero<TX>();
    for (int i = 0; i < g.len; ++i) {
        const int k = g.k_fw + g.dir * i;
        const int row = k * H + r;
        const TX bv = (row < n) ? b[row] : zero<TX>();
        cp_async_wait<D - 1>();
        __syncwarp();
        const TF* mat = ring + (i % D) * HH;
        TA p = zero<TA>();
#pragma unroll
        for (int q = 0; q < CPL; ++q) p = fma_x(mat[r * H + c + 4 * q], prev[q], p);
        __syncwarp();  // every lane has read the slot
        ring_issue<H, D>(blk, ring, g.k_fw + g.dir * (i + D), 0, i % D, i + D < g.len);
        p = reduce4(p);
        const TX zv = sub_x(bv, p);
        if (c == 0) Z[row] = zv;
#pragma unroll
        for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(zv, 4 * (c + 4 * q));
    }
    cp_async_wait<0>();
}

// middle block by both warps of the pair: x_c = S^{-1}(b_c - L_c z_{c-1} - M_c w_{c+1});
// both keep it in prev (the start of their backward walks) and return the lane's
// row of it; the caller stores it after a barrier, since x may share its rows
// with b (the correction solved in place of the residual) and the other warp of
// the pair reads b_c here
template <int H, class TF, class TX, class TA>
__device__ TX chain_middle(const TX* b, const TX* Z, int n, const TF* __restrict__ blk, int half,
                           TX (&prev)[H / 4]) {
    constexpr int CPL = H / 4;
    constexpr int HH = H * H;
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const ChainGeom<H> g(n, half);
    const int cm = g.cm, nb = g.nb;
    auto coef = [&](int which, int q) -> TF { return blk[(size_t)cm * 3 * HH + which * HH + r * H + c + 4 * q]; };
    TA t = zero<TA>();
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int col = c + 4 * q;
        if (cm > 0) t = fma_x(coef(0, q), Z[(cm - 1) * H + col], t);
        if (cm < nb - 1) t = fma_x(coef(2, q), Z[(cm + 1) * H + col], t);
    }
    t = reduce4(t);
    const int row = cm * H + r;
    const TX bv = (row < n) ? b[row] : zero<TX>();
    const TX rv = sub_x(bv, t);
    TX rr[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) rr[q] = shfl_idx(rv, 4 * (c + 4 * q));
    TA xa = zero<TA>();
#pragma unroll
    for (int q = 0; q < CPL; ++q) xa = fma_x(coef(1, q), rr[q], xa);
    const TX xv = fin(reduce4(xa));
#pragma unroll
    for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(xv, 4 * (c + 4 * q));
    return xv;
}

// the middle block's rows of x, by half 0 of the pair (after the barrier that
// ends the middle phase)
template <int H, class TX>
__device__ __forceinline__ void chain_middle_store(TX* x, int n, int half, TX xv) {
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const int row = ((n + H - 1) / H / 2) * H + r;
    if (half == 0 && c == 0 && row < n) x[row] = xv;
}

// Z_k := [1]_k Z_k for every block k except the middle one, one warp per block
// (warp w of nw), DU blocks in flight per warp: their coefficient and Z loads are
// issued together before any product, so the pass costs a few load latencies
// rather than one per block.  Rows at or beyond n stay untouched.
constexpr int DU = 4;
template <int H, class TF, class TX, class TA>
__device__ void chain_diag(TX* Z, int n, const TF* __restrict__ blk, int w, int nw) {
    constexpr int CPL = H / 4;
    constexpr int HH = H * H;
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const int nb = (n + H - 1) / H, cm = nb / 2;
    for (int k0 = w; k0 < nb; k0 += nw * DU) {
        TF a[DU][CPL];
        TX z[DU][CPL];
#pragma unroll
        for (int u = 0; u < DU; ++u) {
            const int k = k0 + u * nw;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int col = k * H + c + 4 * q;
                const bool ok = k < nb && k != cm;
                a[u][q] = ok ? blk[(size_t)k * 3 * HH + HH + r * H + c + 4 * q] : zero<TF>();
                z[u][q] = (ok && col < n) ? Z[col] : zero<TX>();
            }
        }
        TX wv[DU];
#pragma unroll
        for (int u = 0; u < DU; ++u) {
            TA t = zero<TA>();
#pragma unroll
            for (int q = 0; q < CPL; ++q) t = fma_x(a[u][q], z[u][q], t);
            wv[u] = fin(reduce4(t));
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < DU; ++u) {
            const int k = k0 + u * nw;
            const int row = k * H + r;
            if (k < nb && k != cm && c == 0 && row < n) Z[row] = wv[u];
        }
        __syncwarp();
    }
}

// backward walk away from the middle block: x_k = W_k - [2]_k x_prev
template <int H, int D, class TF, class TX, class TA>
__device__ void chain_backward(const TX* W, TX* x, int n, const TF* __restrict__ blk, int half, TX (&prev)[H / 4],
                               TF* ring) {
    constexpr int CPL = H / 4;
    constexpr int HH = H * H;
    const int lane = threadIdx.x & 31;
    const int r = lane >> 2, c = lane & 3;
    const ChainGeom<H> g(n, half);
    const int bdir = half ? 1 : -1;
#pragma unroll
    for (int i = 0; i < D; ++i) ring_issue<H, D>(blk, ring, g.k_bw + bdir * i, 2, i, i < g.len);
    for (int i = 0; i < g.len; ++i) {
        const int k = g.k_bw + bdir * i;
        const int row = k * H + r;
        const TX wv = (row < n) ? W[row] : zero<TX>();
        cp_async_wait<D - 1>();
        __syncwarp();
        const TF* mat = ring + (i % D) * HH;
        TA ph = zero<TA>();
#pragma unroll
        for (int q = 0; q < CPL; ++q) ph = fma_x(mat[r * H + c + 4 * q], prev[q], ph);
        __syncwarp();
        ring_issue<H, D>(blk, ring, g.k_bw + bdir * (i + D), 2, i % D, i + D < g.len);
        ph = reduce4(ph);
        const TX p = sub_x(wv, ph);
        if (c == 0 && row < n) x[row] = p;
#pragma unroll
        for (int q = 0; q < CPL; ++q) prev[q] = shfl_idx(p, 4 * (c + 4 * q));
    }
    cp_async_wait<0>();
}

// Whole-CTA driver of the phased solve for up to two systems: system 1 by the
// warp pair (w1, w1 + 1), system 2 (n2 > 0) by (w2, w2 + 1).  ring: shared memory
// for 4 x D matrices (one ring per walking warp: system 1's pair first).  Every
// thread of the CTA calls it; it ends with a __syncthreads that publishes x, x2.
template <int D, class TF, class TX, class TA>
__device__ void cta_chain_solve(const TX* b, TX* Z, TX* x, int n, const TF* __restrict__ blk, int w1, const TX* b2,
                                TX* Z2, TX* x2, int n2, const TF* __restrict__ blk2, int w2, TF* ring) {
    constexpr int HH = 64;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool in1 = warp == w1 || warp == w1 + 1, in2 = n2 > 0 && (warp == w2 || warp == w2 + 1);
    TF* my_ring = ring + (in1 ? warp - w1 : 2 + warp - w2) * D * HH;
    if (in1) chain_forward<8, D, TF, TX, TA>(b, Z, n, blk, warp - w1, my_ring);
    if (in2) chain_forward<8, D, TF, TX, TA>(b2, Z2, n2, blk2, warp - w2, my_ring);
    __syncthreads();
    TX prev[2];
    TX xm = zero<TX>();
    if (in1) xm = chain_middle<8, TF, TX, TA>(b, Z, n, blk, warp - w1, prev);
    if (in2) xm = chain_middle<8, TF, TX, TA>(b2, Z2, n2, blk2, warp - w2, prev);
    __syncthreads();
    if (in1) chain_middle_store<8>(x, n, warp - w1, xm);
    if (in2) chain_middle_store<8>(x2, n2, warp - w2, xm);
    chain_diag<8, TF, TX, TA>(Z, n, blk, warp, nw);
    if (n2 > 0) chain_diag<8, TF, TX, TA>(Z2, n2, blk2, warp, nw);
    __syncthreads();
    if (in1) chain_backward<8, D, TF, TX, TA>(Z, x, n, blk, warp - w1, prev, my_ring);
    if (in2) chain_backward<8, D, TF, TX, TA>(Z2, x2, n2, blk2, warp - w2, prev, my_ring);
    __syncthreads();
}

// Ring depths of the phased chains: double-float streamfunction chains 6
// matrices (1 KB each) per walking warp, FP32 temperature chains 8 (256 bytes)
constexpr int RD_DD = 6;
constexpr int RD_32 = 8;

// Join of the streamfunction block solved in two halves (rows [0, nA) by warps
// 0-1, [nA, n) by warps 6-7; DevFactors psplit): x holds each half's own solution
// g.  The interface unknowns, A's last block and B's first, are
// [x_A,last; x_B,first] = Rj [g_A,last; g_B,first], Rj the inverse of
// [[I, V_last], [W_first, I]]; then x_A = g_A - V x_B,first and
// x_B = g_B - W x_A,last with the spikes V = D_A^{-1} E, W = D_B^{-1} F (spk rows
// < nA: V, the rest: W).  Whole CTA, after a __syncthreads that published x;
// ends with one.  act = false: no memory accesses.
__device__ void split_join(double2* x, int n, int nA, const double2* __restrict__ spk, const double2* __restrict__ rj,
                           bool act) {
    __shared__ double2 xi[16];
    const int tid = threadIdx.x;
    if (act && tid < 16) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll 4
        for (int c = 0; c < 16; ++c) acc = cfma(__ldg(&rj[tid * 16 + c]), x[c < 8 ? nA - 8 + c : nA + c - 8], acc);
        xi[tid] = acc;
    }
    __syncthreads();
    if (act)
        for (int i = tid; i < n; i += blockDim.x) {
            const double2* row = spk + (size_t)i * 8;
            const double2* v = (i < nA) ? xi + 8 : xi;
            double2 t = x[i];
#pragma unroll
            for (int c = 0; c < 8; ++c) t = fms(t, __ldg(&row[c]), v[c]);
            x[i] = t;
        }
    __syncthreads();
}

// The same join in double-float arithmetic on the FP32 pipe (double-float
// chains): x, the spikes and the interface inverse as complex double-floats.  The
// 16 interface values are summed by 64 threads (four partial sums each, joined
// by shuffles); the rows go two per thread and pass, loads first.
__device__ void split_join_dd(ddc* x, int n, int nA, const ddc* __restrict__ spk, const ddc* __restrict__ rj,
                              bool act) {
    __shared__ ddc xi[16];
    const int tid = threadIdx.x;
    if (act && tid < 64) {
        const int o = tid >> 2, part = tid & 3;  // output o, columns part*4 .. part*4+3
        dacc acc = zero<dacc>();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = part * 4 + j;
            acc = fma_x(rj[o * 16 + c], x[c < 8 ? nA - 8 + c : nA + c - 8], acc);
        }
        acc = reduce4(acc);
        if (part == 0) xi[o] = fin(acc);
    }
    __syncthreads();
    if (act)
        for (int i0 = tid; i0 < n; i0 += 2 * blockDim.x) {
            const int i1 = i0 + blockDim.x;
            ddc s0[8], s1[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                s0[c] = spk[(size_t)i0 * 8 + c];
                s1[c] = (i1 < n) ? spk[(size_t)i1 * 8 + c] : zero<ddc>();
            }
            const ddc* v0 = (i0 < nA) ? xi + 8 : xi;
            const ddc* v1 = (i1 < nA) ? xi + 8 : xi;
            dacc a0 = zero<dacc>(), a1 = zero<dacc>();
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                a0 = fma_x(s0[c], v0[c], a0);
                a1 = fma_x(s1[c], v1[c], a1);
            }
            x[i0] = sub_x(x[i0], a0);
            if (i1 < n) x[i1] = sub_x(x[i1], a1);
        }
    __syncthreads();
}

// The same join for the FP32 temperature block split in halves (real spikes
// and interface inverse, complex FP32 values).
__device__ void split_join32(float2* x, int n, int nA, const float* __restrict__ spk, const float* __restrict__ rj) {
    __shared__ float2 xi[16];
    const int tid = threadIdx.x;
    if (tid < 16) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
            const float r = __ldg(&rj[tid * 16 + c]);
            const float2 v = x[c < 8 ? nA - 8 + c : nA + c - 8];
            acc.x = fmaf(r, v.x, acc.x);
            acc.y = fmaf(r, v.y, acc.y);
        }
        xi[tid] = acc;
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        const float* row = spk + (size_t)i * 8;
        const float2* v = (i < nA) ? xi + 8 : xi;
        float2 t = x[i];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float r = __ldg(&row[c]);
            t.x = fmaf(-r, v[c].x, t.x);
            t.y = fmaf(-r, v[c].y, t.y);
        }
        x[i] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Schur step of Appendix A by one warp: sol[PB..] = D^{-1} h on entry;
// sol[0..PB) = S^{-1}(g - B sol[PB..]) on exit.  B: PB x (nc-PB) real tau rows.
template <int PB, class TF>
__device__ void warp_schur(double2* sol, const double2* g, int nc, const double* __restrict__ B,
                           const TF* __restrict__ Sinv) {
    const int lane = threadIdx.x & 31;
    const int n = nc - PB;
    double2 t[PB];
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = make_double2(0.0, 0.0);
    for (int j = lane; j < n; j += 32) {
        const double2 xv = sol[PB + j];
#pragma unroll
        for (int r = 0; r < PB; ++r) {
            const double b = __ldg(&B[(size_t)r * n + j]);
            t[r].x = fma(b, xv.x, t[r].x);
            t[r].y = fma(b, xv.y, t[r].y);
        }
    }
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = csub(g ? g[r] : make_double2(0.0, 0.0), warp_sum(t[r]));
    if (lane < PB) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < PB; ++c) acc = cadd(acc, mul(Sinv[lane * PB + c], t[c]));
        sol[lane] = acc;
    }
    __syncwarp();
}

// y2 -= Y y1 over the rows of one system, threads [t0, t0 + nt)
template <int PB, class TF>
__device__ void schur_update(double2* sol, int nc, const TF* __restrict__ Y, int t0, int nt) {
    const int n = nc - PB;
    double2 y1[PB];
#pragma unroll
    for (int c = 0; c < PB; ++c) y1[c] = sol[c];
    for (int j = threadIdx.x - t0; j < n; j += nt) {
        double2 acc = sol[PB + j];
#pragma unroll
        for (int c = 0; c < PB; ++c) acc = fms(acc, Y[(size_t)j * PB + c], y1[c]);
        sol[PB + j] = acc;
    }
}

// Row-block dot products by the whole CTA: t_r = sum_{j < nj} R[r nj + j] x[j]
// for the PB rows r of a real row block R (tau rows restricted to some columns)
// against a complex vector, FP64 or FP32.  Each thread takes a stride of j (a few
// loads in flight per thread instead of one warp walking all of them), a
// butterfly per warp, then the warp partials summed in warp order.  Lane r < PB
// of warp 0 gets t_r (every other thread zero).  Contains one __syncthreads; the
// caller's next barrier must come before any thread calls it again.
__device__ __forceinline__ void acc_rx(double2& t, double b, double2 x) {
    t.x = fma(b, x.x, t.x);
    t.y = fma(b, x.y, t.y);
}
__device__ __forceinline__ void acc_rx(float2& t, float b, float2 x) {
    t.x = fmaf(b, x.x, t.x);
    t.y = fmaf(b, x.y, t.y);
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ float2 add_x(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add_x(double2 a, double2 b) { return cadd(a, b); }

template <int PB, class TX, class TR>
__device__ TX block_rows_dot(const TX* x, int nj, const TR* __restrict__ R) {
    __shared__ TX part[NTHREADS_S / 32][PB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    TX t[PB];
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = zero<TX>();
    for (int j = tid; j < nj; j += blockDim.x) {
        const TX xv = x[j];
#pragma unroll
        for (int r = 0; r < PB; ++r) acc_rx(t[r], __ldg(&R[(size_t)r * nj + j]), xv);
    }
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = warp_sum(t[r]);
    if (lane == 0)
#pragma unroll
        for (int r = 0; r < PB; ++r) part[warp][r] = t[r];
    __syncthreads();
    TX v = zero<TX>();
    if (warp == 0 && lane < PB)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = add_x(v, part[w][lane]);
    return v;
}

// Schur step of Appendix A by the whole CTA: sol[PB..] = D^{-1} h on entry;
// sol[0..PB) = S^{-1}(g - B sol[PB..]) on exit (g = 0 when null), visible to
// every thread.  B: PB x (nc-PB) real tau rows; S^{-1} complex or real.
template <int PB, class TS>
__device__ void block_schur(double2* sol, const double2* g, int nc, const double* __restrict__ B,
                            const TS* __restrict__ Sinv) {
    const double2 t = block_rows_dot<PB>(sol + PB, nc - PB, B);
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        const double2 gv = (lane < PB) ? csub(g ? g[lane] : make_double2(0.0, 0.0), t) : make_double2(0.0, 0.0);
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < PB; ++c) {
            const double2 gc = shfl_idx(gv, c);
            if (lane < PB) acc = cadd(acc, mul(Sinv[lane * PB + c], gc));
        }
        if (lane < PB) sol[lane] = acc;
    }
    __syncthreads();
}

// FP32 Schur step of the temperature system by the whole CTA: sol[2..] = D^{-1} r
// on entry, sol[0..2) = S^{-1}(g - B sol[2..]) on exit, g = the residual's tau
// rows; B: 2 x (nc-2) tau rows in FP32, Sinv real 2 x 2.  Ends with __syncthreads.
__device__ void block_schur32_dir(float2* sol, const float2* g, int nc, const float* __restrict__ B,
                                  const float* __restrict__ Sinv) {
    const float2 t = block_rows_dot<2>(sol + 2, nc - 2, B);
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        const float2 gv = (lane < 2) ? make_float2(g[lane].x - t.x, g[lane].y - t.y) : make_float2(0.f, 0.f);
        const float2 g0 = shfl_idx(gv, 0), g1 = shfl_idx(gv, 1);
        if (lane < 2) {
            const float a = Sinv[lane * 2], b = Sinv[lane * 2 + 1];
            sol[lane] = make_float2(fmaf(a, g0.x, b * g1.x), fmaf(a, g0.y, b * g1.y));
        }
    }
    __syncthreads();
}

// FP32 Schur step of the temperature system by one warp: sol[2..] = D^{-1} r on
// entry, sol[0..2) = S^{-1}(g - B sol[2..]) on exit, g = the residual's tau rows;
// B: 2 x (nc-2) tau rows in FP32, Sinv real 2 x 2.
__device__ void warp_schur32_dir(float2* sol, const float2* g, int nc, const float* __restrict__ B,
                                 const float* __restrict__ Sinv) {
    const int lane = threadIdx.x & 31;
    const int n = nc - 2;
    float2 t[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int j = lane; j < n; j += 32) {
        const float2 xv = sol[2 + j];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float b = __ldg(&B[(size_t)r * n + j]);
            t[r].x = fmaf(b, xv.x, t[r].x);
            t[r].y = fmaf(b, xv.y, t[r].y);
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t[r].x += __shfl_xor_sync(0xffffffffu, t[r].x, o);
            t[r].y += __shfl_xor_sync(0xffffffffu, t[r].y, o);
        }
        t[r] = make_float2(g[r].x - t[r].x, g[r].y - t[r].y);
    }
    __syncwarp();
    if (lane < 2) {
        const float a = Sinv[lane * 2], b = Sinv[lane * 2 + 1];
        sol[lane] = make_float2(fmaf(a, t[0].x, b * t[1].x), fmaf(a, t[0].y, b * t[1].y));
    }
    __syncwarp();
}

// FP32 y2 -= Y y1 for the temperature system, threads [t0, t0 + nt)
__device__ void schur_update32_dir(float2* sol, int nc, const float* __restrict__ Y, int t0, int nt) {
    const int n = nc - 2;
    const float2 y0 = sol[0], y1 = sol[1];
    for (int j = threadIdx.x - t0; j < n; j += nt) {
        const float a = Y[(size_t)j * 2], b = Y[(size_t)j * 2 + 1];
        float2 acc = sol[2 + j];
        acc.x -= fmaf(a, y0.x, b * y1.x);
        acc.y -= fmaf(a, y0.y, b * y1.y);
        sol[2 + j] = acc;
    }
}

template <int H>
__device__ __forceinline__ double2 band_row_c(const double* __restrict__ band, const double2* x, int k, int nc) {
    const double* row = band + (size_t)k * (2 * H + 1);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int d = 0; d <= 2 * H; ++d) {
        const int n = k - H + d;
        if (n >= 0 && n < nc) {
            const double c = __ldg(&row[d]);
            acc.x = fma(c, x[n].x, acc.x);
            acc.y = fma(c, x[n].y, acc.y);
        }
    }
    return acc;
}

// mass / implicit operators applied to one mode's new state
__device__ void apply_row(const StepParams& P, int m, int k, const double2* xp, const double2* xt, const double* xu,
                          VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp) {
    const int nc = P.nc;
    const double mu = (double)m * m;
    const double dm = (double)m;
    double2 mp = make_double2(0.0, 0.0), ip = make_double2(0.0, 0.0);
    double2 mt = make_double2(0.0, 0.0), it = make_double2(0.0, 0.0);
    if (m > 0 && k >= 4) {
        if (want_mass) {
            const double2 a0 = band_row_c<8>(P.ops.band[OP_A0], xp, k, nc);
            const double2 a2 = band_row_c<8>(P.ops.band[OP_A2], xp, k, nc);
            mp = make_double2(fma(mu, a2.x, a0.x), fma(mu, a2.y, a0.y));
        }
        if (want_imp) {
            const double2 b0 = band_row_c<6>(P.ops.band[OP_B0], xp, k, nc);
            const double2 b2 = band_row_c<6>(P.ops.band[OP_B2], xp, k, nc);
            const double2 b4 = band_row_c<6>(P.ops.band[OP_B4], xp, k, nc);
            const double2 c = band_row_c<8>(P.ops.band[OP_C], xp, k, nc);
            const double ce = 2.0 * dm / P.E;
            ip.x = b0.x + mu * (b2.x + mu * b4.x) - ce * c.y;
            ip.y = b0.y + mu * (b2.y + mu * b4.y) + ce * c.x;
            if (P.buoy_imp)  // (Ra/Pr)(i m/s_o) C^I theta
                ip = cadd(ip, cmul_i(band_row_c<8>(P.ops.band[OP_C], xt, k, nc), P.Ra / P.Pr * dm / P.s_o));
        }
    }
    if (k >= 2) {
        if (want_mass) mt = band_row_c<4>(P.ops.band[OP_D], xt, k, nc);
        if (want_imp) {
            const double2 f0 = band_row_c<2>(P.ops.band[OP_F0], xt, k, nc);
            const double2 f2 = band_row_c<2>(P.ops.band[OP_F2], xt, k, nc);
            const double ip_ = 1.0 / P.Pr;
            it = make_double2((f0.x + mu * f2.x) * ip_, (f0.y + mu * f2.y) * ip_);
        }
    }
    if (want_mass) {
        mass_out.psi[(size_t)m * nc + k] = mp;
        mass_out.th[(size_t)m * nc + k] = mt;
    }
    if (want_imp) {
        imp_out.psi[(size_t)m * nc + k] = ip;
        imp_out.th[(size_t)m * nc + k] = it;
    }
    if (m == 0) {
        double mu_ = 0.0, iu = 0.0;
        if (k >= 2) {
            const double* rd = P.ops.band[OP_D] + (size_t)k * 9;
            const double* re = P.ops.band[OP_EZ] + (size_t)k * 5;
            for (int d = 0; d < 9; ++d) {
                const int n = k - 4 + d;
                if (n >= 0 && n < nc) mu_ = fma(__ldg(&rd[d]), xu[n], mu_);
            }
            for (int d = 0; d < 5; ++d) {
                const int n = k - 2 + d;
                if (n >= 0 && n < nc) iu = fma(__ldg(&re[d]), xu[n], iu);
            }
        }
        if (want_mass) mass_out.u[k] = mu_;
        if (want_imp) imp_out.u[k] = iu;
    }
}

// Epilogue of a solve for row k of mode m: the mass term of the new state
// (A^I_m Psi, D^I theta, D^I u) and, from the solved equation
// (Mass - gamma dt Lin) y = f on the rows below the tau rows, its implicit term
// Lin y = (Mass y - f)/(gamma dt), which saves the banded B^I, C^I, F^I, E^I
// applies.  f is the right-hand side of the solve (recomputed here from the
// same terms in the same order).
__device__ void epilogue_row(const StepParams& P, const RhsSpec& R, double gdt, int m, int k, const double2* xp,
                             const double2* xt, const double* xu, VecSet mass_out, VecSet imp_out, bool want_mass,
                             bool want_imp, const double2* fps = nullptr, const double2* fts = nullptr,
                             const double* fus = nullptr) {
    const int nc = P.nc;
    const double mu = (double)m * m;
    double2 mp = make_double2(0.0, 0.0), mt = make_double2(0.0, 0.0);
    double muu = 0.0;
    if (m > 0 && k >= 4) {
        const double2 a0 = band_row_c<8>(P.ops.band[OP_A0], xp, k, nc);
        const double2 a2 = band_row_c<8>(P.ops.band[OP_A2], xp, k, nc);
        mp = make_double2(fma(mu, a2.x, a0.x), fma(mu, a2.y, a0.y));
    }
    if (k >= 2) {
        mt = band_row_c<4>(P.ops.band[OP_D], xt, k, nc);
        if (m == 0) {
            const double* rd = P.ops.band[OP_D] + (size_t)k * 9;
            for (int d = 0; d < 9; ++d) {
                const int n = k - 4 + d;
                if (n >= 0 && n < nc) muu = fma(__ldg(&rd[d]), xu[n], muu);
            }
        }
    }
    const size_t idx = (size_t)m * nc + k;
    if (want_imp) {  // before any store: an output may be one of the terms of f
        double2 fp = make_double2(0.0, 0.0), ft = make_double2(0.0, 0.0);
        double fu = 0.0;
        if (fps) {  // kept by the caller (the same sums)
            fp = fps[k];
            ft = fts[k];
            if (m == 0) fu = fus[k];
        }
        for (int t = 0; t < (fps ? 0 : R.nterms); ++t) {
            const double c = R.t[t].c;
            const double2 vp = R.t[t].v.psi[idx];
            const double2 vt = R.t[t].v.th[idx];
            fp.x = fma(c, vp.x, fp.x);
            fp.y = fma(c, vp.y, fp.y);
            ft.x = fma(c, vt.x, ft.x);
            ft.y = fma(c, vt.y, ft.y);
            if (m == 0) fu = fma(c, R.t[t].v.u[k], fu);
        }
        const double ig = 1.0 / gdt;
        imp_out.psi[idx] = (m > 0 && k >= 4) ? cscale(csub(mp, fp), ig) : make_double2(0.0, 0.0);
        imp_out.th[idx] = (k >= 2) ? cscale(csub(mt, ft), ig) : make_double2(0.0, 0.0);
        if (m == 0) imp_out.u[k] = (k >= 2) ? (muu - fu) * ig : 0.0;
    }
    if (want_mass) {
        mass_out.psi[idx] = mp;
        mass_out.th[idx] = mt;
        if (m == 0) mass_out.u[k] = muu;
    }
}

// shared-memory layout of one CTA, per mode mi < MB:
//   streamfunction: pf rhs (then the refinement residual), pw forward-chain
//                   values, px solution, pd correction
//   temperature:    tf rhs, tw forward-chain values, tx solution
// and for the zonal flow (the CTA holding m = 0): uf rhs, ux solution (real); its
// chain scratch is the temperature warp's, reused after the temperature solve.
struct SolveSmem {
    double2 *pf[2], *pw[2], *px[2], *pd[2], *tf[2], *tw[2], *tx[2];
    double *uf, *ux;
    float2 *tr, *tq, *td;  // refined FP32 temperature solves: residual, chain scratch, correction (MB = 1)
    float* ring32;         // coefficient rings of the FP32 temperature walks (one CTA per system)
    // the streamfunction and zonal-flow right-hand sides as assembled (pf and uf
    // become residuals), for the epilogue; past the end of solve_smem_doubles,
    // present when the launch adds keep_f_doubles (MB = 1)
    double2* fp;
    double* fu;
};

__host__ __device__ inline int round8(int n) { return (n + 7) / 8 * 8; }

// DEEP (the FP32-refined temperature solve): the FP64 temperature chain scratch
// tw is not used, so it is left out (at N_c = 1365 this lets the epilogue keep
// the assembled right-hand sides in shared memory)
__host__ __device__ inline size_t solve_smem_doubles(int nc, int MB, bool deep = false) {
    const int b = round8(nc);
    return (size_t)MB * 2 * (deep ? 6 : 7) * b + 2 * (size_t)b + 3 * (size_t)b;  // last: 3 b float2
}

__host__ __device__ inline size_t keep_f_doubles(int nc) { return 3 * (size_t)round8(nc); }

template <int MB, bool DEEP = false>
__device__ SolveSmem carve(double2* base, int nc) {
    SolveSmem s;
    const int b = round8(nc);
    double2* p = base;
    for (int i = 0; i < MB; ++i) {
        s.pf[i] = p; p += b;
        s.pw[i] = p; p += b;
        s.px[i] = p; p += b;
        s.pd[i] = p; p += b;
        s.tf[i] = p; p += b;
        if (DEEP) {
            s.tw[i] = nullptr;
        } else {
            s.tw[i] = p; p += b;
        }
        s.tx[i] = p; p += b;
    }
    double* d = reinterpret_cast<double*>(p);
    s.uf = d; d += b;
    s.ux = d; d += b;
    float2* f = reinterpret_cast<float2*>(d);
    s.tr = f; f += b;
    s.tq = f; f += b;
    s.td = f; f += b;
    s.fp = reinterpret_cast<double2*>(f);
    s.fu = reinterpret_cast<double*>(s.fp + b);
    return s;
}

// One FP64 refinement step of the zonal-flow solve (the CTA of m = 0, large N_c):
// r = f - L u over the assembled rows and the tau rows, solved with the same
// factors, u += correction.  The residual replaces the right-hand side; the
// correction and its chain scratch use streamfunction arrays, which mode 0 leaves
// unused.
__device__ void refine_zonal_flow(const StepParams& P, const DevFactors& F, SolveSmem& s) {
    const int nc = P.nc, nt = nc - 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    for (int k = 2 + tid; k < nc; k += nth) {
        const double* row = F.uBand + (size_t)(k - 2) * 9;
        double acc = s.uf[k];
        for (int d = 0; d < 9; ++d) {
            const int n = k - 4 + d;
            if (n >= 0 && n < nc) acc = fma(-__ldg(&row[d]), s.ux[n], acc);
        }
        s.uf[k] = acc;
    }
    if (warp == 0) {  // tau rows: r = 0 - tau u
        double t0 = 0.0, t1 = 0.0;
        for (int j = lane; j < nc; j += 32) {
            t0 = fma(__ldg(&P.ops.tau_dir[j]), s.ux[j], t0);
            t1 = fma(__ldg(&P.ops.tau_dir[nc + j]), s.ux[j], t1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        }
        if (lane < 2) s.uf[lane] = -(lane ? t1 : t0);
    }
    __syncthreads();
    double* du = reinterpret_cast<double*>(s.pw[0]);
    if (warp == 4 || warp == 5) {
        pair_block_solve<8, PFB>(s.uf + 2, reinterpret_cast<double*>(s.pf[0]), du + 2, nt, F.uBlk, true, warp - 4, 3);
        if (warp == 4) {
            double t0 = 0.0, t1 = 0.0;
            for (int j = lane; j < nt; j += 32) {
                t0 = fma(__ldg(&P.ops.tau_dir_B[j]), du[2 + j], t0);
                t1 = fma(__ldg(&P.ops.tau_dir_B[nt + j]), du[2 + j], t1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
            }
            const double g0 = s.uf[0], g1 = s.uf[1];
            __syncwarp();
            if (lane < 2) du[lane] = F.uSinv[lane * 2] * (g0 - t0) + F.uSinv[lane * 2 + 1] * (g1 - t1);
            __syncwarp();
        }
    }
    __syncthreads();
    {
        const double u0 = du[0], u1 = du[1];
        for (int j = tid; j < nt; j += nth) du[2 + j] -= F.uY[(size_t)j * 2] * u0 + F.uY[(size_t)j * 2 + 1] * u1;
    }
    __syncthreads();
    for (int n = tid; n < nc; n += nth) s.ux[n] += du[n];
    __syncthreads();
}

// FP64 residual r = f - L x of the temperature system of mode m0 (MB == 1),
// rounded to FP32 into s.tr: the assembled rows by the whole CTA, the two tau
// rows (r = 0 - tau x) by warp tw.  The caller synchronises.
__device__ void temperature_residual(const StepParams& P, const DevFactors& F, SolveSmem& s, int m0, int tw) {
    const int nc = P.nc, nt = nc - 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    for (int k = 2 + tid; k < nc; k += nth) {
        const double* row = F.tBand + ((size_t)m0 * nt + (k - 2)) * 9;
        double2 acc = s.tf[0][k];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int n = k - 4 + d;
            if (n >= 0 && n < nc) acc = fms(acc, __ldg(&row[d]), s.tx[0][n]);
        }
        s.tr[k] = to_f2(acc);
    }
    if (warp == tw) {
        double2 t0 = make_double2(0.0, 0.0), t1 = t0;
        for (int j = lane; j < nc; j += 32) {
            const double2 xv = s.tx[0][j];
            const double b0 = __ldg(&P.ops.tau_dir[j]), b1 = __ldg(&P.ops.tau_dir[nc + j]);
            t0.x = fma(b0, xv.x, t0.x);
            t0.y = fma(b0, xv.y, t0.y);
            t1.x = fma(b1, xv.x, t1.x);
            t1.y = fma(b1, xv.y, t1.y);
        }
        t0 = warp_sum(t0);
        t1 = warp_sum(t1);
        if (lane < 2) s.tr[lane] = to_f2(lane ? make_double2(-t1.x, -t1.y) : make_double2(-t0.x, -t0.y));
    }
}

// The FP32 temperature solve D td = tr of the kernel with one CTA per system:
// one block walked by warps 2-3, or (tsplit) its two halves by warps 2-3 and 4-5
// joined through the spikes.  Whole CTA; ends with a barrier.
__device__ void theta32_chains(const DevFactors& F, SolveSmem& s, int m, int nt, int nbt) {
    const float* tb = (F.tsplit ? F.tBlk32S : F.tBlk32) + (size_t)m * nbt * 192;
    if (F.tsplit) {
        const int ntA = 8 * (nbt / 2);
        cta_chain_solve<RD_32, float, float2, float2>(s.tr + 2, s.tq, s.td + 2, ntA, tb, 2, s.tr + 2 + ntA, s.tq + ntA,
                                                      s.td + 2 + ntA, nt - ntA, tb + (size_t)(nbt / 2) * 192, 4,
                                                      s.ring32);
        split_join32(s.td + 2, nt, ntA, F.tSpk32 + (size_t)m * nt * 8, F.tRj32 + (size_t)m * 256);
    } else {
        cta_chain_solve<RD_32, float, float2, float2>(s.tr + 2, s.tq, s.td + 2, nt, tb, 2, nullptr, nullptr, nullptr, 0,
                                                      nullptr, 0, s.ring32);
    }
}

// The same residual with the tau rows summed by the whole CTA (kernel with one
// CTA per system, where no other system's warps run beside it).  Contains one
// __syncthreads; the caller's next barrier publishes s.tr.
__device__ void temperature_residual_block(const StepParams& P, const DevFactors& F, SolveSmem& s, int m0) {
    const int nc = P.nc, nt = nc - 2;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    for (int k = 2 + tid; k < nc; k += nth) {
        const double* row = F.tBand + ((size_t)m0 * nt + (k - 2)) * 9;
        double2 acc = s.tf[0][k];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int n = k - 4 + d;
            if (n >= 0 && n < nc) acc = fms(acc, __ldg(&row[d]), s.tx[0][n]);
        }
        s.tr[k] = to_f2(acc);
    }
    const double2 t = block_rows_dot<2>(s.tx[0], nc, P.ops.tau_dir);
    if (warp == 0 && lane < 2) s.tr[lane] = to_f2(make_double2(-t.x, -t.y));
}

// The FP32-refined temperature solve of the kernel with one CTA per system:
// ir_t corrections x += S32^{-1}(f - L x), every reduction by the whole CTA.
__device__ void temperature_corrections_roles(const StepParams& P, const DevFactors& F, SolveSmem& s, int m0) {
    const int nc = P.nc, nt = nc - 2, nbt = (nt + 7) / 8;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
    for (int it = 0; it < F.ir_t; ++it) {
        temperature_residual_block(P, F, s, m0);
        __syncthreads();
        theta32_chains(F, s, m0, nt, nbt);
        block_schur32_dir(s.td, s.tr, nc, P.ops.tau_dir_B32, F.tSinv32 + (size_t)m0 * 4);
        schur_update32_dir(s.td, nc, F.tY32 + (size_t)m0 * nt * 2, 0, nth);
        __syncthreads();
        for (int n = tid; n < nc; n += nth) s.tx[0][n] = cadd(s.tx[0][n], to_d2_bits(s.td[n]));
        __syncthreads();
    }
}

// The FP32-refined temperature solve (F.ir_t > 0, MB == 1): x += S32^{-1}(f - L x)
// for the passes it0 .. ir_t - 1 (pass 0 may have run beside the streamfunction
// refinement), then the FP64 refinement of the zonal flow (mode 0).
template <int MB, bool DEEP>
__device__ void temperature_corrections(const StepParams& P, const DevFactors& F, SolveSmem& s, int m0, bool has_u,
                                        int it0) {
    const int nc = P.nc, nt = nc - 2, nbt = (nt + 7) / 8;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
    constexpr int PT = DEEP ? PFB_DEEP_T : PFB;
    if (F.ir_t) {
        for (int it = it0; it < F.ir_t; ++it) {
            temperature_residual(P, F, s, m0, 0);
            __syncthreads();
            if (warp == 2 || warp == 3)
                pair_block_solve<8, PT>(s.tr + 2, s.tq, s.td + 2, nt, F.tBlk32 + (size_t)m0 * nbt * 192, true, warp - 2, 2);
            __syncthreads();
            if (warp == 2) warp_schur32_dir(s.td, s.tr, nc, P.ops.tau_dir_B32, F.tSinv32 + (size_t)m0 * 4);
            __syncthreads();
            schur_update32_dir(s.td, nc, F.tY32 + (size_t)m0 * nt * 2, 0, nth);
            __syncthreads();
            for (int n = tid; n < nc; n += nth) s.tx[0][n] = cadd(s.tx[0][n], to_d2_bits(s.td[n]));
            __syncthreads();
        }
        if (has_u) refine_zonal_flow(P, F, s);  // FP64
    }
}

template <int MB, bool DEEP, bool DDP = false>
__global__ void __launch_bounds__(NTHREADS_S) k_solve(StepParams P, RhsSpec R, DevFactors F, VecSet y_out,
                                                      VecSet mass_out, VecSet imp_out, int want_mass,
                                                      int want_imp, int keep_f) {
    extern __shared__ double2 sm[];
    const int nc = P.nc, M = P.M;
    const int m0 = P.m_lo + blockIdx.x * MB;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int np = nc - 4, nt = nc - 2;
    const int nbp = (np + 7) / 8, nbt = (nt + 7) / 8;
    const int nA = 8 * (nbp / 2);  // first half of a split streamfunction block (F.psplit)
    SolveSmem s = carve<MB, DEEP>(sm, nc);
    const bool has_u = (m0 == 0);
    constexpr int PP = DEEP ? PFB_DEEP_P : PFB, PT = DEEP ? PFB_DEEP_T : PFB;

    // 1. right-hand side sum_t c_t V_t (tau rows zero)
    for (int idx = tid; idx < MB * nc; idx += nth) {
        const int mi = idx / nc, n = idx - mi * nc, m = m0 + mi;
        if (m >= M) continue;
        double2 ap = make_double2(0.0, 0.0), at = make_double2(0.0, 0.0);
        double au = 0.0;
#pragma unroll 4
        for (int t = 0; t < R.nterms; ++t) {
            const double c = R.t[t].c;
            const double2 vp = R.t[t].v.psi[(size_t)m * nc + n];
            const double2 vt = R.t[t].v.th[(size_t)m * nc + n];
            ap.x = fma(c, vp.x, ap.x);
            ap.y = fma(c, vp.y, ap.y);
            at.x = fma(c, vt.x, at.x);
            at.y = fma(c, vt.y, at.y);
            if (m == 0) au = fma(c, R.t[t].v.u[n], au);
        }
        s.pf[mi][n] = (n < 4 || m == 0) ? make_double2(0.0, 0.0) : ap;
        // double-float streamfunction chains (explicit buoyancy, MB = 1): the
        // right-hand side as double-floats in pd, which the correction fills later
        if (DDP && m > 0) reinterpret_cast<ddc*>(s.pd[0])[n] = dd_from_bits(s.pf[0][n]);
        s.tf[mi][n] = (n < 2) ? make_double2(0.0, 0.0) : at;
        if (F.ir_t) s.tr[n] = to_f2(s.tf[mi][n]);  // MB == 1 with ir_t
        if (m == 0) s.uf[n] = (n < 2) ? 0.0 : au;
        if (MB == 1 && keep_f) {  // for the epilogue: pf and uf become residuals
            s.fp[n] = s.pf[mi][n];
            if (m == 0) s.fu[n] = s.uf[n];
        }
    }
    __syncthreads();

    // 2.-4. banded solves, Schur steps and Y updates.  With explicit buoyancy the
    //    streamfunction and temperature systems are independent and run together;
    //    with implicit buoyancy (Section 4) the temperature (and zonal flow) goes
    //    first, then g (Ra/Pr)(i m/s_o) C^I theta_new joins the streamfunction rows.
    const int npass = P.buoy_imp ? 2 : 1;
    for (int pass = 0; pass < npass; ++pass) {
        const bool do_p = !P.buoy_imp || pass == 1;
        const bool do_t = !P.buoy_imp || pass == 0;
        if (P.buoy_imp && pass == 1) {
            if (m0 > 0) {
                const double cb = F.gdt * P.Ra / P.Pr * (double)m0 / P.s_o;
                for (int k = 4 + tid; k < nc; k += nth)
                    s.pf[0][k] = cadd(s.pf[0][k], cmul_i(band_row_c<8>(P.ops.band[OP_C], s.tx[0], k, nc), cb));
            }
            __syncthreads();
        }
        // 2. banded solves by warp pairs meeting at their middle blocks: warps 0-1
        //    streamfunction, 2-3 temperature, 4-5 zonal flow (m = 0 only; its chain
        //    scratch is the streamfunction correction array, unused until step 5)
        if (warp < 2) {
            if (do_p) {
                const bool act = m0 > 0;
                if constexpr (DDP)
                    pair_block_solve<8, PP, ddc, ddc, dacc>(
                        reinterpret_cast<ddc*>(s.pd[0]) + 4, reinterpret_cast<ddc*>(s.pw[0]),
                        reinterpret_cast<ddc*>(s.px[0]) + 4, F.psplit ? nA : np,
                        reinterpret_cast<const ddc*>(F.pBlkDD) + (size_t)(act ? m0 : 0) * nbp * 192, act, warp, 1);
                else
                    pair_block_solve<8, PP>(s.pf[0] + 4, s.pw[0], s.px[0] + 4, F.psplit ? nA : np,
                                            F.pBlk + (size_t)(act ? m0 : 0) * nbp * 192, act, warp, 1);
            }
        } else if (warp >= 6) {
            if (do_p && F.psplit) {  // the second half of the streamfunction block
                const bool act = m0 > 0;
                if constexpr (DDP)
                    pair_block_solve<8, PP, ddc, ddc, dacc>(
                        reinterpret_cast<ddc*>(s.pd[0]) + 4 + nA, reinterpret_cast<ddc*>(s.pw[0]) + nA,
                        reinterpret_cast<ddc*>(s.px[0]) + 4 + nA, np - nA,
                        reinterpret_cast<const ddc*>(F.pBlkDD) + ((size_t)(act ? m0 : 0) * nbp + nbp / 2) * 192, act,
                        warp - 6, 4);
                else
                    pair_block_solve<8, PP>(s.pf[0] + 4 + nA, s.pw[0] + nA, s.px[0] + 4 + nA, np - nA,
                                            F.pBlk + ((size_t)(act ? m0 : 0) * nbp + nbp / 2) * 192, act, warp - 6, 4);
            }
        } else if (warp < 4) {
            if (do_t) {
                if (F.ir_t)
                    pair_block_solve<8, PT>(s.tr + 2, s.tq, s.td + 2, nt, F.tBlk32 + (size_t)m0 * nbt * 192, true, warp - 2,
                                        2);
                else
                    pair_block_solve<8, PP>(s.tf[0] + 2, s.tw[0], s.tx[0] + 2, nt, F.tBlk + (size_t)m0 * nbt * 192, true,
                                        warp - 2, 2);
            }
        } else if (warp < 6 && has_u) {
            if (do_t)
                pair_block_solve<8, PFB>(s.uf + 2, reinterpret_cast<double*>(s.pd[0]), s.ux + 2, nt, F.uBlk, true, warp - 4,
                                    3);
        }
        __syncthreads();
        if (DDP && do_p && m0 > 0) {  // the solution back from double-floats
            const ddc* xd = reinterpret_cast<const ddc*>(s.px[0]);
            for (int n = 4 + tid; n < nc; n += nth) s.px[0][n] = dd_compose(xd[n]);
            __syncthreads();
        }
        if (do_p && F.psplit)
            split_join(s.px[0] + 4, np, nA, F.pSpk + (size_t)(m0 > 0 ? m0 : 0) * np * 8,
                       F.pRj + (size_t)(m0 > 0 ? m0 : 0) * 256, m0 > 0);

        // 3. Schur steps: warp 0 streamfunction, 2 temperature, 4 zonal flow
        if (warp == 0) {
            if (do_p && m0 > 0) warp_schur<4>(s.px[0], nullptr, nc, P.ops.tau_psi_B, F.pSinv + (size_t)m0 * 16);
        } else if (warp == 2) {
            if (do_t) {
                if (F.ir_t)
                    warp_schur32_dir(s.td, s.tr, nc, P.ops.tau_dir_B32, F.tSinv32 + (size_t)m0 * 4);
                else
                    warp_schur<2>(s.tx[0], nullptr, nc, P.ops.tau_dir_B, F.tSinv + (size_t)m0 * 4);
            }
        } else if (warp == 4 && has_u && do_t) {
            double t0 = 0.0, t1 = 0.0;
            for (int j = lane; j < nt; j += 32) {
                t0 = fma(__ldg(&P.ops.tau_dir_B[j]), s.ux[2 + j], t0);
                t1 = fma(__ldg(&P.ops.tau_dir_B[nt + j]), s.ux[2 + j], t1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
            }
            if (lane < 2) s.ux[lane] = -(F.uSinv[lane * 2] * t0 + F.uSinv[lane * 2 + 1] * t1);
            __syncwarp();
        }
        __syncthreads();
        // 4. y2 -= Y y1 (threads split evenly over the systems of the CTA)
        {
            const int per = nth / (2 * MB);
            const int sys = tid / per, t0 = sys * per;
            if (sys < MB) {
                const int m = m0 + sys;
                if (do_p && m < M && m > 0) schur_update<4>(s.px[sys], nc, F.pY + (size_t)m * np * 4, t0, per);
            } else if (sys < 2 * MB) {
                const int mi = sys - MB, m = m0 + mi;
                if (do_t && m < M) {
                    if (F.ir_t)
                        schur_update32_dir(s.td, nc, F.tY32 + (size_t)m * nt * 2, t0, per);
                    else
                        schur_update<2>(s.tx[mi], nc, F.tY + (size_t)m * nt * 2, t0, per);
                }
            }
            if (has_u && do_t) {
                __syncthreads();
                const double u0 = s.ux[0], u1 = s.ux[1];
                for (int j = tid; j < nt; j += nth)
                    s.ux[2 + j] -= F.uY[(size_t)j * 2] * u0 + F.uY[(size_t)j * 2 + 1] * u1;
            }
        }
        __syncthreads();
        if (F.ir_t && do_t) {  // the FP32 temperature solve becomes the FP64 iterate
            for (int n = tid; n < nc; n += nth) s.tx[0][n] = to_d2_bits(s.td[n]);
            __syncthreads();
        }
        if (P.buoy_imp && pass == 0) temperature_corrections<MB, DEEP>(P, F, s, m0, has_u, 0);
    }

    // 5. one refinement step of the streamfunction solve: r = f - L x (a second
    //    step gains nothing: FP64 residuals limit the accuracy to ~cond * eps).
    //    With the FP32-refined temperature solve and explicit buoyancy the first
    //    temperature correction runs beside it: its chain (FP32, warps 2-3) beside
    //    the streamfunction chains (FP64), on disjoint arrays.
    const bool fuse_t = F.ir_t && !P.buoy_imp;
    for (int it = 0; it < 1; ++it) {
    for (int idx = tid; idx < MB * nc; idx += nth) {
        const int mi = idx / nc, k = idx - mi * nc, m = m0 + mi;
        if (m >= M || m == 0 || k < 4) continue;
        const double2* row = F.pBand + ((size_t)m * np + (k - 4)) * 17;
        // pass 0: r = f - L x; later passes: r <- r - L d (d: the last correction)
        const double2* x = it ? s.pd[mi] : s.px[mi];
        double2 acc = s.pf[mi][k];
#pragma unroll
        for (int d = 0; d < 17; ++d) {
            const int n = k - 8 + d;
            if (n >= 0 && n < nc) acc = fms(acc, __ldg(&row[d]), x[n]);
        }
        s.pf[mi][k] = acc;  // the residual replaces the right-hand side
        if (DDP) reinterpret_cast<ddc*>(s.pf[0])[k] = dd_from_bits(acc);  // in place, as double-floats
    }
    if (warp < MB) {  // tau rows: r = 0 - tau x
        const int m = m0 + warp;
        if (m < M && m > 0) {
            double2 t[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) t[r] = make_double2(0.0, 0.0);
            for (int j = lane; j < nc; j += 32) {
                const double2 xv = it ? s.pd[warp][j] : s.px[warp][j];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const double b = __ldg(&P.ops.tau_psi[(size_t)r * nc + j]);
                    t[r].x = fma(b, xv.x, t[r].x);
                    t[r].y = fma(b, xv.y, t[r].y);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) t[r] = warp_sum(t[r]);
            if (lane < 4) s.pf[warp][lane] = csub(s.pf[warp][lane], t[lane]);
        }
    }
    if (fuse_t) temperature_residual(P, F, s, m0, 1);
    __syncthreads();
    if (warp < 2) {
        const bool act = m0 > 0;
        if constexpr (DDP) {
            pair_block_solve<8, PP, ddc, ddc, dacc>(
                reinterpret_cast<ddc*>(s.pf[0]) + 4, reinterpret_cast<ddc*>(s.pw[0]), reinterpret_cast<ddc*>(s.pd[0]) + 4,
                F.psplit ? nA : np, reinterpret_cast<const ddc*>(F.pBlkDD) + (size_t)(act ? m0 : 0) * nbp * 192, act,
                warp, 1);
            if (!F.psplit && act) {  // the pair converts its solution back, then warp 0 takes the Schur step
                const ddc* xd = reinterpret_cast<const ddc*>(s.pd[0]);
                for (int n = 4 + (tid & 63); n < nc; n += 64) s.pd[0][n] = dd_compose(xd[n]);
                pair_sync(1);
                if (warp == 0) warp_schur<4>(s.pd[0], s.pf[0], nc, P.ops.tau_psi_B, F.pSinv + (size_t)m0 * 16);
            }
        } else {
            pair_block_solve<8, PP>(s.pf[0] + 4, s.pw[0], s.pd[0] + 4, F.psplit ? nA : np,
                                    F.pBlk + (size_t)(act ? m0 : 0) * nbp * 192, act, warp, 1);
            if (!F.psplit && act && warp == 0)
                warp_schur<4>(s.pd[0], s.pf[0], nc, P.ops.tau_psi_B, F.pSinv + (size_t)m0 * 16);
        }
    } else if (warp >= 6 && F.psplit) {
        const bool act = m0 > 0;
        if constexpr (DDP)
            pair_block_solve<8, PP, ddc, ddc, dacc>(
                reinterpret_cast<ddc*>(s.pf[0]) + 4 + nA, reinterpret_cast<ddc*>(s.pw[0]) + nA,
                reinterpret_cast<ddc*>(s.pd[0]) + 4 + nA, np - nA,
                reinterpret_cast<const ddc*>(F.pBlkDD) + ((size_t)(act ? m0 : 0) * nbp + nbp / 2) * 192, act, warp - 6, 4);
        else
            pair_block_solve<8, PP>(s.pf[0] + 4 + nA, s.pw[0] + nA, s.pd[0] + 4 + nA, np - nA,
                                    F.pBlk + ((size_t)(act ? m0 : 0) * nbp + nbp / 2) * 192, act, warp - 6, 4);
    } else if (fuse_t && warp < 4) {
        pair_block_solve<8, PT>(s.tr + 2, s.tq, s.td + 2, nt, F.tBlk32 + (size_t)m0 * nbt * 192, true, warp - 2, 2);
        if (warp == 2) warp_schur32_dir(s.td, s.tr, nc, P.ops.tau_dir_B32, F.tSinv32 + (size_t)m0 * 4);
    }
    __syncthreads();
    if (DDP && F.psplit && m0 > 0) {  // the split solution back from double-floats before the join
        const ddc* xd = reinterpret_cast<const ddc*>(s.pd[0]);
        for (int n = 4 + tid; n < nc; n += nth) s.pd[0][n] = dd_compose(xd[n]);
        __syncthreads();
    }
    if (F.psplit) {
        split_join(s.pd[0] + 4, np, nA, F.pSpk + (size_t)(m0 > 0 ? m0 : 0) * np * 8,
                   F.pRj + (size_t)(m0 > 0 ? m0 : 0) * 256, m0 > 0);
        if (m0 > 0 && warp == 0) warp_schur<4>(s.pd[0], s.pf[0], nc, P.ops.tau_psi_B, F.pSinv + (size_t)m0 * 16);
        __syncthreads();
    }
    {
        const int per = nth / MB;
        const int sys = tid / per, t0 = sys * per;
        const int m = m0 + sys;
        if (sys < MB && m < M && m > 0) schur_update<4>(s.pd[sys], nc, F.pY + (size_t)m * np * 4, t0, per);
        if (fuse_t) schur_update32_dir(s.td, nc, F.tY32 + (size_t)m0 * nt * 2, 0, nth);
    }
    __syncthreads();
    for (int idx = tid; idx < MB * nc; idx += nth) {
        const int mi = idx / nc, n = idx - mi * nc, m = m0 + mi;
        if (m >= M) continue;
        s.px[mi][n] = (m == 0) ? make_double2(0.0, 0.0) : cadd(s.px[mi][n], s.pd[mi][n]);
        if (fuse_t) s.tx[0][n] = cadd(s.tx[0][n], to_d2_bits(s.td[n]));
    }
    __syncthreads();
    }
    if (!P.buoy_imp) temperature_corrections<MB, DEEP>(P, F, s, m0, has_u, fuse_t ? 1 : 0);

    // 6. store, then mass / implicit operators for later stages
    for (int idx = tid; idx < MB * nc; idx += nth) {
        const int mi = idx / nc, n = idx - mi * nc, m = m0 + mi;
        if (m >= M) continue;
        y_out.psi[(size_t)m * nc + n] = s.px[mi][n];
        y_out.th[(size_t)m * nc + n] = s.tx[mi][n];
        if (m == 0) y_out.u[n] = s.ux[n];
        if (want_mass || want_imp)
            epilogue_row(P, R, F.gdt, m, n, s.px[mi], s.tx[mi], s.ux, mass_out, imp_out, want_mass, want_imp,
                         (MB == 1 && keep_f) ? s.fp : nullptr, s.tf[mi], s.fu);
    }
}

// ---------------------------------------------------------------------------
// The same solve split by system over two CTAs per mode (large N_c, FP32-refined
// temperature, explicit buoyancy): role 0 the streamfunction system, role 1 the
// temperature system (and, for m = 0, the zonal flow after it).  The systems are
// independent when the buoyancy is explicit; each role holds only its own arrays
// in shared memory (at N_c = 1365: 109 KB and 98 KB instead of 219 KB) and the
// kernel is capped at 128 registers, so two CTAs share an SM and one's block
// chains overlap the other's residual, Schur and epilogue phases.  Interleaved
// roles (block 2m + role) give every SM a mix.  The same arithmetic as k_solve
// with fuse_t = 0; chain prefetch depth 2.
// ---------------------------------------------------------------------------
__device__ void epilogue_row_psi(const StepParams& P, const RhsSpec& R, double gdt, int m, int k, const double2* xp,
                                 VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp,
                                 const double2* fps) {
    const int nc = P.nc;
    const double mu = (double)m * m;
    double2 mp = make_double2(0.0, 0.0);
    if (m > 0 && k >= 4) {
        // A^I_m = A0 + m^2 A2 assembled tap by tap: three FMAs a tap instead of four
        const double* r0 = P.ops.band[OP_A0] + (size_t)k * 17;
        const double* r2 = P.ops.band[OP_A2] + (size_t)k * 17;
#pragma unroll
        for (int d = 0; d < 17; ++d) {
            const int n = k - 8 + d;
            if (n >= 0 && n < nc) {
                const double c = fma(mu, __ldg(&r2[d]), __ldg(&r0[d]));
                mp.x = fma(c, xp[n].x, mp.x);
                mp.y = fma(c, xp[n].y, mp.y);
            }
        }
    }
    const size_t idx = (size_t)m * nc + k;
    if (want_imp) {  // before any store: an output may be one of the terms of f
        const double2 fp = fps[k];
        imp_out.psi[idx] = (m > 0 && k >= 4) ? cscale(csub(mp, fp), 1.0 / gdt) : make_double2(0.0, 0.0);
    }
    if (want_mass) mass_out.psi[idx] = mp;
}

__device__ void epilogue_row_theta(const StepParams& P, const RhsSpec& R, double gdt, int m, int k, const double2* xt,
                                   const double* xu, VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp,
                                   const double2* fts) {
    const int nc = P.nc;
    double2 mt = make_double2(0.0, 0.0);
    double muu = 0.0;
    if (k >= 2) {
        mt = band_row_c<4>(P.ops.band[OP_D], xt, k, nc);
        if (m == 0) {
            const double* rd = P.ops.band[OP_D] + (size_t)k * 9;
            for (int d = 0; d < 9; ++d) {
                const int n = k - 4 + d;
                if (n >= 0 && n < nc) muu = fma(__ldg(&rd[d]), xu[n], muu);
            }
        }
    }
    const size_t idx = (size_t)m * nc + k;
    if (want_imp) {  // before any store: an output may be one of the terms of f
        const double2 ft = fts[k];
        double fu = 0.0;
        if (m == 0)
            for (int t = 0; t < R.nterms; ++t) fu = fma(R.t[t].c, R.t[t].v.u[k], fu);
        const double ig = 1.0 / gdt;
        imp_out.th[idx] = (k >= 2) ? cscale(csub(mt, ft), ig) : make_double2(0.0, 0.0);
        if (m == 0) imp_out.u[k] = (k >= 2) ? (muu - fu) * ig : 0.0;
    }
    if (want_mass) {
        mass_out.th[idx] = mt;
        if (m == 0) mass_out.u[k] = muu;
    }
}

// Shared memory of the kernel with one CTA per system, bytes: the larger role.
// Role 0 with double-float chains: pf, pw, px, fp (double2) and the rings of its
// four walking warps (RD_DD matrices of complex double-floats each); with FP64
// chains pf, pw, px, pd, fp.  Role 1: tf, tx (double2), tr, tq, td (float2), uf,
// ux (double) and the rings of its (up to four) walking warps (RD_32 FP32 matrices).
__host__ __device__ inline size_t solve_roles_smem_bytes(int nc, bool ddp) {
    const size_t b = (size_t)round8(nc);
    const size_t psi = ddp ? 4 * b * 16 + 4 * (size_t)RD_DD * 64 * 16 : 5 * b * 16;
    const size_t th = 2 * b * 16 + 3 * b * 8 + 2 * b * 8 + 4 * (size_t)RD_32 * 64 * 4;
    return psi > th ? psi : th;
}

template <bool DDP>
__global__ void __launch_bounds__(NTHREADS_S, 2) k_solve_roles(StepParams P, RhsSpec R, DevFactors F, VecSet y_out,
                                                                VecSet mass_out, VecSet imp_out, int want_mass,
                                                                int want_imp) {
    extern __shared__ double2 sm[];
    const int nc = P.nc;
    const int m = P.m_lo + (int)(blockIdx.x >> 1), role = blockIdx.x & 1;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int np = nc - 4, nt = nc - 2;
    const int nbp = (np + 7) / 8;
    const int nA = 8 * (nbp / 2);
    const int b = round8(nc);
    SolveSmem s{};
    if (role == 0) {
        // ---------------------------------------------------- streamfunction
        s.pf[0] = sm;
        s.pw[0] = sm + b;
        s.px[0] = sm + 2 * b;
        s.pd[0] = DDP ? nullptr : sm + 3 * b;  // double-float chains: the correction in place of the residual
        s.fp = DDP ? sm + 3 * b : sm + 4 * b;
        ddc* ring = reinterpret_cast<ddc*>(sm + 4 * b);  // double-float chains only
        if (m == 0) {  // Psi_0 = 0
            for (int n = tid; n < nc; n += nth) {
                y_out.psi[n] = make_double2(0.0, 0.0);
                if (want_mass) mass_out.psi[n] = make_double2(0.0, 0.0);
                if (want_imp) imp_out.psi[n] = make_double2(0.0, 0.0);
            }
            return;
        }
        // two rows per thread and pass: twice the loads in flight
        for (int n0 = tid; n0 < nc; n0 += 2 * nth) {
            const int n1 = n0 + nth;
            double2 a0 = make_double2(0.0, 0.0), a1 = a0;
#pragma unroll 4
            for (int t = 0; t < R.nterms; ++t) {
                const double c = R.t[t].c;
                const double2 v0 = R.t[t].v.psi[(size_t)m * nc + n0];
                const double2 v1 = (n1 < nc) ? R.t[t].v.psi[(size_t)m * nc + n1] : make_double2(0.0, 0.0);
                a0.x = fma(c, v0.x, a0.x);
                a0.y = fma(c, v0.y, a0.y);
                a1.x = fma(c, v1.x, a1.x);
                a1.y = fma(c, v1.y, a1.y);
            }
            s.pf[0][n0] = (n0 < 4) ? make_double2(0.0, 0.0) : a0;
            s.fp[n0] = s.pf[0][n0];
            if (n1 < nc) {
                s.pf[0][n1] = (n1 < 4) ? make_double2(0.0, 0.0) : a1;
                s.fp[n1] = s.pf[0][n1];
            }
        }
        __syncthreads();
        const double2* blk = F.pBlk + (size_t)m * nbp * 192;
        const ddc* blkd = reinterpret_cast<const ddc*>(F.pBlkDD) + (size_t)m * nbp * 192;
        ddc* zd = reinterpret_cast<ddc*>(s.pw[0]);
        for (int it = 0; it < 2; ++it) {  // solve, then one refinement step
            // double-float chains: pass 0 solves into px, pass 1 (the correction)
            // into pf, over its own right-hand side (the residual): the walks read
            // a block's right-hand side before they write its solution
            double2* x = it ? (DDP ? s.pf[0] : s.pd[0]) : s.px[0];
            if constexpr (DDP) {
                // The conversions between FP64 and double-float run on the FP64
                // pipe, so they happen here for the whole vector at once, off the
                // chains' dependent path: the right-hand side in place (f stays in
                // fp for the residual and the epilogue), the solution back from
                // double-floats in place.
                ddc* bd = reinterpret_cast<ddc*>(s.pf[0]);
                ddc* xd = reinterpret_cast<ddc*>(x);
                for (int n = 4 + tid; n < nc; n += nth) bd[n] = dd_from(s.pf[0][n]);
                __syncthreads();
                cta_chain_solve<RD_DD, ddc, ddc, dacc>(bd + 4, zd, xd + 4, F.psplit ? nA : np, blkd, 0, bd + 4 + nA, zd + nA,
                                                       xd + 4 + nA, F.psplit ? np - nA : 0,
                                                       blkd + (size_t)(nbp / 2) * 192, 6, ring);
                if (F.psplit)
                    split_join_dd(xd + 4, np, nA, reinterpret_cast<const ddc*>(F.pSpkDD) + (size_t)m * np * 8,
                                  reinterpret_cast<const ddc*>(F.pRjDD) + (size_t)m * 256, true);
                for (int n = 4 + tid; n < nc; n += nth) x[n] = dd_compose(xd[n]);
            } else {
                if (warp < 2)
                    pair_block_solve<8, PFB>(s.pf[0] + 4, s.pw[0], x + 4, F.psplit ? nA : np, blk, true, warp, 1);
                else if (warp >= 6 && F.psplit)
                    pair_block_solve<8, PFB>(s.pf[0] + 4 + nA, s.pw[0] + nA, x + 4 + nA, np - nA,
                                             blk + (size_t)(nbp / 2) * 192, true, warp - 6, 4);
            }
            __syncthreads();
            if (!DDP && F.psplit)
                split_join(x + 4, np, nA, F.pSpk + (size_t)m * np * 8, F.pRj + (size_t)m * 256, true);
            block_schur<4>(x, it ? s.pf[0] : nullptr, nc, P.ops.tau_psi_B, F.pSinv + (size_t)m * 16);
            schur_update<4>(x, nc, F.pY + (size_t)m * np * 4, 0, nth);
            __syncthreads();
            if (it == 0) {
                // residual r = f - L x over the assembled rows, and the tau rows
                // (whose f is zero)
                for (int k = 4 + tid; k < nc; k += nth) {
                    const double2* row = F.pBand + ((size_t)m * np + (k - 4)) * 17;
                    double2 acc = s.fp[k];
#pragma unroll
                    for (int d = 0; d < 17; ++d) {
                        const int n = k - 8 + d;
                        if (n >= 0 && n < nc) acc = fms(acc, __ldg(&row[d]), s.px[0][n]);
                    }
                    s.pf[0][k] = acc;
                }
                const double2 t = block_rows_dot<4>(s.px[0], nc, P.ops.tau_psi);
                if (warp == 0 && lane < 4) s.pf[0][lane] = make_double2(-t.x, -t.y);
                __syncthreads();
            }
        }
        {
            const double2* d = DDP ? s.pf[0] : s.pd[0];
            for (int n = tid; n < nc; n += nth) s.px[0][n] = cadd(s.px[0][n], d[n]);
        }
        __syncthreads();
        for (int n = tid; n < nc; n += nth) {
            y_out.psi[(size_t)m * nc + n] = s.px[0][n];
            if (want_mass || want_imp)
                epilogue_row_psi(P, R, F.gdt, m, n, s.px[0], mass_out, imp_out, want_mass, want_imp, s.fp);
        }
        return;
    }
    // ------------------------------------------- temperature (and zonal flow)
    // FP32-refined (ir_t): tf, tx, then the FP32 tr, tq, td; otherwise FP64 blocks
    // with tw as chain scratch in the place of tr
    s.tf[0] = sm;
    s.tx[0] = sm + b;
    float2* f32 = reinterpret_cast<float2*>(sm + 2 * b);
    s.tr = f32;
    s.tq = f32 + b;
    s.td = f32 + 2 * b;
    s.tw[0] = reinterpret_cast<double2*>(f32);  // FP64 path: b double2 over tr and tq
    double* d64 = reinterpret_cast<double*>(f32 + 3 * b);
    s.uf = d64;
    s.ux = d64 + b;
    s.ring32 = reinterpret_cast<float*>(d64 + 2 * b);
    const int nbt = (nt + 7) / 8;
    for (int n0 = tid; n0 < nc; n0 += 2 * nth) {  // two rows per thread and pass
        const int n1 = n0 + nth;
        double2 a0 = make_double2(0.0, 0.0), a1 = a0;
        double u0 = 0.0, u1 = 0.0;
#pragma unroll 4
        for (int t = 0; t < R.nterms; ++t) {
            const double c = R.t[t].c;
            const double2 v0 = R.t[t].v.th[(size_t)m * nc + n0];
            const double2 v1 = (n1 < nc) ? R.t[t].v.th[(size_t)m * nc + n1] : make_double2(0.0, 0.0);
            a0.x = fma(c, v0.x, a0.x);
            a0.y = fma(c, v0.y, a0.y);
            a1.x = fma(c, v1.x, a1.x);
            a1.y = fma(c, v1.y, a1.y);
            if (m == 0) {
                u0 = fma(c, R.t[t].v.u[n0], u0);
                if (n1 < nc) u1 = fma(c, R.t[t].v.u[n1], u1);
            }
        }
        s.tf[0][n0] = (n0 < 2) ? make_double2(0.0, 0.0) : a0;
        if (F.ir_t) s.tr[n0] = to_f2(s.tf[0][n0]);
        if (m == 0) s.uf[n0] = (n0 < 2) ? 0.0 : u0;
        if (n1 < nc) {
            s.tf[0][n1] = (n1 < 2) ? make_double2(0.0, 0.0) : a1;
            if (F.ir_t) s.tr[n1] = to_f2(s.tf[0][n1]);
            if (m == 0) s.uf[n1] = (n1 < 2) ? 0.0 : u1;
        }
    }
    __syncthreads();
    if (F.ir_t) {
        theta32_chains(F, s, m, nt, nbt);
        block_schur32_dir(s.td, s.tr, nc, P.ops.tau_dir_B32, F.tSinv32 + (size_t)m * 4);
        schur_update32_dir(s.td, nc, F.tY32 + (size_t)m * nt * 2, 0, nth);
        __syncthreads();
        for (int n = tid; n < nc; n += nth) s.tx[0][n] = to_d2_bits(s.td[n]);
        __syncthreads();
        temperature_corrections_roles(P, F, s, m);
    } else {
        if (warp == 2 || warp == 3)
            pair_block_solve<8, PFB>(s.tf[0] + 2, s.tw[0], s.tx[0] + 2, nt, F.tBlk + (size_t)m * nbt * 192, true,
                                     warp - 2, 2);
        __syncthreads();
        block_schur<2>(s.tx[0], nullptr, nc, P.ops.tau_dir_B, F.tSinv + (size_t)m * 4);
        schur_update<2>(s.tx[0], nc, F.tY + (size_t)m * nt * 2, 0, nth);
        __syncthreads();
    }
    if (m == 0) {
        // the zonal flow after the temperature, in its freed FP32 arrays (the
        // same footprint in doubles): chain scratch in tq, correction in td, the
        // refinement's chain scratch in tr
        s.pd[0] = reinterpret_cast<double2*>(s.tq);
        s.pw[0] = reinterpret_cast<double2*>(s.td);
        s.pf[0] = reinterpret_cast<double2*>(s.tr);
        if (warp == 4 || warp == 5)
            pair_block_solve<8, PFB>(s.uf + 2, reinterpret_cast<double*>(s.pd[0]), s.ux + 2, nt, F.uBlk, true, warp - 4, 3);
        __syncthreads();
        if (warp == 4) {
            double t0 = 0.0, t1 = 0.0;
            for (int j = lane; j < nt; j += 32) {
                t0 = fma(__ldg(&P.ops.tau_dir_B[j]), s.ux[2 + j], t0);
                t1 = fma(__ldg(&P.ops.tau_dir_B[nt + j]), s.ux[2 + j], t1);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
            }
            if (lane < 2) s.ux[lane] = -(F.uSinv[lane * 2] * t0 + F.uSinv[lane * 2 + 1] * t1);
            __syncwarp();
        }
        __syncthreads();
        {
            const double u0 = s.ux[0], u1 = s.ux[1];
            for (int j = tid; j < nt; j += nth) s.ux[2 + j] -= F.uY[(size_t)j * 2] * u0 + F.uY[(size_t)j * 2 + 1] * u1;
        }
        __syncthreads();
        if (F.ir_t) refine_zonal_flow(P, F, s);
    }
    for (int n = tid; n < nc; n += nth) {
        y_out.th[(size_t)m * nc + n] = s.tx[0][n];
        if (m == 0) y_out.u[n] = s.ux[n];
        if (want_mass || want_imp)
            epilogue_row_theta(P, R, F.gdt, m, n, s.tx[0], s.ux, mass_out, imp_out, want_mass, want_imp, s.tf[0]);
    }
}

// ---------------------------------------------------------------------------
// Galerkin-basis solve (Appendix B; option "radial" = 2).  Per mode the square
// systems P_4 (A - g dt B) S_Psi x = P_4 r and P_2 (D - g dt F/Pr) S_D x = P_2 r
// (and the zonal-flow one) are solved with their banded LU factors with partial
// pivoting (host_ops.h, band_lu_pivot), then expanded to Chebyshev coefficients:
// f_hat_k = (1/(C w_k)) sum_i S(k, n) x_n.  The same discrete problem as the tau
// solve, without border rows, Schur steps or refinement.
//
// A system is solved by one warp in two sweeps of n dependent steps each.  The
// rows the next steps touch sit in a register window across the lanes:
//   forward (L, interchanges interleaved): lanes 0..KL hold b[j..j+KL]; step j
//     swaps row j with row j + piv[j], lanes 1..KL subtract l_t b_j, the window
//     shifts down one lane and lane KL takes b[j+KL+1];
//   backward (U, column by column, with U's columns divided by their diagonal
//     entries): lanes 0..KK hold y[i..i-KK]; step i takes y_i final, lanes
//     1..KK subtract (U(i-t, i)/U_ii) y_i, the window shifts; x_i = y_i / U_ii
//     is formed afterwards by the whole CTA (off the chain).
// A step's chain is two shuffles and one or two dependent FMAs; the factors are
// staged through shared memory in chunks of GCH rows by asynchronous copies, the
// next chunk in flight while the current one is used.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double shfl_down_x(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double2 shfl_down_x(double2 v) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Asynchronous 16-byte global -> shared copies (cp.async): a lane's copies
// complete at cp.async.wait_group; __syncwarp then publishes them to the warp.

constexpr int GCH = 32;  // rows of factors staged per chunk

// Copy rows [r0, r1) of a row-major factor array (W entries of TF per row, W *
// sizeof(TF) a multiple of 16 bytes, the array 16-byte aligned) to dst, by one warp.
template <int W, class TF>
__device__ __forceinline__ void stage_rows(TF* dst, const TF* src, int r0, int r1) {
    constexpr int PER = W * (int)sizeof(TF) / 16;
    static_assert(PER * 16 == W * (int)sizeof(TF), "factor rows must be whole 16-byte pieces");
    const char* s = reinterpret_cast<const char*>(src + (size_t)r0 * W);
    char* d = reinterpret_cast<char*>(dst);
    for (int q = threadIdx.x & 31; q < (r1 - r0) * PER; q += 32) cp_async16(d + 16 * q, s + 16 * q);
}

// b: right-hand side (n entries, row-scaled), overwritten by the forward result;
// x: y = U_ii x_i (n entries; the caller multiplies by Uc[i][0] = 1/U_ii).
// Lm [n][KL], Uc [n][UW] (UW >= KK+1, padded to whole 16-byte rows):
// band_lu_pivot's factors; pv: the pivot offsets in shared memory.
// stg: shared staging of 2 GCH rows of Uc (which also holds 2 GCH rows of Lm):
// chunk k+1 of the factors is copied while chunk k is used.
template <int KL, int KK, int UW, class TF, class TX>
__device__ void warp_band_solve(TX* b, TX* x, int n, const TF* __restrict__ Lm, const TF* __restrict__ Uc,
                                const unsigned char* pv, TF* stg) {
    static_assert(KK < 32 && KL <= KK && UW >= KK + 1, "window wider than a warp");
    const int lane = threadIdx.x & 31;
    const bool lrow = lane >= 1 && lane <= KL, urow = lane >= 1 && lane <= KK;
    // forward: L z = P b
    TX w = (lane <= KL && lane < n) ? b[lane] : zero<TX>();
    stage_rows<KL>(stg, Lm, 0, min(n, GCH));
    cp_async_commit();
    for (int c0 = 0, k = 0; c0 < n; c0 += GCH, k ^= 1) {
        const int c1 = min(n, c0 + GCH);
        if (c1 < n) stage_rows<KL>(stg + (k ^ 1) * GCH * KL, Lm, c1, min(n, c1 + GCH));
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const TF* sl = stg + k * GCH * KL;
        for (int j = c0; j < c1; ++j) {
            const int p = pv[j];
            const TF l = lrow ? sl[(j - c0) * KL + lane - 1] : zero<TF>();
            const TX in = (lane == KL && j + KL + 1 < n) ? b[j + KL + 1] : zero<TX>();
            const TX bj = shfl_idx(w, p);
            const TX w0 = shfl_idx(w, 0);
            if (lane == p) w = w0;
            if (lrow) w = fms_x(l, bj, w);
            if (lane == 0) b[j] = bj;
            w = shfl_down_x(w);
            if (lane == KL) w = in;
        }
        __syncwarp();
    }
    // backward: U x = z, chunks of rows taken from the bottom
    TX v = (lane <= KK && n - 1 - lane >= 0) ? b[n - 1 - lane] : zero<TX>();
    stage_rows<UW>(stg, Uc, max(0, n - GCH), n);
    cp_async_commit();
    for (int c1 = n, k = 0; c1 > 0; c1 -= GCH, k ^= 1) {
        const int c0 = max(0, c1 - GCH);
        if (c0 > 0) stage_rows<UW>(stg + (k ^ 1) * GCH * UW, Uc, max(0, c0 - GCH), c0);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const TF* su = stg + k * GCH * UW;
        for (int i = c1 - 1; i >= c0; --i) {
            const TF u = urow ? su[(i - c0) * UW + lane] : zero<TF>();
            const TX in2 = (lane == KK && i - KK - 1 >= 0) ? b[i - KK - 1] : zero<TX>();
            const TX yi = shfl_idx(v, 0);
            if (lane == 0) x[i] = yi;
            if (urow) v = fms_x(u, yi, v);
            v = shfl_down_x(v);
            if (lane == KK) v = in2;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(NTHREADS_S) k_solve_galerkin(StepParams P, RhsSpec R, DevFactors F, VecSet y_out,
                                                               VecSet mass_out, VecSet imp_out, int want_mass,
                                                               int want_imp) {
    extern __shared__ double2 sm[];
    const int nc = P.nc, m = P.m_lo + blockIdx.x;
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
    const int np = nc - 4, nt = nc - 2;
    SolveSmem s = carve<1>(sm, nc);
    const bool has_u = (m == 0);
    double2 *pf = s.pf[0], *tf = s.tf[0], *px = s.px[0], *tx = s.tx[0], *xp = s.pw[0], *xt = s.tw[0];
    double* xu = reinterpret_cast<double*>(s.pd[0]);
    // after the FP64 solve arrays (over the FP32 refinement arrays of the tau
    // path, unused here): factor staging (2 GCH rows per system) and pivots
    double2* stp = sm + 8 * round8(nc);
    double* stt = reinterpret_cast<double*>(stp + 2 * GCH * 21);
    double* stu = stt + 2 * GCH * 12;
    unsigned char* pvp = reinterpret_cast<unsigned char*>(stu + 2 * GCH * 12);
    unsigned char* pvt = pvp + round8(nc);
    unsigned char* pvu = pvt + round8(nc);
    for (int n = tid; n < nt; n += nth) {
        if (n < np && m > 0) pvp[n] = F.gpPiv[(size_t)m * np + n];
        pvt[n] = F.gtPiv[(size_t)m * nt + n];
        if (has_u) pvu[n] = F.guPiv[n];
    }

    // right-hand side sum_t c_t V_t; the rows of the integrated equations
    // (k >= 4 for Psi, k >= 2 otherwise) times the row scales of the factors
    for (int n = tid; n < nc; n += nth) {
        double2 ap = make_double2(0.0, 0.0), at = make_double2(0.0, 0.0);
        double au = 0.0;
#pragma unroll 4
        for (int t = 0; t < R.nterms; ++t) {
            const double c = R.t[t].c;
            const double2 vp = R.t[t].v.psi[(size_t)m * nc + n];
            const double2 vt = R.t[t].v.th[(size_t)m * nc + n];
            ap.x = fma(c, vp.x, ap.x);
            ap.y = fma(c, vp.y, ap.y);
            at.x = fma(c, vt.x, at.x);
            at.y = fma(c, vt.y, at.y);
            if (has_u) au = fma(c, R.t[t].v.u[n], au);
        }
        pf[n] = (n < 4 || m == 0) ? make_double2(0.0, 0.0) : ap;
        tf[n] = (n < 2) ? make_double2(0.0, 0.0) : cscale(at, F.gtR[(size_t)m * nt + n - 2]);
        if (has_u) s.uf[n] = (n < 2) ? 0.0 : au * F.guR[n - 2];
    }
    __syncthreads();
    const double ic = 1.0 / P.cnorm;  // 1/(C w_k), w_0 = 1/2
    // implicit buoyancy (Section 4): temperature first, then the streamfunction
    // rows with g dt (Ra/Pr)(i m/s_o) C^I theta_new; otherwise all in one pass
    const int npass = P.buoy_imp ? 2 : 1;
    for (int pass = 0; pass < npass; ++pass) {
        const bool do_p = !P.buoy_imp || pass == 1, do_t = !P.buoy_imp || pass == 0;
        if (do_p && m > 0) {
            if (P.buoy_imp) {
                const double cb = F.gdt * P.Ra / P.Pr * (double)m / P.s_o;
                for (int k = 4 + tid; k < nc; k += nth)
                    pf[k] = cadd(pf[k], cmul_i(band_row_c<8>(P.ops.band[OP_C], tx, k, nc), cb));
                __syncthreads();
            }
            for (int k = 4 + tid; k < nc; k += nth) pf[k] = cscale(pf[k], F.gpR[(size_t)m * np + k - 4]);
            __syncthreads();
        }
        if (warp == 0) {
            if (do_p && m > 0)
                warp_band_solve<8, 20, 21>(pf + 4, xp, np, F.gpL + (size_t)m * np * 8,
                                           F.gpU + (size_t)m * np * 21, pvp, stp);
        } else if (warp == 1) {
            if (do_t)
                warp_band_solve<4, 10, 12>(tf + 2, xt, nt, F.gtL + (size_t)m * nt * 4,
                                           F.gtU + (size_t)m * nt * 12, pvt, stt);
        } else if (warp == 2) {
            if (do_t && has_u) warp_band_solve<4, 10, 12>(s.uf + 2, xu, nt, F.guL, F.guU, pvu, stu);
        }
        __syncthreads();
        // x_n = y_n / U_nn
        for (int n = tid; n < nt; n += nth) {
            if (do_p && m > 0 && n < np) xp[n] = mul(F.gpU[((size_t)m * np + n) * 21], xp[n]);
            if (do_t) {
                xt[n] = mul(F.gtU[((size_t)m * nt + n) * 12], xt[n]);
                if (has_u) xu[n] *= F.guU[(size_t)n * 12];
            }
        }
        __syncthreads();
        // expansion to f_hat: Psi_k = sum_i gamma_i^{k-i} x_{k-i}, f_k = x_{k-2} - x_k
        for (int k = tid; k < nc; k += nth) {
            const double h = (k == 0) ? 2.0 * ic : ic;
            if (do_p) {
                double2 a = make_double2(0.0, 0.0);
                if (m > 0) {
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const int n = k - i;
                        if (n >= 0 && n < np) {
                            const double g = __ldg(&F.gam[n * 5 + i]);
                            a.x = fma(g, xp[n].x, a.x);
                            a.y = fma(g, xp[n].y, a.y);
                        }
                    }
                }
                px[k] = cscale(a, h);
            }
            if (do_t) {
                double2 a = (k < nt) ? make_double2(-xt[k].x, -xt[k].y) : make_double2(0.0, 0.0);
                if (k >= 2) a = cadd(a, xt[k - 2]);
                tx[k] = cscale(a, h);
                if (has_u) s.ux[k] = h * (((k >= 2) ? xu[k - 2] : 0.0) - ((k < nt) ? xu[k] : 0.0));
            }
        }
        __syncthreads();
    }

    // store, then mass / implicit operators for later stages
    for (int n = tid; n < nc; n += nth) {
        y_out.psi[(size_t)m * nc + n] = px[n];
        y_out.th[(size_t)m * nc + n] = tx[n];
        if (has_u) y_out.u[n] = s.ux[n];
        if (want_mass || want_imp)
            epilogue_row(P, R, F.gdt, m, n, px, tx, s.ux, mass_out, imp_out, want_mass, want_imp);
    }
}

__global__ void __launch_bounds__(NTHREADS_S) k_apply(StepParams P, VecSet y, VecSet mass_out, VecSet imp_out,
                                                      int want_mass, int want_imp) {
    extern __shared__ double2 sm[];
    const int m = P.m_lo + blockIdx.x;
    const int nc = P.nc;
    double2* xp = sm;
    double2* xt = xp + nc;
    double* xu = reinterpret_cast<double*>(xt + nc);
    for (int n = threadIdx.x; n < nc; n += blockDim.x) {
        xp[n] = (m > 0) ? y.psi[(size_t)m * nc + n] : make_double2(0.0, 0.0);
        xt[n] = y.th[(size_t)m * nc + n];
        if (m == 0) xu[n] = y.u[n];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) apply_row(P, m, k, xp, xt, xu, mass_out, imp_out, want_mass, want_imp);
}

// Sets *flag when any entry of the state (Psi, theta, u_bar and, for
// collocation, omega) is NaN or infinite.
__global__ void k_check_finite(VecSet y, size_t n2, int nu, int* __restrict__ flag) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = y.psi[i], b = y.th[i];
        bad |= !(isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y));
        if (y.w) {
            const double2 c = y.w[i];
            bad |= !(isfinite(c.x) && isfinite(c.y));
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += gridDim.x * blockDim.x) bad |= !isfinite(y.u[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

size_t smem_solve_mb(const StepParams& P, int MB, bool deep = false) {
    return sizeof(double) * solve_smem_doubles(P.nc, MB, deep);
}

}  // namespace


cudaError_t launch_solve(const StepParams& P, const RhsSpec& rhs, const DevFactors& F, VecSet y_out,
                         VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp, cudaStream_t st) {
    if (F.gal) {
        // the FP64 solve arrays (16 round8(nc) doubles), the staging of the factors
        // (double2 x 2 GCH x 21, double x 2 GCH x 12 twice) and 3 pivot rows
        const size_t smg = sizeof(double) * 16 * round8(P.nc) + sizeof(double2) * 2 * GCH * 21 +
                           sizeof(double) * 2 * 2 * GCH * 12 + 3 * round8(P.nc);
        cudaError_t err = cudaFuncSetAttribute(k_solve_galerkin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg);
        if (err != cudaSuccess) return err;
        k_solve_galerkin<<<slab_modes(P), NTHREADS_S, smg, st>>>(P, rhs, F, y_out, mass_out, imp_out, want_mass ? 1 : 0,
                                                      want_imp ? 1 : 0);
        return cudaGetLastError();
    }
    // the systems with FP32-refined temperature solves (N_c > 600): with explicit
    // buoyancy one CTA per system (two per mode, two per SM), else the deep chain
    // prefetch (one CTA per SM by shared memory)
    const bool large = P.nc > 600;
    if (!P.buoy_imp && (P.solve_roles > 0 || (P.solve_roles < 0 && large))) {
        // double-float streamfunction chains: option psi_chain_dd, by default
        // from N_c > 600 (where the roles kernel is the default)
        const bool ddp = F.pBlkDD && (P.psi_dd > 0 || (P.psi_dd < 0 && large));
        const size_t smr = solve_roles_smem_bytes(P.nc, ddp);
        auto kern = ddp ? k_solve_roles<true> : k_solve_roles<false>;
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
        // two CTAs per SM need the largest shared-memory carveout
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
        if (err != cudaSuccess) return err;
        kern<<<2 * slab_modes(P), NTHREADS_S, smr, st>>>(P, rhs, F, y_out, mass_out, imp_out, want_mass ? 1 : 0,
                                                         want_imp ? 1 : 0);
        return cudaGetLastError();
    }
    // one CTA per mode: the deep chain prefetch for the large systems (one CTA per
    // SM); below N_c = 600 double-float streamfunction chains (option
    // psi_chain_dd, by default from N_c > 64 with explicit buoyancy: n_r = 129,
    // 257, 513 solve 47.6 -> 45.4, 87.8 -> 74.2, 335.5 -> 279.3 us; at n_r = 33
    // the conversions cost more than the chains save, 34.5 -> 36.5 us)
    const bool ddp = !large && !P.buoy_imp && F.pBlkDD && (P.psi_dd > 0 || (P.psi_dd < 0 && P.nc > 64));
    auto kern = large ? k_solve<1, true> : (ddp ? k_solve<1, false, true> : k_solve<1, false>);
    const size_t sm = smem_solve_mb(P, 1, large);
    // the epilogue reads the assembled right-hand sides from shared memory where
    // they fit (up to N_c ~ 1300), else sums the terms again
    int dev = 0, smax = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    cudaFuncAttributes fa;
    err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    const size_t smk = sm + sizeof(double) * keep_f_doubles(P.nc);
    const int keep = smk + fa.sharedSizeBytes <= (size_t)smax ? 1 : 0;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(keep ? smk : sm));
    if (err != cudaSuccess) return err;
    kern<<<slab_modes(P), NTHREADS_S, keep ? smk : sm, st>>>(P, rhs, F, y_out, mass_out, imp_out, want_mass ? 1 : 0,
                                                   want_imp ? 1 : 0, keep);
    return cudaGetLastError();
}

// acc[0] += sum_n w_n Re theta_hat_0n = Nu - 1 of the state (one warp, a fixed
// summation order: the lane sums, then a butterfly of shuffles)
__global__ void k_nusselt_accumulate(const double2* __restrict__ th0, const double* __restrict__ w, int nc,
                                     double* acc) {
    double t = 0.0;
    for (int n = threadIdx.x; n < nc; n += 32) t = fma(w[n], th0[n].x, t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) acc[0] += t;
}

cudaError_t launch_nusselt_accumulate(const StepParams& P, VecSet y, const double* w, double* acc,
                                      cudaStream_t st) {
    k_nusselt_accumulate<<<1, 32, 0, st>>>(y.th, w, P.nc, acc);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const StepParams& P, VecSet y, int* flag, cudaStream_t st) {
    k_check_finite<<<152, 256, 0, st>>>(y, (size_t)P.M * P.nc, P.nc, flag);
    return cudaGetLastError();
}

cudaError_t launch_apply(const StepParams& P, VecSet y, VecSet mass_out, VecSet imp_out, bool want_mass,
                         bool want_imp, cudaStream_t st) {
    const size_t sm = sizeof(double2) * 2 * P.nc + sizeof(double) * P.nc;
    cudaError_t err = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_apply<<<slab_modes(P), NTHREADS_S, sm, st>>>(P, y, mass_out, imp_out, want_mass ? 1 : 0, want_imp ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pz
