// Implicit stage of one IMEX step: right-hand-side assembly (Eqs. multistep1
// and dirks of Section 4) and the bordered banded solve of Appendix A of
// Gastine, pizza, GJI 2019, one CTA per azimuthal mode m.
//
// For each mode the tau system  [tau rows; Mass - gamma dt Lin] y = [0; r]  is
//   (A B; C D)(y1; y2) = (0; h),   D banded (half width 8 for Psi, 4 for theta
//   and u_bar), factored at set-up without pivoting,
//   x = D^{-1} h,  y1 = S^{-1}(0 - B x) with S = A - B D^{-1} C,  y2 = x - Y y1,
//   Y = D^{-1} C precomputed.
// Warp 0 solves Psi_m, warp 1 theta_m, warp 2 u_bar (m = 0).  The epilogue
// applies the banded mass (A^I_m, D^I) and implicit (B^I_m, F^I_m/Pr, E^I)
// operators to the new state for later stages.
#include "device_common.cuh"

namespace pz {

namespace {

constexpr int NTHREADS_S = 128;
constexpr int PF = 8;  // factor rows prefetched ahead by the solving warp

__device__ __forceinline__ double2 mul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 mul(double a, double2 b) { return cscale(b, a); }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
template <class T>
__device__ __forceinline__ T zero();
template <>
__device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ double zero<double>() { return 0.0; }

// Unpivoted banded LU solve by one warp.  x (shared memory) has n entries;
// L[j*H + t] = L(j+1+t, j), U[j*H + t] = U(j, j+1+t), invd[j] = 1/U(j,j).
template <int H, class TF, class TX>
__device__ void warp_band_solve(TX* x, int n, const TF* __restrict__ Lf, const TF* __restrict__ Uf,
                                const TF* __restrict__ invd) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < H;
    // forward: L z = h
    TF cur[PF], nxt[PF];
#pragma unroll
    for (int i = 0; i < PF; ++i) {
        const int j = i;
        cur[i] = (act && j < n) ? Lf[(size_t)j * H + lane] : zero<TF>();
    }
    for (int j0 = 0; j0 < n; j0 += PF) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int j = j0 + PF + i;
            nxt[i] = (act && j < n) ? Lf[(size_t)j * H + lane] : zero<TF>();
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int j = j0 + i;
            if (j < n) {
                const TX z = x[j];
                if (act && j + 1 + lane < n) x[j + 1 + lane] = sub(x[j + 1 + lane], mul(cur[i], z));
                __syncwarp();
            }
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) cur[i] = nxt[i];
    }
    // backward: U x = z  (column oriented)
    TF dcur = zero<TF>(), dnxt = zero<TF>();
    {
        // cur[i] holds U(j-1-lane, j) for j = top - i; lane < PF also holds invd
        const int top = n - 1;
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int j = top - i, r = j - 1 - lane;
            cur[i] = (act && r >= 0) ? Uf[(size_t)r * H + lane] : zero<TF>();
        }
        dcur = (lane < PF && top - lane >= 0) ? invd[top - lane] : zero<TF>();
    }
    for (int j0 = n - 1; j0 >= 0; j0 -= PF) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int j = j0 - PF - i, r = j - 1 - lane;
            nxt[i] = (act && j >= 0 && r >= 0) ? Uf[(size_t)r * H + lane] : zero<TF>();
        }
        {
            const int j = j0 - PF - lane;
            dnxt = (lane < PF && j >= 0) ? invd[j] : zero<TF>();
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int j = j0 - i;
            if (j >= 0) {
                TF di;
                if constexpr (sizeof(TF) == sizeof(double2)) {
                    double2 dd = *reinterpret_cast<double2*>(&dcur);
                    dd.x = __shfl_sync(0xffffffffu, dd.x, i);
                    dd.y = __shfl_sync(0xffffffffu, dd.y, i);
                    di = *reinterpret_cast<TF*>(&dd);
                } else {
                    double dd = *reinterpret_cast<double*>(&dcur);
                    dd = __shfl_sync(0xffffffffu, dd, i);
                    di = *reinterpret_cast<TF*>(&dd);
                }
                const TX xj = mul(di, x[j]);
                __syncwarp();
                if (lane == 0) x[j] = xj;
                if (act && j - 1 - lane >= 0) x[j - 1 - lane] = sub(x[j - 1 - lane], mul(cur[i], xj));
                __syncwarp();
            }
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) cur[i] = nxt[i];
        dcur = dnxt;
    }
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Schur step of Appendix A for one field, by one warp: x holds the full vector of
// length n_c; on entry x[p..] = D^{-1} h; on exit the solution.  B: p x (n_c-p)
// real tau rows; Sinv: p x p; Y: (n_c-p) x p.
template <int PB, class TF>
__device__ void warp_schur(double2* x, int nc, const double* __restrict__ B, const TF* __restrict__ Sinv) {
    const int lane = threadIdx.x & 31;
    const int n = nc - PB;
    double2 t[PB];
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = make_double2(0.0, 0.0);
    for (int j = lane; j < n; j += 32) {
        const double2 xv = x[PB + j];
#pragma unroll
        for (int r = 0; r < PB; ++r) {
            const double b = __ldg(&B[(size_t)r * n + j]);
            t[r].x = fma(b, xv.x, t[r].x);
            t[r].y = fma(b, xv.y, t[r].y);
        }
    }
#pragma unroll
    for (int r = 0; r < PB; ++r) t[r] = warp_sum(t[r]);
    if (lane < PB) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < PB; ++c) acc = csub(acc, mul(Sinv[lane * PB + c], t[c]));
        x[lane] = acc;
    }
    __syncwarp();
}

template <int PB, class TF>
__device__ void block_schur_update(double2* x, int nc, const TF* __restrict__ Y) {
    const int n = nc - PB;
    double2 y1[PB];
#pragma unroll
    for (int c = 0; c < PB; ++c) y1[c] = x[c];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 acc = x[PB + j];
#pragma unroll
        for (int c = 0; c < PB; ++c) acc = csub(acc, mul(Y[(size_t)j * PB + c], y1[c]));
        x[PB + j] = acc;
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

// mass / implicit operators applied to the state held in shared memory
__device__ void apply_epilogue(const StepParams& P, int m, const double2* xp, const double2* xt, const double* xu,
                               VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp) {
    const int nc = P.nc;
    const double mu = (double)m * m;
    const double dm = (double)m;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
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
}

__global__ void __launch_bounds__(NTHREADS_S) k_solve(StepParams P, RhsSpec R, DevFactors F, VecSet y_out,
                                                      VecSet mass_out, VecSet imp_out, int want_mass,
                                                      int want_imp) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
    const int nc = P.nc;
    double2* xp = sm;
    double2* xt = xp + nc;
    double* xu = reinterpret_cast<double*>(xt + nc);
    const int tid = threadIdx.x, warp = tid >> 5;

    // right-hand side: sum_t c_t V_t, tau rows zero
    for (int n = tid; n < nc; n += blockDim.x) {
        double2 ap = make_double2(0.0, 0.0), at = make_double2(0.0, 0.0);
        double au = 0.0;
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
        xp[n] = (n < 4 || m == 0) ? make_double2(0.0, 0.0) : ap;
        xt[n] = (n < 2) ? make_double2(0.0, 0.0) : at;
        if (m == 0) xu[n] = (n < 2) ? 0.0 : au;
    }
    __syncthreads();
    const int np = nc - 4, nt = nc - 2;
    if (warp == 0 && m > 0) {
        warp_band_solve<8>(xp + 4, np, F.pL + (size_t)m * np * 8, F.pU + (size_t)m * np * 8,
                           F.pInvd + (size_t)m * np);
        warp_schur<4>(xp, nc, P.ops.tau_psi_B, F.pSinv + (size_t)m * 16);
    } else if (warp == 1) {
        warp_band_solve<4>(xt + 2, nt, F.tL + (size_t)m * nt * 4, F.tU + (size_t)m * nt * 4,
                           F.tInvd + (size_t)m * nt);
        warp_schur<2>(xt, nc, P.ops.tau_dir_B, F.tSinv + (size_t)m * 4);
    } else if (warp == 2 && m == 0) {
        warp_band_solve<4>(xu + 2, nt, F.uL, F.uU, F.uInvd);
        // real Schur step
        const int lane = tid & 31;
        double t0 = 0.0, t1 = 0.0;
        for (int j = lane; j < nt; j += 32) {
            t0 = fma(__ldg(&P.ops.tau_dir_B[j]), xu[2 + j], t0);
            t1 = fma(__ldg(&P.ops.tau_dir_B[nt + j]), xu[2 + j], t1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        }
        if (lane < 2) xu[lane] = -(F.uSinv[lane * 2] * t0 + F.uSinv[lane * 2 + 1] * t1);
        __syncwarp();
    }
    __syncthreads();
    if (m > 0) block_schur_update<4>(xp, nc, F.pY + (size_t)m * np * 4);
    block_schur_update<2>(xt, nc, F.tY + (size_t)m * nt * 2);
    if (m == 0) {
        const double u0 = xu[0], u1 = xu[1];
        for (int j = tid; j < nt; j += blockDim.x)
            xu[2 + j] -= F.uY[(size_t)j * 2] * u0 + F.uY[(size_t)j * 2 + 1] * u1;
    }
    __syncthreads();
    for (int n = tid; n < nc; n += blockDim.x) {
        y_out.psi[(size_t)m * nc + n] = xp[n];
        y_out.th[(size_t)m * nc + n] = xt[n];
        if (m == 0) y_out.u[n] = xu[n];
    }
    if (want_mass || want_imp) apply_epilogue(P, m, xp, xt, xu, mass_out, imp_out, want_mass, want_imp);
}

__global__ void __launch_bounds__(NTHREADS_S) k_apply(StepParams P, VecSet y, VecSet mass_out, VecSet imp_out,
                                                      int want_mass, int want_imp) {
    extern __shared__ double2 sm[];
    const int m = blockIdx.x;
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
    apply_epilogue(P, m, xp, xt, xu, mass_out, imp_out, want_mass, want_imp);
}

}  // namespace

size_t smem_solve(const StepParams& P) { return sizeof(double2) * 2 * P.nc + sizeof(double) * P.nc; }

cudaError_t launch_solve(const StepParams& P, const RhsSpec& rhs, const DevFactors& F, VecSet y_out,
                         VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp, cudaStream_t st) {
    const size_t sm = smem_solve(P);
    cudaError_t err = cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_solve<<<P.M, NTHREADS_S, sm, st>>>(P, rhs, F, y_out, mass_out, imp_out, want_mass ? 1 : 0,
                                         want_imp ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_apply(const StepParams& P, VecSet y, VecSet mass_out, VecSet imp_out, bool want_mass,
                         bool want_imp, cudaStream_t st) {
    const size_t sm = smem_solve(P);
    cudaError_t err = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_apply<<<P.M, NTHREADS_S, sm, st>>>(P, y, mass_out, imp_out, want_mass ? 1 : 0, want_imp ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pz
