// Internal declarations shared by the CUDA translation units of libpizza.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "host_ops.h"

namespace pz {

constexpr int MAX_PASSES = 16;
constexpr int MAX_RHS_TERMS = 10;

// Mixed-radix (3 * 2^j) Stockham plan for one transform length.
struct FftPlan {
    int L;
    int npass;
    int tws;  // stride of the twiddle table: tw[tws * j] = exp(-2 pi i j / L)
    int radix[MAX_PASSES];   // FP64 and double-float transforms: radix 3, then 4s and 2s
    int npass8;
    int radix8[MAX_PASSES];  // FP32 transforms: radix 3, then 8s, 4s and 2s (fewer passes)
    const double2* tw;  // tw[j] = exp(-2 pi i j / L), j < L
    const float2* twf;  // the same, rounded to FP32 (mixed-precision explicit stage)
    const float4* twdd; // the same as double-float pairs (hi, lo) of (re, im), or null
};

// One set of per-field vectors: Psi and theta complex [M][nc], u real [nc]; the
// collocation formulation adds the vorticity w [M][n_r] (and stores grid values).
struct VecSet {
    double2* psi;
    double2* th;
    double* u;
    double2* w;
};

// Banded m-independent operators (band storage, half width h, row-major [nc][2h+1]).
struct DevOps {
    const double* band[OP_COUNT];
    const double* bandT[OP_COUNT];  // transposed operators in the same band storage (adjoint)
    const double* tau_psi_B;  // 4 x (nc-4): tau rows restricted to columns 4..
    const double* tau_dir_B;  // 2 x (nc-2)
    const double* tau_psi;    // 4 x nc: the full streamfunction tau rows
    const double* tau_dir;    // 2 x nc: the full Dirichlet tau rows
    const float* tau_dir_B32;  // tau_dir_B rounded to FP32 (refined FP32 temperature solves)
};

// Factored bordered systems (Appendix A) for one implicit weight gamma*dt.  The
// banded block is held as a block-tridiagonal LU (host_ops.h, block_lu): per
// block k of H rows three H x H matrices L_{k,k-1}, Uinv_k, H_k.
struct DevFactors {
    double gdt;
    // streamfunction, complex, H = 8: blocks [M][nb_p][3][64], Y [M][n_p][4],
    // Sinv [M][16], assembled rows 4..nc-1 of A^I_m - gamma dt B^I_m [M][n_p][17]
    double2 *pBlk, *pY, *pSinv, *pBand;
    // streamfunction block split in two halves (psplit = 1 when n_p has >= 40
    // blocks; rows [0, n_A), n_A = 8 floor(nb_p/2), and [n_A, n_p)): pBlk then
    // holds each half's two-sided factors, A's blocks first; spikes pSpk
    // [M][n_p][8] (rows < n_A: V = D_A^{-1} E, the coupling of A's last block rows
    // to B's first block columns; rows >= n_A: W = D_B^{-1} F); pRj [M][16][16]
    // the inverse of the interface system [[I, V_last], [W_first, I]]
    int psplit;
    double2 *pSpk, *pRj;
    // the same blocks, spikes and interface inverses as complex double-floats
    // [re.hi, re.lo, im.hi, im.lo] for the double-float chains (option psi_chain_dd)
    float4 *pBlkDD, *pSpkDD, *pRjDD;
    // temperature, real, blocks of H = 8 rows (band half width 4, padded): blocks
    // [M][nb_t][3][64], nb_t = ceil(n_t/8), Y [M][n_t][2], Sinv [M][4],
    // assembled rows 2..nc-1 of D^I - gamma dt F^I_m/Pr [M][n_t][9]
    double *tBlk, *tY, *tSinv, *tBand;
    // zonal flow, real, H = 8: blocks [nb_t][3][64], Y [n_t][2], Sinv [4], band [n_t][9]
    double *uBlk, *uY, *uSinv, *uBand;
    // temperature by mixed-precision iterative refinement (large N_c): ir_t > 0
    // solves with the block factors, Y and S^{-1} rounded to FP32 and corrects
    // ir_t times from FP64 residuals of the assembled system
    int ir_t;
    float *tBlk32, *tY32, *tSinv32;
    // the FP32 temperature block split in two halves for the kernel with one CTA
    // per system (tsplit = 1 from 40 blocks, with ir_t; rows [0, n_tA),
    // n_tA = 8 floor(nb_t/2), and [n_tA, n_t)): tBlk32S each half's factors (A's
    // first), tSpk32 [M][n_t][8] the spikes (V, then W) and tRj32 [M][16][16] the
    // interface inverse, as for the streamfunction
    int tsplit;
    float *tBlk32S, *tSpk32, *tRj32;
    // Galerkin bases (option "radial" = 2, Appendix B): banded LU with partial
    // pivoting of the square integrated systems (host_ops.h, band_lu_pivot).
    // Streamfunction, complex, 8 diagonals below / 12 above: gpL [M][n_p][8],
    // gpU [M][n_p][21], gpPiv [M][n_p], row scales gpR [M][n_p]; temperature, real,
    // 4 / 6: gtL [M][n_t][4], gtU [M][n_t][12] (11 used), gtPiv, gtR; zonal flow
    // guL [n_t][4], guU [n_t][12], guPiv, guR; gam [n_p][5] the coefficients gamma
    int gal;
    double2 *gpL, *gpU;
    double *gpR, *gtL, *gtU, *gtR, *guL, *guU, *guR, *gam;
    unsigned char *gpPiv, *gtPiv, *guPiv;
    // collocation: interior-row columns of the grid-valued inverses, column-major,
    // colW [M][n_r-2][2 n_r] (omega_k, psi_k), colT [M][n_r-2][n_r], colU [n_r-2][n_r]
    double2* colW;
    double *colT, *colU;
};

// Scalar parameters passed by value to every kernel.
// Dense adjoint solves P S^{-H} for the implicit weight of CNAB2, column-major:
// Wp [M][nc][nc-4] complex (streamfunction, rows below its 4 tau rows),
// Wt [M][nc][nc-2], Wu [nc][nc-2] real (temperature, zonal flow).
struct AdjFactors {
    const double2* Wp;
    const double* Wt;
    const double* Wu;
};

struct StepParams {
    int n_r, n_phi, n_m, M, nc, K;   // K = n_r - 1
    double E, Ra, Pr, s_o, inv_a, tc, cnorm, inv_nphi;
    const double* s;      // [n_r] radial grid
    const double* h2;     // [n_r]
    const double* inv_s;  // [n_r]
    const float *s_f, *h2_f, *inv_s_f;  // the same in FP32 (mixed-precision explicit stage)
    const float2 *s_dd, *h2_dd, *inv_s_dd;  // the same as double-floats (hi, lo): lean radial kernels
    FftPlan plan_r;       // length 2K (radial DCT-I as an FFT of the even extension)
    FftPlan plan_h;       // length K, plan_r's twiddles at stride 2 (radial DCT-I, dct1_batched)
    FftPlan plan_p;       // length n_phi (azimuthal)
    DevOps ops;
    // explicit stage in FP32 (option "precision" = mixed): 1 when selected
    int fp32;
    // launch shapes chosen by pizza_autotune (0: the default rule): radial
    // transforms batched per shared-memory pass, threads of the azimuthal kernel
    int nb_r, phi_threads;
    // collocation formulation (Section 3.1): 1 when selected
    int coll;
    const double* beta;   // [n_r] beta = -s/h^2, 0 at s_o
    const double* dbeta;  // [n_r] d beta/ds, 0 at s_o
    const double *cD1, *cD2, *cTm;  // [n_r][n_r] d/ds, d^2/ds^2 on grid values; synthesis matrix
    // Ekman pumping (option "pumping_eps"): 1 when on.  Tables [n_r]:
    //   integration (Eq. approx_pump): pump_ups = Upsilon_eps, pump_cr = 3 s^2/(2 h_eps^2),
    //     pump_ci = 5 s_o/(2 h_eps); pump_F [M][n_r] (the explicit stage's working type)
    //     carries F_eps (m >= 1) and Upsilon_eps u_bar (1 + (E/2) omega_0) (m = 0) from
    //     the synthesis kernel to the analysis kernel
    //   collocation (Eq. pumping_full): pump_ups = Upsilon (0 at s_o), pump_ci =
    //     5 s_o beta/(2 h s) (0 at s_o); pump_cr unused
    int pump;
    const double *pump_ups, *pump_cr, *pump_ci;
    // implicit buoyancy (option "buoy_implicit", Section 4): 1 when the buoyancy
    // term is part of the implicit operator of the streamfunction equation
    int buoy_imp;
    // azimuthal products of the FP64 explicit stage in double-float arithmetic on
    // the FP32 pipe (option "azimuthal_dd"): 1 when selected (plan_p.twdd set)
    int phi_dd;
    double2* pump_F;
    // m-slab decomposition (pizza_set_slab): the per-mode kernels (a1, a3, solve)
    // take modes [m_lo, m_lo + m_n), the per-radius kernel (a2) radii
    // [k_lo, k_lo + k_n); a count of 0 means every mode / radius
    int m_lo, m_n, k_lo, k_n;
    // Courant guard (option "cfl_alpha", Eq. cfl): when cfl_max is set the
    // azimuthal kernel folds max |u_s|/ds_k and max |u_phi|/(s_k dphi) of the
    // synthesised state into cfl_max[0], cfl_max[1] (atomic maxima)
    // the solve with explicit buoyancy in one CTA per system instead of one per
    // mode (option "solve_roles"): 1 always, 0 never, -1 (default) from N_c > 600
    int solve_roles;
    // FP64 radial kernels in the three-array layout (option "radial_lean"):
    // 1 from n_r = 129 (the half-length DCT-I), 0 never, -1 (default) from n_r = 513
    int radial_lean;
    // double-float DCT-I and derivative scans in the lean radial kernels (option
    // "radial_dd"): 1 always, 0 never, -1 (default) from n_r = 513
    int radial_dd;
    // streamfunction block chains of the solve in double-float arithmetic
    // (option "psi_chain_dd", explicit buoyancy): 1 always, 0 never, -1
    // (default) from N_c > 64
    int psi_dd;
    double* cfl_max;
    const double* cfl_ds;  // [n_r] local Gauss-Lobatto spacing
    double cfl_dphi;       // 2 pi / n_phi
};

__host__ __device__ inline int slab_modes(const StepParams& P) { return P.m_n > 0 ? P.m_n : P.M; }
__host__ __device__ inline int slab_radii(const StepParams& P) { return P.k_n > 0 ? P.k_n : P.n_r; }

struct RhsTerm {
    VecSet v;
    double c;
};

struct RhsSpec {
    int nterms;
    RhsTerm t[MAX_RHS_TERMS];
};

// kernel launchers (k_explicit.cu, k_implicit.cu)
cudaError_t launch_spec_to_grid(const StepParams& P, VecSet y, double2* G1, cudaStream_t st);
cudaError_t launch_phi_products(const StepParams& P, const double2* G1, double2* G2, cudaStream_t st);
cudaError_t launch_grid_to_spec(const StepParams& P, const double2* G2, VecSet y, VecSet e, cudaStream_t st);
cudaError_t launch_solve(const StepParams& P, const RhsSpec& rhs, const DevFactors& F, VecSet y_out,
                         VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp, cudaStream_t st);
cudaError_t launch_apply(const StepParams& P, VecSet y, VecSet mass_out, VecSet imp_out, bool want_mass,
                         bool want_imp, cudaStream_t st);
cudaError_t launch_check_finite(const StepParams& P, VecSet y, int* flag, cudaStream_t st);
cudaError_t launch_nusselt_accumulate(const StepParams& P, VecSet y, const double* w, double* acc,
                                      cudaStream_t st);
cudaError_t launch_coll_spec_to_grid(const StepParams& P, VecSet y, double2* G1, cudaStream_t st);
cudaError_t launch_coll_grid_rows(const StepParams& P, const double2* G1, const double2* G2, VecSet e,
                                  cudaStream_t st);
cudaError_t launch_coll_solve(const StepParams& P, const RhsSpec& R, const DevFactors& F, VecSet y_out,
                              VecSet mass_out, VecSet imp_out, bool want_mass, bool want_imp, cudaStream_t st);
cudaError_t launch_coll_apply(const StepParams& P, VecSet y, VecSet imp_out, cudaStream_t st);
cudaError_t launch_coll_from_hat(const StepParams& P, VecSet hat, VecSet y, cudaStream_t st);
cudaError_t launch_coll_to_hat(const StepParams& P, VecSet y, VecSet out, cudaStream_t st);
cudaError_t launch_phi_fields(const StepParams& P, const double2* G1, double* us, double* uphi, double* omega,
                              double* theta, cudaStream_t st);
cudaError_t launch_adj_explicit(const StepParams& P, VecSet w, VecSet y, VecSet lam, const double2* G1, double2* Gb2,
                                double2* Gb1, double* ra, cudaStream_t st);
cudaError_t launch_adj_solve(const StepParams& P, const AdjFactors& A, VecSet lam, VecSet rho, cudaStream_t st);
cudaError_t launch_adj_apply(const StepParams& P, VecSet g, VecSet rho, VecSet rho_next, VecSet lam, VecSet w,
                             double dt, double c, double c2, cudaStream_t st);
cudaError_t launch_vec_add(const StepParams& P, VecSet a, VecSet b, cudaStream_t st);
// *acc += sum_m ra[m] (m < M, a fixed summation order), one warp
cudaError_t launch_ra_accumulate(const double* ra, int M, double* acc, cudaStream_t st);
cudaError_t launch_diagnostics(const StepParams& P, const double2* G1, const double* q, double* mode_sums,
                               double* radius_max, cudaStream_t st);

// message returned by pizza_last_error(NULL)
void set_global_error(const char* msg);

// Stockham radix plan (3 * 2^j or 2^j) and twiddle table exp(-2 pi i j/L), j < L.
bool make_fft_plan(int L, FftPlan& pl);
std::vector<double2> fft_twiddles(int L);

size_t smem_spec_to_grid(const StepParams& P);
size_t smem_adj_grid_to_spec(const StepParams& P);
size_t smem_adj_spec_to_grid(const StepParams& P);
size_t smem_phi_products(const StepParams& P);
size_t smem_grid_to_spec(const StepParams& P);
size_t smem_coll_spec_to_grid(const StepParams& P);
size_t smem_coll_grid_rows(const StepParams& P);

}  // namespace pz
