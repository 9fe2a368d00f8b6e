// Host-side construction of the radial operators of the Chebyshev-integration
// formulation and of the factored tau systems (Sections 3.2 and Appendix A of
// Gastine, pizza, GJI 2019).  Pure C++; no CUDA.
#pragma once
#include <complex>
#include <vector>

namespace pz {

using cplx = std::complex<double>;

struct Geom {
    double eta, s_o, s_i, a, b;   // s = a x + b, a = d/2 with d = s_o - s_i = 1
};
Geom make_geom(double eta);

// Conduction-profile coefficient alpha/ln(eta) (Section 2, below Eq. temp).
double tc_coefficient(double eta);

// Operator ids of pizza_host_operator.
enum OpId { OP_A0 = 0, OP_A2, OP_B0, OP_B2, OP_B4, OP_C, OP_D, OP_F0, OP_F2, OP_EZ, OP_G, OP_COUNT };

// Number of integrations q of an operator and its half bandwidth h.
int op_q(int id);
int op_h(int id);

// Dense n_c x n_c matrix (row-major) acting on the paper's f_hat coefficients of
// an n_r-point grid; rows below q are zero.
std::vector<double> build_operator(int id, int n_r, int n_c, const Geom& g);

// Band storage of an operator: band[k*(2h+1) + (n-k+h)] for |n-k| <= h.
std::vector<double> to_band(const std::vector<double>& dense, int n_c, int h);

// Tau rows acting on f_hat (Eqs. bcs_coll_dirichlet, bcs_coll_neumann,
// bc_d3psi_coll), in the order used by the systems:
//  streamfunction: f(s_o), f(s_i), f'''(s_o), f'(s_i);  Dirichlet: f(s_o), f(s_i).
std::vector<double> tau_rows_psi(int n_r, int n_c);
std::vector<double> tau_rows_dir(int n_r, int n_c);

// Factored bordered system (Appendix A) for p border rows and a banded block
// D of half bandwidth kl = ku = h, factored by LU without pivoting:
//   L[i*h + t] = L(i+1+t, i),  U[i*h + t] = U(i, i+1+t),  invd[i] = 1/U(i,i),
//   Y = D^{-1} C stored [i*p + c] (refined twice with residuals summed in twice the
//   working precision),  Sinv = (A - B Y)^{-1} stored [r*p + c].
template <class T>
struct Bordered {
    int n = 0, p = 0, h = 0;
    std::vector<T> L, U, invd, Y, Sinv;
};

// Block-tridiagonal LU of the banded block D (rows and columns p..n_c-1 of the
// band storage, half width h) with blocks of h rows (nb = ceil(n/h), padding
// rows identity):  D = L U with L unit block-lower-bidiagonal, U block upper
// bidiagonal;  U_kk = D_kk - L_{k,k-1} D_{k-1,k},  L_{k,k-1} = D_{k,k-1} U_{k-1,k-1}^{-1}.
// The diagonal blocks are inverted by Gauss-Jordan with partial pivoting.
//   D x = b  <=>  z_k = b_k - L_{k,k-1} z_{k-1}  (k = 0..nb-1),
//                 x_k = Uinv_k z_k - H_k x_{k+1}  (k = nb-1..0),  H_k = Uinv_k D_{k,k+1}.
// Stored per block k as three row-major h x h matrices [k][0] L_{k,k-1},
// [k][1] Uinv_k, [k][2] H_k.  Returns false if a diagonal block is singular.
template <class T>
bool block_lu(const std::vector<T>& band, int n_c, int h, int p, std::vector<T>& out);

// Two-sided ("twisted") block factorisation of the same block-tridiagonal D,
// meeting at the middle block c = nb/2: the top blocks k < c are factored from
// the top as in block_lu, the bottom blocks k > c from the bottom, and the
// middle block takes both Schur complements.  Stored per block k as three
// row-major h x h matrices:
//   k < c:  [0] L_k = D_{k,k-1} U_{k-1}^{-1}, [1] U_k^{-1}, [2] U_k^{-1} D_{k,k+1}
//   k > c:  [0] M_k = D_{k,k+1} V_{k+1}^{-1}, [1] V_k^{-1}, [2] V_k^{-1} D_{k,k-1}
//   k = c:  [0] L_c, [1] S^{-1}, [2] M_c,  S = D_cc - L_c D_{c-1,c} - M_c D_{c+1,c}
// with U_k = D_kk - L_k D_{k-1,k} and V_k = D_kk - M_k D_{k+1,k}.  Then D x = b by
//   z_k = b_k - L_k z_{k-1} (k < c),  w_k = b_k - M_k w_{k+1} (k > c),
//   x_c = S^{-1}(b_c - L_c z_{c-1} - M_c w_{c+1}),
//   x_k = U_k^{-1} z_k - [2]_k x_{k+1} (k < c),  x_k = V_k^{-1} w_k - [2]_k x_{k-1} (k > c):
// two chains of about nb/2 blocks each instead of one of nb.
template <class T>
bool block_lu_twisted(const std::vector<T>& band, int n_c, int h, int p, std::vector<T>& out);

// Assemble and factor the tau system  [tau rows; Mass - gdt*Lin]  for one m.
// mass_band / lin_band: band storage with half bandwidth h (complex).
template <class T>
bool factor_bordered(const std::vector<T>& mass_lin_band, int n_c, int h,
                     const std::vector<double>& tau, int p, Bordered<T>& out);

// ---------------------------------------------------------------------------
// Galerkin bases (Appendix B).  gamma_0..gamma_4 of the streamfunction basis
// function phi_n = sum_i gamma_i T_{n+i} (gamma_0 = 1), which meets the four
// boundary conditions of the tau rows; the Dirichlet basis is T_{n+2} - T_n.
void galerkin_gamma(int n, double g[5]);

// Banded LU with partial pivoting of an n x n matrix with kl diagonals below and
// ku above, given by rows: band[i*(kl+ku+1) + (c - i + kl)] = G(i, c) for
// i - kl <= c <= i + ku.  The row interchanges stay interleaved with the
// elimination (as in LAPACK's band factorisation): at column j the row j + piv[j]
// (piv[j] in 0..kl) is swapped with row j, then rows j+1..j+kl are eliminated with
// the multipliers Lm[j*kl + t] (row j+1+t); U gains up to kl + ku diagonals above.
// Output per column i of U: Ucol[i*(kl+ku+1)] = 1/U(i,i) and
// Ucol[i*(kl+ku+1) + t] = U(i-t, i)/U(i,i) (t = 1..kl+ku, zero above row 0), i.e.
// the unit upper factor U D^{-1} with x = D^{-1} z', z' = (U D^{-1})^{-1} z.
// Every row is first scaled to unit maximum (rs[i] = 1/max_c |G(i, c)|; the
// right-hand side takes the same scaling).  Returns false on a zero pivot.
template <class T>
bool band_lu_pivot(int n, int kl, int ku, const std::vector<T>& band, std::vector<T>& Lm, std::vector<T>& Ucol,
                   std::vector<unsigned char>& piv, std::vector<double>& rs);

// Solve with band_lu_pivot's factors, in place: b (n entries) <- G^{-1} b.
template <class T>
void band_lu_pivot_solve(int n, int kl, int ku, const std::vector<T>& Lm, const std::vector<T>& Ucol,
                         const std::vector<unsigned char>& piv, const std::vector<double>& rs, T* b);

// ---------------------------------------------------------------------------
// Chebyshev collocation (Section 3.1), fields held as Gauss-Lobatto grid values.
// ---------------------------------------------------------------------------
struct CollGrid {
    int N = 0;
    std::vector<double> s;            // radial grid, s_0 = s_o
    std::vector<double> beta, dbeta;  // beta = -s/h^2 and d beta/ds; 0 at s_o (a boundary row)
    std::vector<double> D1, D2;       // d/ds and d^2/ds^2 of the interpolant, row-major N x N
    std::vector<double> T;            // T[k*N + n] = C w_n T_n(x_k) (Eq. cheb; T T = I, Eq. icheb)
    // Ekman pumping (Eq. pumping_full), empty when off: Upsilon = (s_o/E)^(1/2) h^(-3/2)
    // and c5 = 5 s_o beta/(2 h s), both 0 at s_o (a boundary row)
    std::vector<double> ups, c5;
};
CollGrid coll_grid(int n_r, const Geom& g);
// Fill c.ups and c.c5 for Ekman number E.
void coll_pumping(CollGrid& c, const Geom& g, double E);

// Columns 1..N-2 (the interior right-hand-side rows) of the inverse of the
// vorticity-streamfunction system of mode m >= 1 for implicit weight gdt:
// G[i*(N-2) + j], i < 2N (omega_0..omega_{N-1}, psi_0..psi_{N-1}).  With c.ups set
// the vorticity rows carry the exact Ekman pumping (Eq. psiomcoll's A^C and B^C).
bool coll_inverse_wpsi(const CollGrid& c, double E, int m, double gdt, std::vector<cplx>& G);
// Same for  f - gdt*(kappa*(D2 + D1/s - q/s^2) - Upsilon) f  with Dirichlet rows,
// G[i*(N-2) + j], i < N; the Upsilon term (Eq. uphicoll) only with pump and c.ups set.
bool coll_inverse_dir(const CollGrid& c, double kappa, double q, double gdt, std::vector<double>& G,
                      bool pump = false);

// Inverse of a dense n x n matrix (row-major) by LU with row equilibration,
// partial pivoting and one refinement step (coll_ops.cpp).
bool dense_inverse(int n, const std::vector<cplx>& A, std::vector<cplx>& inv);
bool dense_inverse(int n, const std::vector<double>& A, std::vector<double>& inv);

}  // namespace pz
