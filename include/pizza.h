/*
 * pizza.h -- C interface of a GB300 (sm_103a) implementation of one IMEX time
 * step of the pseudo-spectral 2-D spherical quasi-geostrophic convection model
 * of Gastine, "pizza: an open-source pseudo-spectral code for spherical
 * quasi-geostrophic convection" (GJI 2019).
 *
 * The library owns all device memory it allocates; callers pass plain pointers
 * and sizes.  Every call returns a status code (enum pizza_status); no call
 * aborts the process.  A failing call leaves a message for pizza_last_error().
 *
 * Problem and notation (Section 2 of the paper):
 *   annulus s_i <= s <= s_o with gap d = s_o - s_i = 1, radius ratio eta = s_i/s_o,
 *   Ekman number E, Rayleigh number Ra, Prandtl number Pr; unknowns are the
 *   temperature perturbation theta, the regularised streamfunction Psi of the
 *   Chebyshev-integration method (Section 3.2: u_s = (h^2/s) dPsi/dphi,
 *   u_phi = u_bar - h^2 dPsi/ds + 3 s Psi, h^2 = s_o^2 - s^2) and the
 *   axisymmetric zonal flow u_bar.  No-slip, fixed-temperature walls; Ekman
 *   pumping off.
 *
 * Discretisation (Section 3): n_phi azimuthal points with N_m = n_phi/3
 * retained wavenumbers m = 0..N_m (Eqs. fft, ifft); n_r Gauss-Lobatto radial
 * points x_k = cos(pi k/(n_r-1)), k = 0..n_r-1 (k = 0 is the outer wall s_o);
 * N_c Chebyshev coefficients per mode, N_c = floor(2 (n_r-1)/3) for the
 * integration method (Eq. psi_int and the dealiasing rule below Eq. temp_int).
 *
 * Chebyshev-collocation formulation (Section 3.1; option "radial" = 0): the
 * unknowns are the vorticity omega and the streamfunction psi itself
 * (u_s = (1/s) dpsi/dphi, u_phi = u_bar - dpsi/ds - beta psi, beta = -s/h^2,
 * Eq. vel_def), theta and u_bar, with N_c = n_r coefficients; the equations are
 * imposed at the interior Gauss-Lobatto points (Eqs. psiomcoll, uphicoll,
 * tempcoll) and the boundary conditions at the walls (Eqs. bcs_coll_dirichlet,
 * bcs_coll_neumann).  The per-mode systems are dense; their inverses restricted
 * to the interior right-hand-side rows are built on the host (LU with partial
 * pivoting and one refinement step, O(n_r^3) per mode and implicit weight) and
 * kept on the device (2 n_r (n_r-2) complex + n_r (n_r-2) real per mode).
 *
 * Spectral coefficient convention (Eq. cheb): f_m(s_k) = C sum''_{n<N_c}
 * f_hat_{mn} T_n(x_k), C = sqrt(2/(n_r-1)), the double prime halving the n = 0
 * term (and the n = n_r-1 term when present).  Complex arrays are interleaved
 * (re, im) doubles with layout [m][n], m = 0..N_m, n = 0..N_c-1 (row-major).
 */
#ifndef PIZZA_H
#define PIZZA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pizza_ctx pizza_ctx;

/* Time schemes (Section 4, Table 1; Eqs. multistep1 and dirks).  The multistep
 * schemes start with lower-order steps: CNAB2 uses bE = (1) on its first step,
 * SBDF3 one SBDF1 and one SBDF2 step, SBDF2 one SBDF1 step.  ARS443 is the
 * third-order stiffly accurate SDIRK of Ascher, Ruuth & Spiteri (1997);
 * BPR353 the third-order stiffly accurate SDIRK of Boscarino, Pareschi & Russo
 * (2013), Table 1's preferred third-order scheme: five implicit and three
 * explicit terms per step (one explicit evaluation fewer than ARS443), its
 * stages using the implicit term of y_n. */
enum pizza_scheme { PIZZA_CNAB2 = 0, PIZZA_SBDF2 = 1, PIZZA_SBDF3 = 2, PIZZA_ARS443 = 3, PIZZA_BPR353 = 4 };

enum pizza_status {
    PIZZA_OK = 0,
    PIZZA_EINVAL = -1,      /* invalid argument or size                          */
    PIZZA_ENOMEM = -2,      /* device or host allocation failed                  */
    PIZZA_ECUDA = -3,       /* a CUDA runtime call failed (message has details)  */
    PIZZA_ENONFINITE = -4,  /* a NaN/Inf in the state (pizza_diagnostics; with
                               option "check_finite" pizza_synchronize)       */
    PIZZA_ECFL = -5,        /* Courant criterion of Eq. cfl exceeded (cfl_alpha) */
    PIZZA_ETIMEOUT = -6,    /* reserved: a bounded device wait gave up           */
    PIZZA_ESTATE = -7,      /* call out of order (e.g. step before dt is set)    */
    PIZZA_EUNSUPPORTED = -8 /* valid request the library does not implement      */
};

/* Create a context.  Validation: n_r >= 9 with n_r - 1 a power of two (the
 * radial transform is a DCT-I evaluated by a 2(n_r-1)-point FFT); n_phi a
 * multiple of 3 of the form 3*2^j or 2^j, n_phi >= 12; 0 < radius_ratio < 1;
 * E, Pr > 0; scheme one of enum pizza_scheme.  Allocates the device state for
 * the integration/tau formulation on the current CUDA device.  *out receives
 * the context (NULL on failure).  The time step must be set with
 * pizza_set_option(ctx, "dt", value) before pizza_step. */
int pizza_init(pizza_ctx **out, int n_r, int n_phi, double E, double Ra,
               double Pr, double radius_ratio, int scheme);

/* Set a numeric option.  Keys:
 *   "dt"     time step > 0; invalidates the factored implicit operators, which
 *            are rebuilt on the next step;
 *   "radial" 1 = Chebyshev integration with tau rows (Section 3.2, the default),
 *            2 = Chebyshev integration solved in Galerkin bases (Appendix B: the
 *            streamfunction in phi_n = sum_i gamma_i^n T_{n+i}, temperature and
 *            zonal flow in T_{n+2} - T_n; the square integrated systems, 8 and 12
 *            diagonals below and above for Psi, 4 and 6 otherwise, by banded LU
 *            with partial pivoting; the same discrete solution as 1),
 *            0 = Chebyshev collocation (Section 3.1; n_r <= PIZZA_COLL_MAX_NR,
 *            else PIZZA_EUNSUPPORTED).  Changing between 1 and 2 discards the
 *            factored operators and keeps the state; changing to or from 0 also
 *            resets the state to zero and N_c to the new formulation's value; any
 *            other value returns PIZZA_EUNSUPPORTED;
 *   "precision" 0 = FP64 throughout (default); 1 = mixed: the explicit stage
 *            (Chebyshev and Fourier transforms, grid products, flux divergences)
 *            in FP32 on FP32 grid arrays, while the state, the time-scheme
 *            history, the linear buoyancy and conduction couplings, the banded
 *            operators, the boundary rows and the solves stay FP64.  Integration
 *            formulation only (PIZZA_EUNSUPPORTED with collocation);
 *   "pumping_eps" Ekman pumping, 0 = off (default), eps in (0, 1] = on.
 *            Integration formulation: the approximate pumping F_eps of
 *            Eq. approx_pump (Section 3.2, h_eps = ((s_o + eps)^2 - s^2)^(1/2),
 *            Upsilon_eps = (s_o/E)^(1/2) h_eps^(-3/2)), evaluated with the
 *            explicit terms on the radial grid and entering the integrated
 *            streamfunction equation as -F_eps (Eq. psiint), plus Upsilon_eps u_bar
 *            in the zonal-flow equation (Eq. uphi_int).  Collocation: the exact
 *            pumping of Eq. pumping_full and the -Upsilon u_bar of Eq. uphi,
 *            implicit in the factored operators (eps only switches it on).  Both
 *            add the explicit zonal-wind self-interaction (E/2) Upsilon u_bar
 *            omega_0 of Eq. uphicoll.  Set before stepping; changing it discards
 *            the factored operators.  While a tape is recorded: PIZZA_ESTATE;
 *            pizza_tape_begin with pumping on: PIZZA_EUNSUPPORTED;
 *   "buoy_implicit" 0 = buoyancy explicit (default), 1 = the buoyancy term in
 *            the implicit operator (Section 4): (Ra/Pr)(i m/s_o) C^I theta of
 *            Eq. psi_int, or -(Ra/Pr)(i m/s_o) theta on the vorticity rows of
 *            Eq. psiomcoll; each stage solves the temperature first and carries
 *            its buoyancy into the streamfunction (vorticity) system.  The adjoint
 *            refuses it.  Set before stepping;
 *   "azimuthal_dd" 1 (default) = the azimuthal transforms and grid products of
 *            the FP64 explicit stage in double-float arithmetic (pairs of floats,
 *            ~48-bit significands, on the FP32 pipe), their m = 0 modes in FP64;
 *            0 = in FP64.  Both meet the FP64 parity bars of the explicit terms.
 *            The adjoint's azimuthal stage is FP64 either way;
 *   "check_finite" 1 = after every step a small kernel scans the state for NaN
 *            or infinite values and sets a device flag; pizza_synchronize then
 *            returns PIZZA_ENONFINITE (cleared by pizza_set_state).  0 (default) =
 *            no scan; pizza_diagnostics reports a non-finite state either way;
 *   "cfl_alpha" alpha > 0 = the Courant guard of Eq. cfl (Section 4; Table 1
 *            lists each scheme's largest stable alpha): the azimuthal kernel of
 *            every explicit evaluation folds max |u_s|/ds_k and
 *            max |u_phi|/(s_k dphi) over its radii into two running maxima (ds_k
 *            the local Gauss-Lobatto spacing, dphi = 2 pi/n_phi; the rates of
 *            pizza_diagnostics), and pizza_synchronize returns PIZZA_ECFL when
 *            dt > alpha / max(rate) for a state evaluated since the previous
 *            pizza_synchronize, then clears the maxima.  0 (default) = off;
 *            negative: PIZZA_EINVAL;
 *   "radial_lean" the FP64 synthesis and analysis kernels in the layout of
 *            three shared arrays of n_r values, the fields one after another (two
 *            CTAs per SM at n_r = 2049) instead of the batched layout: 1 from
 *            n_r = 129, 0 never, -1 (default) from n_r = 513.  Results agree to
 *            rounding (the DCT-I sums in another order).  In mixed precision
 *            ("precision" = 1) the FP32 kernels take this layout only with 1
 *            (three CTAs per SM; faster at n_r = 2049, but the half-length DCT-I
 *            accumulates the FP32 rounding of its outputs: about 20x the
 *            batched layout's distance from FP64, still within the mixed bar);
 *   "radial_dd" the DCT-I, the Chebyshev derivative scans and the field
 *            arithmetic at each radius of the lean radial kernels in
 *            double-float arithmetic on the FP32 pipe (about 48 significant bits;
 *            stored values, banded applies and couplings in FP64): 1 always
 *            (with the lean layout), 0 never, -1
 *            (default) with the lean layout's default, from n_r = 513.  Results
 *            agree with the FP64 transforms to well within the explicit terms'
 *            FP64 bar, not bitwise;
 *   "solve_roles" with explicit buoyancy, the implicit solve in one CTA per
 *            system (streamfunction; temperature, then the zonal flow for m = 0)
 *            instead of one per mode: 1 always, 0 never, -1 (default) from
 *            N_c > 600, where it fits two CTAs per SM.  The same operations
 *            but for the order of the Schur steps' sums (the whole CTA against
 *            one warp): results agree to the accuracy of the refined solve;
 *   "psi_chain_dd" the block chains of the streamfunction solve (Appendix
 *            A's banded block) in double-float arithmetic on the FP32 pipe
 *            (about 48 significant bits; the Schur step, residual and refinement
 *            stay FP64), explicit buoyancy: 1 always, 0 never (FP64 chains), -1
 *            (default) from N_c > 64 (at N_c <= 64 the conversions cost more
 *            than the shorter chains save).  Results agree with the FP64 chains
 *            to the accuracy of the refined solve, not bitwise;
 *   "theta_fp32" the temperature systems solved by FP32 block chains and two
 *            corrections from FP64 residuals (the zonal flow then refined once
 *            in FP64): 1 always, 0 never (one FP64 solve), -1 (default) from
 *            N_c > 600, where the FP64 solve alone loses digits.  Changing it
 *            drops the factored operators (rebuilt at the next step);
 *   "radial_batch" radial transforms batched per shared-memory pass in the
 *            per-mode explicit kernels: 1, 2 or 4, 0 = the default rule (up to
 *            n_r = 513: 4 in FP64, 2 in mixed precision; else 1); "phi_threads" threads of the per-radius azimuthal
 *            kernel: 128, 256 or 512 (at most 12 points per thread), 0 = default.
 *            Launch shapes only (pizza_autotune picks them by timing): results
 *            are bitwise the same.
 * Returns PIZZA_EINVAL for an unknown key or an invalid value. */
#define PIZZA_COLL_MAX_NR 513
int pizza_set_option(pizza_ctx *ctx, const char *key, double value);

/* Use the given cudaStream_t (passed as void*) for all later device work of
 * this context; NULL selects the context's own stream. */
int pizza_set_stream(pizza_ctx *ctx, void *stream);

/* Report the sizes: n_r, n_phi, N_m = n_phi/3 and N_c.  Any pointer may be NULL. */
int pizza_get_sizes(const pizza_ctx *ctx, int *n_r, int *n_phi, int *n_m, int *n_c);

/* Copy a state in.  theta_hat and psi_hat: complex [N_m+1][nc_in]; uphi0_hat:
 * real [nc_in] (the m = 0 zonal flow).  nc_in <= N_c; missing coefficients are
 * zero; psi_hat of m = 0 is ignored (Psi_0 = 0).  Pointers may be host or
 * device memory (detected); the data are copied and not retained.  Resets the
 * time-scheme history (the next step is a start-up step).
 * Collocation: psi_hat holds the coefficients of psi (not Psi); the vorticity
 * is set to omega = -L_beta psi (Eq. psi) at every grid point, with its limit
 * -(5/4) d^2psi/ds^2 at s_o. */
int pizza_set_state(pizza_ctx *ctx, const double *theta_hat, const double *psi_hat,
                    const double *uphi0_hat, int nc_in);

/* Copy the current state out (layouts as in pizza_set_state with nc_in = N_c).
 * Host or device destination pointers; any may be NULL to skip that field.
 * Synchronises the context stream.  (Collocation: the vorticity, whose wall
 * values are unknowns of their own, is reported by pizza_get_grid.) */
int pizza_get_state(pizza_ctx *ctx, double *theta_hat, double *psi_hat, double *uphi0_hat);

/* Advance nsteps time steps (Sections 3.2 and 4): per explicit evaluation the
 * spectral-to-grid transforms, the grid products and forward transforms, then
 * per implicit stage the right-hand-side assembly and the bordered banded solve
 * of Appendix A.  Work is queued on the context stream; the call returns
 * without waiting.  Returns PIZZA_ESTATE if dt is unset. */
int pizza_step(pizza_ctx *ctx, int nsteps);

/* Evaluate the integrated explicit right-hand sides of the current state (the
 * bracketed terms of Eqs. psi_int and temp_int after C^I and D^I, and of
 * Eq. uphi_int after D^I): e_psi, e_theta complex [N_m+1][N_c], e_uphi real
 * [N_c]; rows n < 4 (psi) and n < 2 (theta, u) are zero.  Host or device
 * destinations.  Synchronises the context stream.
 * Collocation: the explicit parts of Eqs. psiomcoll, tempcoll and uphicoll at
 * the grid points instead, [N_m+1][n_r] (the vorticity rows into e_psi), with
 * the boundary rows k = 0 and n_r-1 zero. */
int pizza_explicit_terms(pizza_ctx *ctx, double *e_psi, double *e_theta, double *e_uphi);

/* Diagnostics of the current state (Section 6.2; Eq. cfl).  <f> is the
 * annulus integral int int f s ds dphi, radial integrals by Clenshaw-Curtis
 * quadrature on the Gauss-Lobatto points.
 *   E_K = <u_s^2 + u_phi^2>/2, E_Z = <u_bar^2>/2, enstrophy = <omega^2>,
 *   Re = sqrt(2 E_K/(pi (s_o^2 - s_i^2))), Ro = Re E,
 *   Nu = 1 + (d theta_0/ds)(s_o) / (dT_c/ds)(s_o)   (heat flux through the outer
 *        wall relative to conduction; the paper defines no Nusselt number),
 *   cfl_s = max |u_s|/ds_k, cfl_phi = max |u_phi|/(s_k dphi) over the physical
 *        grid (ds_k the local Gauss-Lobatto spacing, dphi = 2 pi/n_phi); the
 *        Courant condition of Eq. cfl reads dt <= alpha / max(cfl_s, cfl_phi).
 * Uses the context's work buffers; synchronises the context stream. */
typedef struct pizza_diag {
    double E_K, E_Z, enstrophy, Nu, Re, Ro, cfl_s, cfl_phi;
} pizza_diag;
int pizza_diagnostics(pizza_ctx *ctx, pizza_diag *out);

/* Physical-grid values of the current state (Eq. fft): u_s, u_phi, omega and
 * theta at (s_k, phi_j = 2 pi j/n_phi), each real [n_r][n_phi] (row-major).
 * Host or device destinations; any may be NULL.  Uses the context's work
 * buffers (allocating a 32 n_r n_phi byte staging buffer on the first call);
 * synchronises the context stream. */
int pizza_get_grid(pizza_ctx *ctx, double *us, double *uphi, double *omega, double *theta);

/* Discrete adjoint of CNAB2 runs (integration formulation, FP64, n_phi <= 3072,
 * n_r <= 1025; PIZZA_EUNSUPPORTED otherwise), for gradients of J = sum_{n=1..K} j_n(y_n) of
 * the states y_n = (Psi_hat, theta_hat, u_hat) after n steps.  The forward step
 * (Eq. multistep1 with the start-up rule) is
 *   y_{n+1} = S^{-1} P r_n,  r_0 = A y_0 + dt E(y_0),
 *   r_n = A y_n + dt (3/2 E(y_n) - 1/2 E(y_{n-1})),
 * A = Mass + (dt/2) Lin, S the tau system of weight dt/2 (Section 3.2) and P the
 * projection zeroing its tau rows, E the explicit terms.  With the inner product
 * <a, b> = Re sum conj(a) b over the stored arrays, the reverse sweep is
 *   rho_n = P S^{-H} lambda_{n+1},
 *   lambda_n = g_n + A^H rho_n + J_E(y_n)* w_n,  w_n = dt (c_n rho_n - 1/2 rho_{n+1}),
 * c_0 = 1, c_n = 3/2, rho_K = 0, g_n = dj_n/dy_n; dJ/dRa = sum_n < w_n, dE/dRa(y_n) >.
 *
 * pizza_tape_begin: start recording, right after pizza_set_state (n = 0); the
 * following pizza_step calls store a checkpoint (y_n, E(y_{n-1})) every
 * checkpoint_every steps.  The dense adjoint solves are built on the host the
 * first time (O(N_c^3) per mode).
 * pizza_adjoint_step: reverse one recorded step.  The k-th call (k = 1..K) takes
 * g_{K-k+1} (theta and Psi complex [N_m+1][N_c], u real [N_c]; host or device; NULL
 * = zero) and leaves lambda_{K-k} without its own g; the states needed are
 * recomputed segment by segment from the checkpoints (which overwrites the
 * forward state of the context).  *dJ_dRa (may be NULL) receives the running total
 * of the Ra derivative (accumulated on the device); with dJ_dRa NULL the call only
 * enqueues work on the context's stream, otherwise it waits for it.  PIZZA_ESTATE
 * when no recorded step is left.
 * pizza_get_adjoint: copy lambda (after K calls: dJ/dy_0) out.
 * pizza_explicit_adjoint: J_E(y)* applied to (e_psi_bar, e_theta_bar, e_u_bar) at
 * the current state, without the tape (verification). */
int pizza_tape_begin(pizza_ctx *ctx, int checkpoint_every);
int pizza_adjoint_step(pizza_ctx *ctx, const double *g_theta, const double *g_psi, const double *g_u,
                       double *dJ_dRa);
int pizza_get_adjoint(pizza_ctx *ctx, double *theta_bar, double *psi_bar, double *uphi0_bar);
int pizza_explicit_adjoint(pizza_ctx *ctx, const double *e_psi_bar, const double *e_theta_bar,
                           const double *e_u_bar, double *psi_bar, double *theta_bar, double *uphi0_bar);

/* Weights w[n] (N_c reals) of the Nusselt number of the integration state:
 * Nu - 1 = (d theta_0/ds)(s_o)/(dT_c/ds)(s_o) = sum_n w_n Re theta_hat_0n (the
 * definition used by pizza_diagnostics; the paper defines no Nusselt number).
 * PIZZA_EUNSUPPORTED for the collocation formulation. */
int pizza_nusselt_weights(const pizza_ctx *ctx, double *w);

/* Running sum of Nu - 1 on the device: after pizza_nusselt_begin every completed
 * step adds sum_n w_n Re theta_hat_0n of its new state to a device accumulator
 * (a one-warp kernel on the context's stream, fixed summation order); then
 * pizza_nusselt_end synchronises the stream and writes the sum and the number
 * of steps it covers (steps may be NULL).  The time average of the objective of
 * the adjoint, J = (1/K) sum_{n=1..K} (Nu_n - 1), without a state copy per step.
 * PIZZA_EUNSUPPORTED for collocation and slab contexts; pizza_nusselt_end
 * without begin: PIZZA_ESTATE. */
int pizza_nusselt_begin(pizza_ctx *ctx);
int pizza_nusselt_end(pizza_ctx *ctx, double *sum, int *steps);

/* Autotuner: times the explicit stage of the context (on its current state)
 * for each launch shape the device allows -- radial transforms batched one, two
 * or four per shared-memory pass, 128/256/512 threads in the azimuthal kernel --
 * and, with explicit buoyancy and tau rows, the implicit solve with one CTA per
 * mode and with one per system (option "solve_roles"), and keeps the fastest
 * for later steps.  The launch shapes change the schedule, not the arithmetic
 * (bitwise the same results); the solve arrangement changes the order of the
 * Schur steps' sums, so results agree to the accuracy of the refined solve.
 * *nb_r and *phi_threads (may be NULL) receive the
 * explicit-stage choice.  Integration formulation only; builds the factored
 * operators if the context has not stepped yet. */
int pizza_autotune(pizza_ctx *ctx, int *nb_r, int *phi_threads);

/* Batches of independent contexts (any sizes, parameters and schemes) advanced
 * by one CUDA graph: pizza_batch_step captures the nsteps steps of every context,
 * each on its own stream forked from the batch's stream, instantiates the graph
 * once and launches it; a later call with the same nsteps relaunches it when every
 * context is back in the slot state the graph started from (e.g. after
 * pizza_set_state, or a whole number of ring periods later) and no option of any
 * context has been set since the capture, else recaptures.
 * Factors are built before the capture.  The call returns without waiting; work
 * later queued on a context's stream is ordered after the graph.  The contexts must
 * outlive the batch and must not record an adjoint tape.  Errors go to
 * pizza_last_error(NULL). */
typedef struct pizza_batch pizza_batch;
int pizza_batch_create(pizza_batch **out, pizza_ctx *const *ctxs, int n);
int pizza_batch_step(pizza_batch *b, int nsteps);
void *pizza_batch_stream(pizza_batch *b);  /* the cudaStream_t the graph is launched on */
void pizza_batch_free(pizza_batch *b);

/* Per-kernel timing.  pizza_profile_begin starts recording a CUDA event pair on
 * the context stream around every later launch of the kernels selected by mask
 * (bit 0 spectral-to-grid, bit 1 azimuthal products, bit 2 grid-to-spectral,
 * bit 3 implicit solve).  pizza_profile_end synchronises the stream, writes the
 * summed device time in milliseconds and the launch count of each of the four
 * kernels into total_ms[4] and launches[4] (either may be NULL) and stops
 * recording. */
int pizza_profile_begin(pizza_ctx *ctx, unsigned mask);
int pizza_profile_end(pizza_ctx *ctx, double *total_ms, int *launches);

/* Block until all queued work of the context is done; returns the first
 * deferred CUDA error, if any, then PIZZA_ENONFINITE (option "check_finite")
 * or PIZZA_ECFL (option "cfl_alpha") when the steps since the last call
 * tripped those checks. */
int pizza_synchronize(pizza_ctx *ctx);

/* Host-side operator construction, exposed for verification without a GPU.
 * which: 0 A0, 1 A2 (A^I_m = A0 + m^2 A2), 2 B0, 3 B2, 4 B4 (B^I_m = B0 + m^2 B2
 * + m^4 B4 + i m (2/E) C^I), 5 C^I, 6 D^I, 7 F0, 8 F2 (F^I_m = F0 + m^2 F2),
 * 9 E^I, 10 G^I = int^2 h^2.  Writes the dense n_c x n_c matrix (row-major,
 * acting on f_hat coefficients of an n_r-point grid; rows below the number of
 * integrations are zero) into out.  Needs no CUDA device. */
int pizza_host_operator(int which, int n_r, int n_c, double radius_ratio, double *out);

/* Host-side collocation set-up (Section 3.1), exposed for verification without a
 * GPU.  Grid values x_k = cos(pi k/(n_r-1)), s_k = ((s_o - s_i)/2) x_k + (s_o + s_i)/2.
 *   which 0: interior-row columns of the inverse of the vorticity-streamfunction
 *            system of mode m (Eq. psiomcoll with the boundary rows of
 *            Eqs. bcs_coll_dirichlet, bcs_coll_neumann; unknowns the grid values
 *            omega_k, psi_k) for implicit weight gdt: complex, row-major
 *            [2 n_r][n_r - 2] (interleaved re, im);
 *   which 1: the same for theta - gdt (1/Pr)(D2 + D1/s - m^2/s^2) theta with
 *            Dirichlet rows (Eq. tempcoll): real [n_r][n_r - 2];
 *   which 2: the zonal flow u - gdt (D2 + D1/s - 1/s^2) u (Eq. uphicoll):
 *            real [n_r][n_r - 2] (m, Pr unused);
 *   which 3, 4: the differentiation matrices d/ds, d^2/ds^2 on grid values,
 *            real [n_r][n_r].
 * Needs no CUDA device.  PIZZA_EINVAL for invalid arguments or a singular system. */
int pizza_host_collocation(int which, int n_r, double radius_ratio, double E, double Pr, int m,
                           double gdt, double *out);

/* Explicit stage without device allocation.  This entry point has no
 * counterpart in the paper; it exists for callers that cannot allocate device
 * memory themselves or through the library -- for example code running inside a
 * host application that owns the device-memory budget and hands out only
 * preallocated arrays, or latency-critical code that must not enter the CUDA
 * allocator (which can synchronise the device) after start-up.
 *
 * Computes the same e_psi, e_theta, e_uphi as pizza_explicit_terms, for the state
 * psi_hat, theta_hat (complex [N_m+1][N_c]) and uphi0_hat (real [N_c]), where
 * N_m = n_phi/3 and N_c = floor(2 (n_r-1)/3).  All six arrays are DEVICE memory
 * owned by the caller; work is queued on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) and the call returns without waiting.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Its intermediate arrays and read-only tables live in static device arrays
 * compiled into the library (about 8.7 MB, held by every device that loads the
 * library until the process exits), so the sizes are limited to
 * n_r <= PIZZA_NOALLOC_MAX_NR and n_phi <= PIZZA_NOALLOC_MAX_NPHI; larger sizes
 * return PIZZA_EINVAL with a message.  The first call on a device, and any
 * call whose (n_r, n_phi, radius_ratio) differ from the previous one on that
 * device, does a synchronous set-up: the address look-up of the static arrays
 * (first call only) and the table upload, which first waits for the whole
 * device (cudaDeviceSynchronize) so that no call queued earlier still reads the
 * old tables, then copies on `stream` and waits for it.  Make that first call
 * before any stream capture.  Ra and Pr change nothing in the tables.  Calls
 * ordered on one stream are therefore correct whatever their sizes; calls whose
 * work overlaps on the GPU (other streams or host threads without ordering)
 * share the static arrays, race and give wrong results.
 * Errors are reported through pizza_last_error(NULL). */
#define PIZZA_NOALLOC_MAX_NR 257
#define PIZZA_NOALLOC_MAX_NPHI 768
int pizza_explicit_terms_noalloc(int n_r, int n_phi, double Ra, double Pr, double radius_ratio,
                                 const double *psi_hat, const double *theta_hat,
                                 const double *uphi0_hat, double *e_psi, double *e_theta,
                                 double *e_uphi, void *stream);

/* m-slab decomposition of one step over ranks (Section 5: the 1-D decomposition
 * of the paper, radius-local for the azimuthal transforms, m-local for the
 * radial work, joined by two all-to-all transposes per explicit evaluation).
 *
 * After this call the context advances only the modes m_lo <= m < m_hi of its
 * state (every per-mode kernel: synthesis a1, analysis a3, right-hand side and
 * solve; the zonal flow on the rank whose slab holds m = 0) and runs the
 * azimuthal products a2 only for the radii k_lo <= k < k_hi.  The grid arrays
 * live in the caller's buffers grid1 and grid2 (DEVICE memory, 16-byte aligned,
 * at least n_r * 4 * (N_m + 1) * 16 bytes each, radius-major [k][field][m]); the
 * library calls
 *     exchange(user, 1, grid1, elem_bytes, stream)   after a1,
 *     exchange(user, 2, grid2, elem_bytes, stream)   after a2,
 * from the thread that called pizza_step, with work already queued on `stream`
 * (the context's cudaStream_t).  Call 1 must leave in grid1, for this rank's
 * radii, the synthesis values of every mode (the other ranks' columns
 * [k][f][m] with m in their slabs); call 2 must leave in grid2, for this rank's
 * modes, the product values of every radius.  elem_bytes is 16 (complex FP64)
 * or 8 (complex FP32, option "precision" = 1).  A nonzero return fails the
 * step with PIZZA_ECUDA.  The state arrays keep their full size; get_state
 * returns meaningful values only for the slab's modes.
 *
 * The full ranges (0, N_m+1, 0, n_r) with exchange = NULL return the context
 * to the whole step.  Integration formulation only (tau rows or Galerkin
 * bases); diagnostics, the physical grid, the adjoint, the autotuner and
 * batches return PIZZA_EUNSUPPORTED on a slab context.  PIZZA_EINVAL for bad
 * ranges, missing buffers or callback. */
typedef int (*pizza_exchange_fn)(void *user, int which, void *grid, int elem_bytes, void *stream);
int pizza_set_slab(pizza_ctx *ctx, int m_lo, int m_hi, int k_lo, int k_hi, void *grid1, void *grid2,
                   pizza_exchange_fn exchange, void *user);

/* Measured FP64 fused multiply-add rate of the current device, in TFLOP/s
 * (2 flops per FMA): one launch of `iters` rounds of 8 independent FMA chains in
 * each of 8 x 256 threads per SM, timed with CUDA events after a short warm-up
 * launch.  A measurement helper with no counterpart in the paper: the FP64
 * kernels of the step are bound by FP64 issue on this GPU, and this is their
 * roofline denominator.  *ms (may be NULL) receives the timed launch's duration.
 * Allocates a small output array; PIZZA_EINVAL for iters < 1 or NULL tflops. */
int pizza_fp64_fma_rate(int iters, double *tflops, double *ms);

void pizza_free(pizza_ctx *ctx);

/* Message of the last failing call on ctx (or of the last failing pizza_init
 * when ctx is NULL).  Never NULL. */
const char *pizza_last_error(const pizza_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIZZA_H */
