// C interface (include/pizza.h): context set-up, factorisation of the tau
// systems for each implicit weight, and the order of kernel launches for the
// multistep (Eq. multistep1) and diagonally implicit (Eq. dirks) schemes of
// Section 4 of Gastine, pizza, GJI 2019.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <algorithm>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/pizza.h"
#include "pizza_internal.h"

using namespace pz;

namespace {

thread_local std::string g_init_error = "no error";

constexpr int NVEC = 16;

}  // namespace

namespace pz {
void set_global_error(const char* msg) { g_init_error = msg; }

// Factor L = 3^a 2^b into Stockham passes: radix 3 first, then (with use8)
// radix 8 while a factor of 8 remains (16 stays 4 x 4), then 4s and 2s.
static int fft_factors(int L, bool use8, int* radix) {
    int n = L, np = 0;
    if (n % 3 == 0) {
        radix[np++] = 3;
        n /= 3;
    }
    if (n <= 0 || (n & (n - 1)) != 0) return -1;
    while (use8 && n % 8 == 0 && n != 16 && np < MAX_PASSES) {
        radix[np++] = 8;
        n /= 8;
    }
    while (n % 4 == 0 && np < MAX_PASSES) {
        radix[np++] = 4;
        n /= 4;
    }
    while (n % 2 == 0 && np < MAX_PASSES) {
        radix[np++] = 2;
        n /= 2;
    }
    return n == 1 ? np : -1;
}

bool make_fft_plan(int L, FftPlan& pl) {
    // FP64 transforms keep radix 4 (radix 8 measured slower there: its
    // butterflies hold more registers); FP32 transforms and the double-float
    // azimuthal and radial transforms take radix 8 (fft_batched's R8)
    const int np = fft_factors(L, false, pl.radix), np8 = fft_factors(L, true, pl.radix8);
    if (np < 0 || np8 < 0) return false;
    pl.L = L;
    pl.npass = np;
    pl.npass8 = np8;
    pl.tws = 1;
    return true;
}

std::vector<double2> fft_twiddles(int L) {
    std::vector<double2> t(L);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < L; ++j) {
        long double a = 2.0L * pi * (long double)j / (long double)L;
        t[j] = make_double2((double)cosl(a), (double)(-sinl(a)));
    }
    return t;
}

}  // namespace pz

struct pizza_ctx {
    int n_r = 0, n_phi = 0, n_m = 0, M = 0, nc = 0, K = 0, scheme = 0;
    double E = 0, Ra = 0, Pr = 0, eta = 0, dt = 0;
    bool dt_set = false;
    int device = 0;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    std::vector<void*> allocs;
    StepParams P{};
    double2 *G1 = nullptr, *G2 = nullptr;
    VecSet vec[NVEC]{};
    std::vector<double> gammas;          // implicit weights in use
    std::vector<DevFactors> factors;     // one per gamma (empty until built)
    std::vector<std::vector<void*>> factor_allocs;
    // scheme bookkeeping
    int n_done = 0;
    bool aux_valid = false;  // mass/imp of the current state computed
    // multistep rings (indices into vec); the collocation path uses four state slots
    int ys[4]{}, es[4]{}, ms[3]{}, is[3]{};
    // DIRK slots
    int stage_y[4]{}, stage_e[4]{}, stage_imp[4]{}, mass_n = 0;
    std::string err = "no error";
    // per-kernel event timing
    unsigned prof_mask = 0;
    struct ProfRec {
        int kernel;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    // diagnostics: quadrature weights q_k (int f s ds ~ sum q_k f_k), outputs
    double *diag_q = nullptr, *diag_modes = nullptr, *diag_radii = nullptr;
    std::vector<double> s_host, ds_host;
    // Chebyshev-collocation formulation (option "radial" = 0)
    bool coll = false;
    // Galerkin bases for the integration formulation's solves (option "radial" = 2)
    bool gal = false;
    // temperature solves with FP32 chains and FP64-residual corrections (option
    // "theta_fp32"): 1 always, 0 never, -1 (default) from N_c > 600
    int theta32 = -1;
    std::vector<void*> vec_allocs;     // state and work vectors (re-made when the formulation changes)
    std::vector<double> coll_d1_row0;  // d/ds at s_o on grid values
    double* grid_out = nullptr;        // pizza_get_grid staging, 4 x n_r x n_phi
    // Ekman pumping (option "pumping_eps"; 0 = off)
    double pump_eps = 0.0;
    // bumped by every accepted option change: a batch graph captured under other
    // options (or other factor buffers) is not relaunched
    unsigned epoch = 0;
    // option "check_finite": scan the state for NaN/Inf after every step
    int check_finite = 0;
    int* finite_flag = nullptr;  // device flag set by the scan, read by pizza_synchronize
    // running sum of Nu - 1 over completed steps (pizza_nusselt_begin/end)
    bool nu_on = false;
    int nu_steps = 0;
    double* nu_buf = nullptr;  // [0] the sum, [1 ..] the weights w_n
    // option "cfl_alpha" (Eq. cfl): > 0 checks dt <= alpha / max(cfl_s, cfl_phi)
    // of every state whose explicit terms were evaluated since the last check
    double cfl_alpha = 0.0;
    double* cfl_buf = nullptr;   // [2] running maxima, then [n_r] local spacing
    double* pump_tab = nullptr;        // 3 x n_r device tables (StepParams pump_*)
    double2* pump_buf = nullptr;       // [M][n_r] working buffer of the integration path
    // discrete adjoint (pizza_tape_begin / pizza_adjoint_step)
    struct Adjoint {
        bool taping = false;       // forward steps are being recorded
        bool ready = false;        // buffers and dense inverses built
        int every = 20;            // checkpoint interval
        int K = 0;                 // recorded steps
        int pos = 0;               // adjoint position: lam holds dJ/dy_pos (without g_pos)
        int seg = -1;              // segment cached in seg_y
        double* dRa_dev = nullptr;  // running dJ/dRa on the device (ra[M])
        std::vector<VecSet> ck_y, ck_e;  // checkpoints: y_{s*every}, E(y_{s*every - 1})
        std::vector<VecSet> seg_y;       // y_{seg*every + i}, i < every
        // grid fields (k_spec_to_grid output) of seg_y[i], written by the segment
        // recomputation's explicit stage for i < seg_g1n (all but the last state)
        std::vector<double2*> seg_G1;
        int seg_g1n = 0;
        VecSet lam{}, rho[2]{}, w{}, g{};
        int rcur = 0;
        double2 *Gb1 = nullptr, *Gb2 = nullptr;
        double* ra = nullptr;
        AdjFactors A{};
        std::vector<void*> allocs;     // buffers and inverses
        std::vector<void*> ck_allocs;  // checkpoints of the current tape
    } adj;
    // m-slab decomposition (pizza_set_slab): this context advances modes
    // [P.m_lo, P.m_lo + P.m_n) and transforms radii [P.k_lo, P.k_lo + P.k_n) in
    // the caller's grid buffers, the exchange callback moving the grid between
    // the two layouts after a1 and after a2
    struct Slab {
        bool on = false;
        void *g1 = nullptr, *g2 = nullptr;
        pizza_exchange_fn fn = nullptr;
        void* user = nullptr;
    } slab;
};

namespace {

int fail(pizza_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_init_error = buf;
    return code;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, PIZZA_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

template <class T>
T* dalloc(pizza_ctx* ctx, size_t n, std::vector<void*>& list) {
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T) + 16) != cudaSuccess) return nullptr;
    list.push_back(p);
    return static_cast<T*>(p);
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int cuda_check(pizza_ctx* ctx, cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(ctx, PIZZA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return PIZZA_OK;
}

void free_factors(pizza_ctx* ctx) {
    for (auto& l : ctx->factor_allocs)
        for (void* p : l) cudaFree(p);
    ctx->factor_allocs.clear();
    ctx->factors.clear();
}

std::vector<double> scheme_gammas(int scheme) {
    switch (scheme) {
        case PIZZA_CNAB2: return {0.5};
        case PIZZA_SBDF2: return {1.0, 2.0 / 3.0};
        case PIZZA_SBDF3: return {1.0, 2.0 / 3.0, 6.0 / 11.0};
        case PIZZA_ARS443: return {0.5};
        case PIZZA_BPR353: return {0.5};
    }
    return {};
}

// ---------------------------------------------------------------------------
// Factorisation (host) of the tau systems for one implicit weight.
// ---------------------------------------------------------------------------
struct HostOps {
    std::vector<double> band[OP_COUNT];  // band storage with each operator's own half width
};

// A banded block D (rows and columns [off, off + n) of a band of half width hw,
// rows of 2 hw + 1 entries) split into halves [0, nA) and [nA, n), coupled
// through 8 columns each way: the spikes V = D_A^{-1} E (E: A's rows x B's first
// 8 columns) and W = D_B^{-1} F (F: B's rows x A's last 8 columns), by pivoted
// band LU of each half with its coupling cut, and the inverse of the 16 x 16
// interface system [[I, V_last], [W_first, I]].  V is nA x 8, W (n - nA) x 8.
template <class T>
bool split_spikes(const std::vector<T>& band, int hw, int off, int n, int nA, std::vector<T>& V, std::vector<T>& W,
                  std::vector<T>& Jinv) {
    const int w = 2 * hw + 1, nB = n - nA;
    auto half = [&](int r0, int nh, std::vector<T>& hb) {
        hb.assign((size_t)nh * w, T(0.0));
        for (int i = 0; i < nh; ++i)
            for (int d = 0; d < w; ++d) {
                const int j = i - hw + d;
                if (j >= 0 && j < nh) hb[(size_t)i * w + d] = band[(size_t)(off + r0 + i) * w + d];
            }
    };
    auto D = [&](int i, int j) -> T {  // D(i, j), i, j < n
        const int d = j - i + hw;
        return (d < 0 || d >= w) ? T(0.0) : band[(size_t)(off + i) * w + d];
    };
    std::vector<T> bandA, bandB, La, Ua, Lb, Ub, col;
    std::vector<unsigned char> pa, pb;
    std::vector<double> ra, rb;
    half(0, nA, bandA);
    half(nA, nB, bandB);
    if (!band_lu_pivot(nA, hw, hw, bandA, La, Ua, pa, ra) || !band_lu_pivot(nB, hw, hw, bandB, Lb, Ub, pb, rb))
        return false;
    V.assign((size_t)nA * 8, T(0.0));
    W.assign((size_t)nB * 8, T(0.0));
    for (int c = 0; c < 8; ++c) {
        col.assign(nA, T(0.0));
        for (int i = 0; i < nA; ++i) col[i] = D(i, nA + c);
        band_lu_pivot_solve(nA, hw, hw, La, Ua, pa, ra, col.data());
        for (int i = 0; i < nA; ++i) V[(size_t)i * 8 + c] = col[i];
        col.assign(nB, T(0.0));
        for (int i = 0; i < nB; ++i) col[i] = D(nA + i, nA - 8 + c);
        band_lu_pivot_solve(nB, hw, hw, Lb, Ub, pb, rb, col.data());
        for (int i = 0; i < nB; ++i) W[(size_t)i * 8 + c] = col[i];
    }
    std::vector<T> J(256, T(0.0));
    for (int r = 0; r < 8; ++r) {
        J[(size_t)r * 16 + r] = T(1.0);
        J[(size_t)(8 + r) * 16 + 8 + r] = T(1.0);
        for (int c = 0; c < 8; ++c) {
            J[(size_t)r * 16 + 8 + c] = V[(size_t)(nA - 8 + r) * 8 + c];
            J[(size_t)(8 + r) * 16 + c] = W[(size_t)r * 8 + c];
        }
    }
    return dense_inverse(16, J, Jinv);
}

int build_factors(pizza_ctx* ctx, const HostOps& H, double gamma, DevFactors& F, std::vector<void*>& al) {
    const int M = ctx->M, nc = ctx->nc, np = nc - 4, nt = nc - 2;
    const double gdt = gamma * ctx->dt;
    const auto tauP = tau_rows_psi(ctx->n_r, nc);
    const auto tauD = tau_rows_dir(ctx->n_r, nc);
    const int nbp = (np + 7) / 8, nbt = (nt + 7) / 8;
    std::vector<double2> hpK((size_t)M * nbp * 3 * 64), hpY((size_t)M * np * 4), hpS((size_t)M * 16),
        hpB((size_t)M * np * 17);
    std::vector<double> htK((size_t)M * nbt * 3 * 64), htY((size_t)M * nt * 2), htS((size_t)M * 4),
        htB((size_t)M * nt * 9);
    std::vector<int> bad(M, 0);
    auto get = [&](int id, int k, int n) -> double {
        const int h = op_h(id);
        const int d = n - k + h;
        if (d < 0 || d > 2 * h) return 0.0;
        return H.band[id][(size_t)k * (2 * h + 1) + d];
    };
    // the streamfunction block split in two halves, rows [0, nA) and [nA, np) of D
    // (rows and columns 4.. of the band), when its chains are long: from 40 blocks
    // of 8 rows (n_r >= 481).  The join (interface solve, spike corrections, two
    // barriers per solve) cost more than the halved chains saved at n_r = 257 (21
    // blocks: solve 89.7 -> 99.6 us); at n_r = 2049 (171 blocks) 7.87 -> 6.56 ms.
    const bool psplit = nbp >= 40;
    const int nA = 8 * (nbp / 2), nB = np - nA;
    std::vector<double2> hpSpk(psplit ? (size_t)M * np * 8 : 0), hpRj(psplit ? (size_t)M * 256 : 0);
    auto split_factors = [&](const std::vector<cplx>& bp, int m, std::vector<cplx>& blk) -> bool {
        std::vector<cplx> ba, bb;
        if (!block_lu_twisted(bp, 4 + nA, 8, 4, ba) || !block_lu_twisted(bp, nc, 8, 4 + nA, bb)) return false;
        blk = ba;
        blk.insert(blk.end(), bb.begin(), bb.end());
        std::vector<cplx> V, Wm, Jinv;
        if (!split_spikes(bp, 8, 4, np, nA, V, Wm, Jinv)) return false;
        for (int i = 0; i < nA; ++i)
            for (int c = 0; c < 8; ++c) {
                const cplx v = V[(size_t)i * 8 + c];
                hpSpk[((size_t)m * np + i) * 8 + c] = make_double2(v.real(), v.imag());
            }
        for (int i = 0; i < nB; ++i)
            for (int c = 0; c < 8; ++c) {
                const cplx v = Wm[(size_t)i * 8 + c];
                hpSpk[((size_t)m * np + nA + i) * 8 + c] = make_double2(v.real(), v.imag());
            }
        for (int i = 0; i < 256; ++i) hpRj[(size_t)m * 256 + i] = make_double2(Jinv[i].real(), Jinv[i].imag());
        return true;
    };
    // Large N_c: the temperature systems lose digits in the unpivoted block
    // factorisation and need a refinement step.  Two FP64-residual corrections of
    // FP32 solves reach the accuracy of the FP64 solve there (1e-13 at N_c = 1365,
    // measured on the tau systems), with the chains on the FP32 pipe; the
    // zonal-flow system (one mode) keeps its FP64 refinement.
    const int ir_t = (ctx->theta32 > 0 || (ctx->theta32 < 0 && nc > 600)) ? 2 : 0;
    // the FP32 temperature block split in two halves like the streamfunction one
    // (the kernel with one CTA per system walks each half with its own warp pair)
    const bool tsplit = ir_t && nbt >= 40;
    const int ntA = 8 * (nbt / 2);
    std::vector<double> htSpk(tsplit ? (size_t)M * nt * 8 : 0), htRj(tsplit ? (size_t)M * 256 : 0),
        htKs(tsplit ? htK.size() : 0);
    auto work = [&](int m0, int m1) {
        std::vector<cplx> bp((size_t)nc * 17);
        std::vector<double> bt((size_t)nc * 9);
        for (int m = m0; m < m1; ++m) {
            const double mu = (double)m * m, dm = (double)m;
            // streamfunction: A_m - gdt B_m, half width 8
            if (m > 0) {
                for (int k = 0; k < nc; ++k)
                    for (int d = 0; d < 17; ++d) {
                        const int n = k - 8 + d;
                        cplx v(0.0, 0.0);
                        if (n >= 0 && n < nc && k >= 4) {
                            const double a = get(OP_A0, k, n) + mu * get(OP_A2, k, n);
                            const double b = get(OP_B0, k, n) + mu * (get(OP_B2, k, n) + mu * get(OP_B4, k, n));
                            const double c = get(OP_C, k, n);
                            v = cplx(a - gdt * b, -gdt * 2.0 * dm / ctx->E * c);
                        }
                        bp[(size_t)k * 17 + d] = v;
                    }
                for (size_t i = 0; i < (size_t)np * 17; ++i)
                    hpB[(size_t)m * np * 17 + i] = make_double2(bp[4 * 17 + i].real(), bp[4 * 17 + i].imag());
                Bordered<cplx> f;
                if (!factor_bordered(bp, nc, 8, tauP, 4, f)) {
                    bad[m] = 1;
                    continue;
                }
                std::vector<cplx> blk;
                if (!psplit) {
                    if (!block_lu_twisted(bp, nc, 8, 4, blk)) {
                        bad[m] = 1;
                        continue;
                    }
                } else if (!split_factors(bp, m, blk)) {
                    bad[m] = 1;
                    continue;
                }
                for (size_t i = 0; i < blk.size(); ++i)
                    hpK[(size_t)m * nbp * 192 + i] = make_double2(blk[i].real(), blk[i].imag());
                for (size_t i = 0; i < (size_t)np * 4; ++i)
                    hpY[(size_t)m * np * 4 + i] = make_double2(f.Y[i].real(), f.Y[i].imag());
                for (int i = 0; i < 16; ++i) hpS[(size_t)m * 16 + i] = make_double2(f.Sinv[i].real(), f.Sinv[i].imag());
            }
            // temperature: D - gdt F_m / Pr, half width 4
            for (int k = 0; k < nc; ++k)
                for (int d = 0; d < 9; ++d) {
                    const int n = k - 4 + d;
                    double v = 0.0;
                    if (n >= 0 && n < nc && k >= 2)
                        v = get(OP_D, k, n) - gdt * (get(OP_F0, k, n) + mu * get(OP_F2, k, n)) / ctx->Pr;
                    bt[(size_t)k * 9 + d] = v;
                }
            Bordered<double> g;
            if (!factor_bordered(bt, nc, 4, tauD, 2, g)) {
                bad[m] = 1;
                continue;
            }
            std::copy(bt.begin() + 2 * 9, bt.end(), htB.begin() + (size_t)m * nt * 9);
            // block chains of 8 rows (the band of half width 4 padded): half the
            // chain steps of 4-row blocks, and every lane of the warp busy
            std::vector<double> tb, bt8((size_t)nc * 17, 0.0);
            for (int k = 0; k < nc; ++k)
                for (int d = 0; d < 9; ++d) bt8[(size_t)k * 17 + d + 4] = bt[(size_t)k * 9 + d];
            if (!block_lu_twisted(bt8, nc, 8, 2, tb)) {
                bad[m] = 1;
                continue;
            }
            std::copy(tb.begin(), tb.end(), htK.begin() + (size_t)m * nbt * 192);
            if (tsplit) {  // and the halves (kept beside: the per-mode kernel walks the whole block)
                std::vector<double> ta, tb2, V, Wm, Jinv;
                if (!block_lu_twisted(bt8, 2 + ntA, 8, 2, ta) || !block_lu_twisted(bt8, nc, 8, 2 + ntA, tb2) ||
                    !split_spikes(bt8, 8, 2, nt, ntA, V, Wm, Jinv)) {
                    bad[m] = 1;
                    continue;
                }
                std::copy(ta.begin(), ta.end(), htKs.begin() + (size_t)m * nbt * 192);
                std::copy(tb2.begin(), tb2.end(), htKs.begin() + (size_t)m * nbt * 192 + ta.size());
                std::copy(V.begin(), V.end(), htSpk.begin() + (size_t)m * nt * 8);
                std::copy(Wm.begin(), Wm.end(), htSpk.begin() + ((size_t)m * nt + ntA) * 8);
                std::copy(Jinv.begin(), Jinv.end(), htRj.begin() + (size_t)m * 256);
            }
            std::copy(g.Y.begin(), g.Y.end(), htY.begin() + (size_t)m * nt * 2);
            std::copy(g.Sinv.begin(), g.Sinv.end(), htS.begin() + (size_t)m * 4);
        }
    };
    unsigned nthr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    const int chunk = (M + (int)nthr - 1) / (int)nthr;
    for (unsigned t = 0; t < nthr; ++t) {
        int a = (int)t * chunk, b = std::min(M, a + chunk);
        if (a < b) th.emplace_back(work, a, b);
    }
    for (auto& t : th) t.join();
    for (int m = 0; m < M; ++m)
        if (bad[m]) return fail(ctx, PIZZA_EINVAL, "tau system of mode m=%d is singular", m);
    // zonal flow: D - gdt E^I
    std::vector<double> bu((size_t)nc * 9);
    for (int k = 0; k < nc; ++k)
        for (int d = 0; d < 9; ++d) {
            const int n = k - 4 + d;
            double v = 0.0;
            if (n >= 0 && n < nc && k >= 2) v = get(OP_D, k, n) - gdt * get(OP_EZ, k, n);
            bu[(size_t)k * 9 + d] = v;
        }
    Bordered<double> fu;
    if (!factor_bordered(bu, nc, 4, tauD, 2, fu)) return fail(ctx, PIZZA_EINVAL, "zonal-flow tau system singular");

    F.gdt = gdt;
#define UPLOAD(dst, T, hv)                                                                        \
    do {                                                                                          \
        dst = dalloc<T>(ctx, (hv).size(), al);                                                    \
        if (!dst) return fail(ctx, PIZZA_ENOMEM, "device allocation of factors failed");          \
        CK(cudaMemcpy(dst, (hv).data(), (hv).size() * sizeof(T), cudaMemcpyHostToDevice));       \
    } while (0)
    std::vector<double> ub, bu8((size_t)nc * 17, 0.0);
    for (int k = 0; k < nc; ++k)
        for (int d = 0; d < 9; ++d) bu8[(size_t)k * 17 + d + 4] = bu[(size_t)k * 9 + d];
    if (!block_lu_twisted(bu8, nc, 8, 2, ub)) return fail(ctx, PIZZA_EINVAL, "zonal-flow tau system singular");
    UPLOAD(F.pBlk, double2, hpK);
    // double-float copies: the nearest float and the float nearest the remainder
    auto to_dd = [](const std::vector<double2>& v) {
        std::vector<float4> d(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const double re = v[i].x, im = v[i].y;
            const float rh = (float)re, ih = (float)im;
            d[i] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
        }
        return d;
    };
    {
        const std::vector<float4> hd = to_dd(hpK);
        UPLOAD(F.pBlkDD, float4, hd);
    }
    F.psplit = psplit ? 1 : 0;
    if (psplit) {
        UPLOAD(F.pSpk, double2, hpSpk);
        UPLOAD(F.pRj, double2, hpRj);
        const std::vector<float4> sd = to_dd(hpSpk), rd = to_dd(hpRj);
        UPLOAD(F.pSpkDD, float4, sd);
        UPLOAD(F.pRjDD, float4, rd);
    }
    UPLOAD(F.pY, double2, hpY);
    UPLOAD(F.pSinv, double2, hpS);
    UPLOAD(F.pBand, double2, hpB);
    if (!ir_t) UPLOAD(F.tBlk, double, htK);  // with ir_t only the FP32 copy is read
    UPLOAD(F.tY, double, htY);
    UPLOAD(F.tSinv, double, htS);
    UPLOAD(F.tBand, double, htB);
    {
        std::vector<double> ubd(bu.begin() + 2 * 9, bu.end());
        UPLOAD(F.uBand, double, ubd);
    }
    F.ir_t = ir_t;
    if (F.ir_t) {
        const std::vector<float> tK32(htK.begin(), htK.end()), tY32(htY.begin(), htY.end()),
            tS32(htS.begin(), htS.end());
        UPLOAD(F.tBlk32, float, tK32);
        UPLOAD(F.tY32, float, tY32);
        UPLOAD(F.tSinv32, float, tS32);
        F.tsplit = tsplit ? 1 : 0;
        if (tsplit) {
            const std::vector<float> ks32(htKs.begin(), htKs.end()), sp32(htSpk.begin(), htSpk.end()),
                rj32(htRj.begin(), htRj.end());
            UPLOAD(F.tBlk32S, float, ks32);
            UPLOAD(F.tSpk32, float, sp32);
            UPLOAD(F.tRj32, float, rj32);
        }
    }
    UPLOAD(F.uBlk, double, ub);
    UPLOAD(F.uY, double, fu.Y);
    UPLOAD(F.uSinv, double, fu.Sinv);
#undef UPLOAD
    return PIZZA_OK;
}

// Factorisation (host) of the Galerkin-basis systems (Appendix B) for one
// implicit weight: the integrated rows of the tau operators (the same entries as
// build_factors) times the stencils and 1/(C w_n), in band rows, then banded LU
// with partial pivoting.
int build_galerkin_factors(pizza_ctx* ctx, const HostOps& H, double gamma, DevFactors& F,
                           std::vector<void*>& al) {
    const int M = ctx->M, nc = ctx->nc, np = nc - 4, nt = nc - 2;
    const double gdt = gamma * ctx->dt;
    if (np < 1) return fail(ctx, PIZZA_EINVAL, "too few coefficients for the Galerkin bases");
    const double cn = std::sqrt(2.0 / (ctx->n_r - 1));
    auto ihs = [&](int j) { return (j == 0 ? 2.0 : 1.0) / cn; };  // 1/(C w_j)
    std::vector<double> gam((size_t)np * 5);
    for (int n = 0; n < np; ++n) galerkin_gamma(n, &gam[(size_t)n * 5]);
    auto get = [&](int id, int k, int n) -> double {
        const int h = op_h(id);
        const int d = n - k + h;
        if (n < 0 || n >= nc || d < 0 || d > 2 * h) return 0.0;
        return H.band[id][(size_t)k * (2 * h + 1) + d];
    };
    std::vector<double2> hpL((size_t)M * np * 8), hpU((size_t)M * np * 21);
    std::vector<double> hpR((size_t)M * np), htL((size_t)M * nt * 4), htU((size_t)M * nt * 12), htR((size_t)M * nt);
    std::vector<unsigned char> hpP((size_t)M * np), htP((size_t)M * nt);
    std::vector<int> bad(M, 0);
    // Dirichlet system of rows k = i + 2 of an operator L(k, j): band rows of
    // G(i, n) = L(i+2, n+2)/(C w_{n+2}) - L(i+2, n)/(C w_n), 4 below, 6 above
    auto dir_band = [&](const std::function<double(int, int)>& L) {
        std::vector<double> b((size_t)nt * 11, 0.0);
        for (int i = 0; i < nt; ++i)
            for (int d = 0; d < 11; ++d) {
                const int n = i - 4 + d;
                if (n >= 0 && n < nt) b[(size_t)i * 11 + d] = L(i + 2, n + 2) * ihs(n + 2) - L(i + 2, n) * ihs(n);
            }
        return b;
    };
    auto work = [&](int m0, int m1) {
        std::vector<cplx> bp((size_t)np * 21), Lm, Uc;
        std::vector<double> rs, Lt, Ut;
        std::vector<unsigned char> pv;
        for (int m = m0; m < m1; ++m) {
            const double mu = (double)m * m, dm = (double)m;
            if (m > 0) {
                // G(i, n) = sum_q L(i+4, n+q) gamma_q^n / (C w_{n+q}), 8 below, 12 above
                auto L = [&](int k, int j) -> cplx {
                    const double a = get(OP_A0, k, j) + mu * get(OP_A2, k, j);
                    const double b = get(OP_B0, k, j) + mu * (get(OP_B2, k, j) + mu * get(OP_B4, k, j));
                    return cplx(a - gdt * b, -gdt * 2.0 * dm / ctx->E * get(OP_C, k, j));
                };
                for (int i = 0; i < np; ++i)
                    for (int d = 0; d < 21; ++d) {
                        const int n = i - 8 + d;
                        cplx v(0.0, 0.0);
                        if (n >= 0 && n < np)
                            for (int q = 0; q < 5; ++q) v += L(i + 4, n + q) * (gam[(size_t)n * 5 + q] * ihs(n + q));
                        bp[(size_t)i * 21 + d] = v;
                    }
                if (!band_lu_pivot(np, 8, 12, bp, Lm, Uc, pv, rs)) {
                    bad[m] = 1;
                    continue;
                }
                for (size_t i = 0; i < Lm.size(); ++i)
                    hpL[(size_t)m * np * 8 + i] = make_double2(Lm[i].real(), Lm[i].imag());
                for (size_t i = 0; i < Uc.size(); ++i)
                    hpU[(size_t)m * np * 21 + i] = make_double2(Uc[i].real(), Uc[i].imag());
                std::copy(pv.begin(), pv.end(), hpP.begin() + (size_t)m * np);
                std::copy(rs.begin(), rs.end(), hpR.begin() + (size_t)m * np);
            }
            const auto bt = dir_band([&](int k, int j) {
                return get(OP_D, k, j) - gdt * (get(OP_F0, k, j) + mu * get(OP_F2, k, j)) / ctx->Pr;
            });
            if (!band_lu_pivot(nt, 4, 6, bt, Lt, Ut, pv, rs)) {
                bad[m] = 1;
                continue;
            }
            std::copy(Lt.begin(), Lt.end(), htL.begin() + (size_t)m * nt * 4);
            for (int i = 0; i < nt; ++i)  // rows padded to 12 (whole 16-byte pieces)
                std::copy(Ut.begin() + (size_t)i * 11, Ut.begin() + (size_t)(i + 1) * 11,
                          htU.begin() + ((size_t)m * nt + i) * 12);
            std::copy(pv.begin(), pv.end(), htP.begin() + (size_t)m * nt);
            std::copy(rs.begin(), rs.end(), htR.begin() + (size_t)m * nt);
        }
    };
    unsigned nthr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    const int chunk = (M + (int)nthr - 1) / (int)nthr;
    for (unsigned t = 0; t < nthr; ++t) {
        int a = (int)t * chunk, b = std::min(M, a + chunk);
        if (a < b) th.emplace_back(work, a, b);
    }
    for (auto& t : th) t.join();
    for (int m = 0; m < M; ++m)
        if (bad[m]) return fail(ctx, PIZZA_EINVAL, "Galerkin system of mode m=%d is singular", m);
    std::vector<double> uL, uU, uR;
    std::vector<unsigned char> uP;
    const auto bu = dir_band([&](int k, int j) { return get(OP_D, k, j) - gdt * get(OP_EZ, k, j); });
    if (!band_lu_pivot(nt, 4, 6, bu, uL, uU, uP, uR)) return fail(ctx, PIZZA_EINVAL, "zonal-flow Galerkin system singular");

    F.gdt = gdt;
    F.gal = 1;
#define UPLOAD(dst, T, hv)                                                                        \
    do {                                                                                          \
        dst = dalloc<T>(ctx, (hv).size(), al);                                                    \
        if (!dst) return fail(ctx, PIZZA_ENOMEM, "device allocation of factors failed");          \
        CK(cudaMemcpy(dst, (hv).data(), (hv).size() * sizeof(T), cudaMemcpyHostToDevice));       \
    } while (0)
    UPLOAD(F.gpL, double2, hpL);
    UPLOAD(F.gpU, double2, hpU);
    UPLOAD(F.gpR, double, hpR);
    UPLOAD(F.gpPiv, unsigned char, hpP);
    UPLOAD(F.gtL, double, htL);
    UPLOAD(F.gtU, double, htU);
    UPLOAD(F.gtR, double, htR);
    UPLOAD(F.gtPiv, unsigned char, htP);
    UPLOAD(F.guL, double, uL);
    std::vector<double> uU12((size_t)nt * 12, 0.0);
    for (int i = 0; i < nt; ++i) std::copy(uU.begin() + (size_t)i * 11, uU.begin() + (size_t)(i + 1) * 11, uU12.begin() + (size_t)i * 12);
    UPLOAD(F.guU, double, uU12);
    UPLOAD(F.guR, double, uR);
    UPLOAD(F.guPiv, unsigned char, uP);
    UPLOAD(F.gam, double, gam);
#undef UPLOAD
    return PIZZA_OK;
}

HostOps host_ops_of(pizza_ctx* ctx) {
    HostOps H;
    Geom g = make_geom(ctx->eta);
    for (int id = 0; id < OP_COUNT; ++id)
        H.band[id] = to_band(build_operator(id, ctx->n_r, ctx->nc, g), ctx->nc, op_h(id));
    return H;
}

int build_coll_factors(pizza_ctx* ctx, const CollGrid& cg, double gamma, DevFactors& F, std::vector<void*>& al);

int ensure_factors(pizza_ctx* ctx) {
    if (!ctx->factors.empty()) return PIZZA_OK;
    if (!ctx->dt_set) return fail(ctx, PIZZA_ESTATE, "dt is not set (pizza_set_option(ctx, \"dt\", v))");
    ctx->gammas = scheme_gammas(ctx->scheme);
    if (ctx->coll) {
        CollGrid cg = coll_grid(ctx->n_r, make_geom(ctx->eta));
        if (ctx->P.pump) coll_pumping(cg, make_geom(ctx->eta), ctx->E);
        for (double g : ctx->gammas) {
            DevFactors F{};
            std::vector<void*> al;
            int rc = build_coll_factors(ctx, cg, g, F, al);
            ctx->factor_allocs.push_back(al);
            if (rc != PIZZA_OK) {
                free_factors(ctx);
                return rc;
            }
            ctx->factors.push_back(F);
        }
        return PIZZA_OK;
    }
    HostOps H = host_ops_of(ctx);
    for (double g : ctx->gammas) {
        DevFactors F{};
        std::vector<void*> al;
        int rc = ctx->gal ? build_galerkin_factors(ctx, H, g, F, al) : build_factors(ctx, H, g, F, al);
        ctx->factor_allocs.push_back(al);
        if (rc != PIZZA_OK) {
            free_factors(ctx);
            return rc;
        }
        ctx->factors.push_back(F);
    }
    return PIZZA_OK;
}

const DevFactors* factors_for(pizza_ctx* ctx, double gamma) {
    for (size_t i = 0; i < ctx->gammas.size(); ++i)
        if (std::fabs(ctx->gammas[i] - gamma) < 1e-14) return &ctx->factors[i];
    return nullptr;
}

void reset_slots(pizza_ctx* ctx) {
    if (ctx->coll) {
        // vec indices: 0..3 state ring (the mass term of a grid state is the state
        // itself); 4..7 explicit ring; 8..10 imp ring; DIRK stages 11..13; 15 scratch
        for (int i = 0; i < 4; ++i) ctx->ys[i] = i;
        for (int i = 0; i < 4; ++i) ctx->es[i] = 4 + i;
        for (int i = 0; i < 3; ++i) ctx->is[i] = 8 + i;
        for (int i = 0; i < 4; ++i) ctx->stage_e[i] = 4 + i;
        ctx->stage_y[1] = 11; ctx->stage_y[2] = 12; ctx->stage_y[3] = 13;
        ctx->stage_imp[0] = 14; ctx->stage_imp[1] = 8; ctx->stage_imp[2] = 9; ctx->stage_imp[3] = 10;
        ctx->mass_n = 0;
        ctx->n_done = 0;
        ctx->aux_valid = false;
        return;
    }
    // vec indices: 0,1 state ring; 2..5 explicit ring; 6..8 mass ring; 9..11 imp ring
    ctx->ys[0] = 0; ctx->ys[1] = 1;
    for (int i = 0; i < 4; ++i) ctx->es[i] = 2 + i;
    for (int i = 0; i < 3; ++i) ctx->ms[i] = 6 + i;
    for (int i = 0; i < 3; ++i) ctx->is[i] = 9 + i;
    // DIRK: stage states 12..14 (y_1..y_3), explicit 2..5 (e_0..e_3), imp 7 (I_0 = Imp y_n,
    // BPR353 only) and 9..11 (I_1..I_3), mass 6
    ctx->stage_y[1] = 12; ctx->stage_y[2] = 13; ctx->stage_y[3] = 14;
    for (int i = 0; i < 4; ++i) ctx->stage_e[i] = 2 + i;
    ctx->stage_imp[0] = 7; ctx->stage_imp[1] = 9; ctx->stage_imp[2] = 10; ctx->stage_imp[3] = 11;
    ctx->mass_n = 6;
    ctx->n_done = 0;
    ctx->aux_valid = false;
}

cudaEvent_t pool_event(pizza_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch through f(), bracketed by an event pair when kernel id k is profiled.
template <class F>
cudaError_t timed_launch(pizza_ctx* ctx, int k, F&& f) {
    if (!(ctx->prof_mask & (1u << k))) return f();
    pizza_ctx::ProfRec r{k, pool_event(ctx), pool_event(ctx)};
    cudaEventRecord(r.a, ctx->stream);
    cudaError_t e = f();
    cudaEventRecord(r.b, ctx->stream);
    ctx->prof.push_back(r);
    return e;
}

int explicit_eval(pizza_ctx* ctx, VecSet y, VecSet e) {
    if (ctx->coll) {
        CK(timed_launch(ctx, 0, [&] { return launch_coll_spec_to_grid(ctx->P, y, ctx->G1, ctx->stream); }));
        CK(timed_launch(ctx, 1, [&] { return launch_phi_products(ctx->P, ctx->G1, ctx->G2, ctx->stream); }));
        CK(timed_launch(ctx, 2, [&] { return launch_coll_grid_rows(ctx->P, ctx->G1, ctx->G2, e, ctx->stream); }));
        return PIZZA_OK;
    }
    if (ctx->slab.on) {
        // a1 on this rank's modes, transpose to radius slabs, a2 on this rank's
        // radii, transpose back, a3 on this rank's modes (Section 5)
        double2* g1 = static_cast<double2*>(ctx->slab.g1);
        double2* g2 = static_cast<double2*>(ctx->slab.g2);
        const int eb = ctx->P.fp32 ? 8 : 16;
        CK(timed_launch(ctx, 0, [&] { return launch_spec_to_grid(ctx->P, y, g1, ctx->stream); }));
        if (int rc = ctx->slab.fn(ctx->slab.user, 1, g1, eb, ctx->stream))
            return fail(ctx, PIZZA_ECUDA, "slab exchange after the synthesis failed (%d)", rc);
        CK(timed_launch(ctx, 1, [&] { return launch_phi_products(ctx->P, g1, g2, ctx->stream); }));
        if (int rc = ctx->slab.fn(ctx->slab.user, 2, g2, eb, ctx->stream))
            return fail(ctx, PIZZA_ECUDA, "slab exchange after the azimuthal products failed (%d)", rc);
        CK(timed_launch(ctx, 2, [&] { return launch_grid_to_spec(ctx->P, g2, y, e, ctx->stream); }));
        return PIZZA_OK;
    }
    CK(timed_launch(ctx, 0, [&] { return launch_spec_to_grid(ctx->P, y, ctx->G1, ctx->stream); }));
    CK(timed_launch(ctx, 1, [&] { return launch_phi_products(ctx->P, ctx->G1, ctx->G2, ctx->stream); }));
    CK(timed_launch(ctx, 2, [&] { return launch_grid_to_spec(ctx->P, ctx->G2, y, e, ctx->stream); }));
    return PIZZA_OK;
}

bool is_multistep(int scheme) { return scheme <= PIZZA_SBDF3; }

// (a, b0, bI, bE) of Eq. multistep1 with the start-up rule
void multistep_coeffs(int scheme, int n_done, std::vector<double>& a, double& b0, std::vector<double>& bI,
                      std::vector<double>& bE) {
    if (scheme == PIZZA_CNAB2) {
        a = {1.0};
        b0 = 0.5;
        bI = {0.5};
        bE = (n_done == 0) ? std::vector<double>{1.0} : std::vector<double>{1.5, -0.5};
        return;
    }
    int order = (scheme == PIZZA_SBDF2) ? 2 : 3;
    int k = std::min(order, n_done + 1);
    if (k == 1) {
        a = {1.0}; b0 = 1.0; bI = {0.0}; bE = {1.0};
    } else if (k == 2) {
        a = {4.0 / 3.0, -1.0 / 3.0}; b0 = 2.0 / 3.0; bI = {0.0, 0.0}; bE = {4.0 / 3.0, -2.0 / 3.0};
    } else {
        a = {18.0 / 11.0, -9.0 / 11.0, 2.0 / 11.0}; b0 = 6.0 / 11.0; bI = {0.0, 0.0, 0.0};
        bE = {18.0 / 11.0, -18.0 / 11.0, 6.0 / 11.0};
    }
}

// Stiffly accurate SDIRK tableaux of Eq. dirks, stage 0 = y_n, y_{n+1} = stage 4.
struct Tableau {
    double aI[5][5], aE[5][5];
};
// ARS443 (Ascher, Ruuth & Spiteri 1997, Section 2.8)
const Tableau ARS443 = {{{0, 0, 0, 0, 0},
                         {0, 0.5, 0, 0, 0},
                         {0, 1.0 / 6.0, 0.5, 0, 0},
                         {0, -0.5, 0.5, 0.5, 0},
                         {0, 1.5, -1.5, 0.5, 0.5}},
                        {{0, 0, 0, 0, 0},
                         {0.5, 0, 0, 0, 0},
                         {11.0 / 18.0, 1.0 / 18.0, 0, 0, 0},
                         {5.0 / 6.0, -5.0 / 6.0, 0.5, 0, 0},
                         {0.25, 1.75, 0.75, -1.75, 0}}};
// BPR353 (Boscarino, Pareschi & Russo 2013, Section 8.3): its first implicit
// column is not zero (the stages use Imp y_n), and its last explicit column is,
// so E(y_3) is never needed: three explicit evaluations per step (Table 1)
const Tableau BPR353 = {{{0, 0, 0, 0, 0},
                         {0.5, 0.5, 0, 0, 0},
                         {5.0 / 18.0, -1.0 / 9.0, 0.5, 0, 0},
                         {0.5, 0, 0, 0.5, 0},
                         {0.25, 0, 0.75, -0.5, 0.5}},
                        {{0, 0, 0, 0, 0},
                         {1.0, 0, 0, 0, 0},
                         {4.0 / 9.0, 2.0 / 9.0, 0, 0, 0},
                         {0.25, 0, 0.75, 0, 0},
                         {0.25, 0, 0.75, 0, 0}}};

const Tableau& tableau_of(int scheme) { return scheme == PIZZA_BPR353 ? BPR353 : ARS443; }

bool column_used(const double (&a)[5][5], int j) {
    for (int i = j + 1; i < 5; ++i)
        if (a[i][j] != 0.0) return true;
    return false;
}

// The stage j in 1..3 whose implicit term the last stage does not read: the last
// solve writes Imp y_{n+1} there, and the slot then becomes I_0 of the next step.
int spare_imp_stage(const Tableau& T) {
    for (int j = 1; j < 4; ++j)
        if (T.aI[4][j] == 0.0) return j;
    return -1;
}

int ensure_aux(pizza_ctx* ctx) {
    if (ctx->aux_valid) return PIZZA_OK;
    VecSet y = ctx->vec[ctx->ys[0]];
    const bool imp0 = !is_multistep(ctx->scheme) && column_used(tableau_of(ctx->scheme).aI, 0);
    if (ctx->coll) {
        if (ctx->scheme == PIZZA_CNAB2) CK(launch_coll_apply(ctx->P, y, ctx->vec[ctx->is[0]], ctx->stream));
        if (imp0) CK(launch_coll_apply(ctx->P, y, ctx->vec[ctx->stage_imp[0]], ctx->stream));
        ctx->aux_valid = true;
        return PIZZA_OK;
    }
    if (is_multistep(ctx->scheme)) {
        CK(launch_apply(ctx->P, y, ctx->vec[ctx->ms[0]], ctx->vec[ctx->is[0]], true,
                        ctx->scheme == PIZZA_CNAB2, ctx->stream));
    } else {
        CK(launch_apply(ctx->P, y, ctx->vec[ctx->mass_n], imp0 ? ctx->vec[ctx->stage_imp[0]] : ctx->vec[ctx->mass_n],
                        true, imp0, ctx->stream));
    }
    ctx->aux_valid = true;
    return PIZZA_OK;
}

int step_multistep(pizza_ctx* ctx) {
    std::vector<double> a, bI, bE;
    double b0;
    multistep_coeffs(ctx->scheme, ctx->n_done, a, b0, bI, bE);
    const double dt = ctx->dt;
    // rotate explicit ring: new e^n goes to the oldest slot
    int e_new = ctx->es[3];
    for (int i = 3; i > 0; --i) ctx->es[i] = ctx->es[i - 1];
    ctx->es[0] = e_new;
    int rc = explicit_eval(ctx, ctx->vec[ctx->ys[0]], ctx->vec[ctx->es[0]]);
    if (rc) return rc;
    RhsSpec R{};
    for (size_t j = 0; j < a.size(); ++j) R.t[R.nterms++] = {ctx->vec[ctx->ms[j]], a[j]};
    for (size_t j = 0; j < bI.size(); ++j)
        if (bI[j] != 0.0) R.t[R.nterms++] = {ctx->vec[ctx->is[j]], dt * bI[j]};
    for (size_t j = 0; j < bE.size(); ++j) R.t[R.nterms++] = {ctx->vec[ctx->es[j]], dt * bE[j]};
    const DevFactors* F = factors_for(ctx, b0);
    if (!F) return fail(ctx, PIZZA_EINVAL, "no factors for implicit weight %g", b0);
    // outputs overwrite the oldest mass / imp slots (each CTA reads its rows first)
    const int m_new = ctx->ms[2], i_new = ctx->is[2];
    const bool want_imp = (ctx->scheme == PIZZA_CNAB2);
    CK(timed_launch(ctx, 3, [&] {
        return launch_solve(ctx->P, R, *F, ctx->vec[ctx->ys[1]], ctx->vec[m_new], ctx->vec[i_new], true, want_imp,
                            ctx->stream);
    }));
    std::swap(ctx->ys[0], ctx->ys[1]);
    ctx->ms[2] = ctx->ms[1]; ctx->ms[1] = ctx->ms[0]; ctx->ms[0] = m_new;
    ctx->is[2] = ctx->is[1]; ctx->is[1] = ctx->is[0]; ctx->is[0] = i_new;
    return PIZZA_OK;
}

// Right-hand side of stage i (Eq. dirks): mass term of y_n plus dt times the
// explicit and implicit terms of the earlier stages that the tableau weights.
RhsSpec dirk_rhs(pizza_ctx* ctx, const Tableau& T, int i, VecSet mass) {
    const double dt = ctx->dt;
    RhsSpec R{};
    R.t[R.nterms++] = {mass, 1.0};
    for (int j = 0; j < i; ++j) {
        if (T.aE[i][j] != 0.0) R.t[R.nterms++] = {ctx->vec[ctx->stage_e[j]], dt * T.aE[i][j]};
        if (T.aI[i][j] != 0.0) R.t[R.nterms++] = {ctx->vec[ctx->stage_imp[j]], dt * T.aI[i][j]};
    }
    return R;
}

int step_dirk(pizza_ctx* ctx) {
    const Tableau& T = tableau_of(ctx->scheme);
    const int nu = 4;
    const bool imp0 = column_used(T.aI, 0);
    const int spare = imp0 ? spare_imp_stage(T) : -1;
    for (int i = 1; i <= nu; ++i) {
        VecSet y_prev = (i == 1) ? ctx->vec[ctx->ys[0]] : ctx->vec[ctx->stage_y[i - 1]];
        if (column_used(T.aE, i - 1)) {
            int rc = explicit_eval(ctx, y_prev, ctx->vec[ctx->stage_e[i - 1]]);
            if (rc) return rc;
        }
        RhsSpec R = dirk_rhs(ctx, T, i, ctx->vec[ctx->mass_n]);
        const DevFactors* F = factors_for(ctx, T.aI[i][i]);
        if (!F) return fail(ctx, PIZZA_EINVAL, "no factors for a_ii");
        if (i < nu) {
            CK(timed_launch(ctx, 3, [&] {
                return launch_solve(ctx->P, R, *F, ctx->vec[ctx->stage_y[i]], ctx->vec[ctx->mass_n],
                                    ctx->vec[ctx->stage_imp[i]], false, true, ctx->stream);
            }));
        } else {
            // y_{n+1} = y_nu (stiffly accurate); its mass term replaces Mass(y_n), and
            // where the stages use Imp y_n, Imp y_{n+1} goes to the spare stage slot
            VecSet imp_out = imp0 ? ctx->vec[ctx->stage_imp[spare]] : ctx->vec[ctx->mass_n];
            CK(timed_launch(ctx, 3, [&] {
                return launch_solve(ctx->P, R, *F, ctx->vec[ctx->ys[1]], ctx->vec[ctx->mass_n], imp_out, true, imp0,
                                    ctx->stream);
            }));
        }
    }
    if (imp0) std::swap(ctx->stage_imp[0], ctx->stage_imp[spare]);
    std::swap(ctx->ys[0], ctx->ys[1]);
    return PIZZA_OK;
}

// Collocation: the mass term of a grid state is the state itself, so the right
// hand side combines states, implicit terms and explicit rows directly; every
// output goes to a slot that is not an input of the same launch.
int step_multistep_coll(pizza_ctx* ctx) {
    std::vector<double> a, bI, bE;
    double b0;
    multistep_coeffs(ctx->scheme, ctx->n_done, a, b0, bI, bE);
    const double dt = ctx->dt;
    int e_new = ctx->es[3];
    for (int i = 3; i > 0; --i) ctx->es[i] = ctx->es[i - 1];
    ctx->es[0] = e_new;
    int rc = explicit_eval(ctx, ctx->vec[ctx->ys[0]], ctx->vec[ctx->es[0]]);
    if (rc) return rc;
    RhsSpec R{};
    for (size_t j = 0; j < a.size(); ++j) R.t[R.nterms++] = {ctx->vec[ctx->ys[j]], a[j]};
    for (size_t j = 0; j < bI.size(); ++j)
        if (bI[j] != 0.0) R.t[R.nterms++] = {ctx->vec[ctx->is[j]], dt * bI[j]};
    for (size_t j = 0; j < bE.size(); ++j) R.t[R.nterms++] = {ctx->vec[ctx->es[j]], dt * bE[j]};
    const DevFactors* F = factors_for(ctx, b0);
    if (!F) return fail(ctx, PIZZA_EINVAL, "no factors for implicit weight %g", b0);
    const int y_new = ctx->ys[3], i_new = ctx->is[2];
    const bool want_imp = (ctx->scheme == PIZZA_CNAB2);
    CK(timed_launch(ctx, 3, [&] {
        return launch_coll_solve(ctx->P, R, *F, ctx->vec[y_new], ctx->vec[y_new], ctx->vec[i_new], false, want_imp,
                                 ctx->stream);
    }));
    for (int i = 3; i > 0; --i) ctx->ys[i] = ctx->ys[i - 1];
    ctx->ys[0] = y_new;
    ctx->is[2] = ctx->is[1]; ctx->is[1] = ctx->is[0]; ctx->is[0] = i_new;
    return PIZZA_OK;
}

int step_dirk_coll(pizza_ctx* ctx) {
    const Tableau& T = tableau_of(ctx->scheme);
    const int nu = 4;
    const bool imp0 = column_used(T.aI, 0);
    const int spare = imp0 ? spare_imp_stage(T) : -1;
    for (int i = 1; i <= nu; ++i) {
        VecSet y_prev = (i == 1) ? ctx->vec[ctx->ys[0]] : ctx->vec[ctx->stage_y[i - 1]];
        if (column_used(T.aE, i - 1)) {
            int rc = explicit_eval(ctx, y_prev, ctx->vec[ctx->stage_e[i - 1]]);
            if (rc) return rc;
        }
        RhsSpec R = dirk_rhs(ctx, T, i, ctx->vec[ctx->ys[0]]);
        const DevFactors* F = factors_for(ctx, T.aI[i][i]);
        if (!F) return fail(ctx, PIZZA_EINVAL, "no factors for a_ii");
        const bool last = (i == nu);
        VecSet out = last ? ctx->vec[ctx->ys[1]] : ctx->vec[ctx->stage_y[i]];
        // the spare slot is not an input of the last stage
        VecSet imp = last ? (imp0 ? ctx->vec[ctx->stage_imp[spare]] : out) : ctx->vec[ctx->stage_imp[i]];
        const bool want_imp = !last || imp0;
        CK(timed_launch(ctx, 3, [&] {
            return launch_coll_solve(ctx->P, R, *F, out, out, imp, false, want_imp, ctx->stream);
        }));
    }
    if (imp0) std::swap(ctx->stage_imp[0], ctx->stage_imp[spare]);
    std::swap(ctx->ys[0], ctx->ys[1]);
    return PIZZA_OK;
}

// Grid-valued inverses of the collocation systems for one implicit weight
// (coll_ops.cpp), one thread range of modes per host thread.
int build_coll_factors(pizza_ctx* ctx, const CollGrid& cg, double gamma, DevFactors& F, std::vector<void*>& al) {
    const int M = ctx->M, N = ctx->n_r, ni = N - 2;
    const double gdt = gamma * ctx->dt;
    std::vector<double2> hW((size_t)M * 2 * N * ni, make_double2(0.0, 0.0));
    std::vector<double> hT((size_t)M * N * ni), hU;
    std::vector<int> bad(M, 0);
    auto work = [&](int m0, int m1) {
        std::vector<cplx> G;
        std::vector<double> Gt;
        for (int m = m0; m < m1; ++m) {
            // stored column-major (one column per interior right-hand-side row)
            if (m > 0) {
                if (!coll_inverse_wpsi(cg, ctx->E, m, gdt, G)) {
                    bad[m] = 1;
                    continue;
                }
                for (int i = 0; i < 2 * N; ++i)
                    for (int j = 0; j < ni; ++j) {
                        const cplx g = G[(size_t)i * ni + j];
                        hW[((size_t)m * ni + j) * 2 * N + i] = make_double2(g.real(), g.imag());
                    }
            }
            if (!coll_inverse_dir(cg, 1.0 / ctx->Pr, (double)m * m, gdt, Gt)) {
                bad[m] = 1;
                continue;
            }
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < ni; ++j) hT[((size_t)m * ni + j) * N + i] = Gt[(size_t)i * ni + j];
        }
    };
    unsigned nthr = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    // interleave the modes so that every thread gets a similar mix
    for (unsigned t = 0; t < nthr; ++t) {
        th.emplace_back([&, t] {
            for (int m = (int)t; m < M; m += (int)nthr) work(m, m + 1);
        });
    }
    for (auto& t : th) t.join();
    for (int m = 0; m < M; ++m)
        if (bad[m]) return fail(ctx, PIZZA_EINVAL, "collocation system of mode m=%d is singular", m);
    {
        std::vector<double> gu;
        if (!coll_inverse_dir(cg, 1.0, 1.0, gdt, gu, true))
            return fail(ctx, PIZZA_EINVAL, "zonal-flow system singular");
        hU.resize(gu.size());
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < ni; ++j) hU[(size_t)j * N + i] = gu[(size_t)i * ni + j];
    }
    F.gdt = gdt;
    auto upload = [&](auto*& dst, const auto& hv) -> int {
        using T = std::remove_reference_t<decltype(*dst)>;
        dst = dalloc<T>(ctx, hv.size(), al);
        if (!dst) return fail(ctx, PIZZA_ENOMEM, "device allocation of the collocation inverses failed");
        CK(cudaMemcpy(dst, hv.data(), hv.size() * sizeof(T), cudaMemcpyHostToDevice));
        return PIZZA_OK;
    };
    int rc = upload(F.colW, hW);
    if (!rc) rc = upload(F.colT, hT);
    if (!rc) rc = upload(F.colU, hU);
    return rc;
}

// (Re)allocate the NVEC work vectors with the coefficient stride of the selected
// formulation (the vorticity field only for collocation), zeroed.
int alloc_vecs(pizza_ctx* ctx) {
    for (void* p : ctx->vec_allocs) cudaFree(p);
    ctx->vec_allocs.clear();
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    for (int i = 0; i < NVEC; ++i) {
        VecSet& v = ctx->vec[i];
        v = VecSet{};
        v.psi = dalloc<double2>(ctx, vsz, ctx->vec_allocs);
        v.th = dalloc<double2>(ctx, vsz, ctx->vec_allocs);
        v.u = dalloc<double>(ctx, ctx->nc, ctx->vec_allocs);
        if (ctx->coll) v.w = dalloc<double2>(ctx, vsz, ctx->vec_allocs);
        if (!v.psi || !v.th || !v.u || (ctx->coll && !v.w))
            return fail(ctx, PIZZA_ENOMEM, "device allocation of state vectors failed");
        CK(cudaMemset(v.psi, 0, vsz * 16));
        CK(cudaMemset(v.th, 0, vsz * 16));
        CK(cudaMemset(v.u, 0, ctx->nc * 8));
        if (v.w) CK(cudaMemset(v.w, 0, vsz * 16));
    }
    return PIZZA_OK;
}

// Ekman pumping tables for the selected formulation (StepParams pump_*): the
// exact Upsilon of Eq. pumping_full for collocation, Upsilon_eps and the
// coefficients of Eq. approx_pump for the integration method.
int set_pumping_tables(pizza_ctx* ctx) {
    StepParams& P = ctx->P;
    if (!(ctx->pump_eps > 0.0)) {
        P.pump = 0;
        return PIZZA_OK;
    }
    const int N = ctx->n_r;
    if (!ctx->pump_tab) {
        ctx->pump_tab = dalloc<double>(ctx, 3 * (size_t)N, ctx->allocs);
        ctx->pump_buf = dalloc<double2>(ctx, (size_t)ctx->M * N, ctx->allocs);
        if (!ctx->pump_tab || !ctx->pump_buf) return fail(ctx, PIZZA_ENOMEM, "device allocation failed");
    }
    std::vector<double> t(3 * (size_t)N, 0.0);
    const Geom g = make_geom(ctx->eta);
    if (ctx->coll) {
        CollGrid cg = coll_grid(N, g);
        coll_pumping(cg, g, ctx->E);
        for (int k = 0; k < N; ++k) {
            t[k] = cg.ups[k];
            t[2 * N + k] = cg.c5[k];
        }
    } else {
        const double so = g.s_o + ctx->pump_eps;
        for (int k = 0; k < N; ++k) {
            const double s = ctx->s_host[k];
            const double he2 = so * so - s * s, he = std::sqrt(he2);
            t[k] = std::sqrt(g.s_o / ctx->E) / (he * std::sqrt(he));
            t[N + k] = 1.5 * s * s / he2;
            t[2 * N + k] = 2.5 * g.s_o / he;
        }
    }
    CK(cudaMemcpy(ctx->pump_tab, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->pump_buf, 0, (size_t)ctx->M * N * sizeof(double2)));
    P.pump = 1;
    P.pump_ups = ctx->pump_tab;
    P.pump_cr = ctx->pump_tab + N;
    P.pump_ci = ctx->pump_tab + 2 * N;
    P.pump_F = ctx->pump_buf;
    return PIZZA_OK;
}

// Switch to the collocation formulation: grid tables on the device.
int enable_collocation(pizza_ctx* ctx) {
    const int N = ctx->n_r;
    CollGrid cg = coll_grid(N, make_geom(ctx->eta));
    auto& al = ctx->allocs;
    double* beta = dalloc<double>(ctx, N, al);
    double* dbeta = dalloc<double>(ctx, N, al);
    double* d1 = dalloc<double>(ctx, (size_t)N * N, al);
    double* d2 = dalloc<double>(ctx, (size_t)N * N, al);
    double* tm = dalloc<double>(ctx, (size_t)N * N, al);
    if (!beta || !dbeta || !d1 || !d2 || !tm) return fail(ctx, PIZZA_ENOMEM, "device allocation failed");
    CK(cudaMemcpy(beta, cg.beta.data(), N * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dbeta, cg.dbeta.data(), N * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d1, cg.D1.data(), (size_t)N * N * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d2, cg.D2.data(), (size_t)N * N * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tm, cg.T.data(), (size_t)N * N * 8, cudaMemcpyHostToDevice));
    ctx->P.beta = beta;
    ctx->P.dbeta = dbeta;
    ctx->P.cD1 = d1;
    ctx->P.cD2 = d2;
    ctx->P.cTm = tm;
    ctx->coll_d1_row0.assign(cg.D1.begin(), cg.D1.begin() + N);
    return PIZZA_OK;
}

// ---------------------------------------------------------------------------
// Discrete adjoint: buffers, dense inverses of the transposed tau systems,
// checkpoints and the recomputation of a segment of forward states.
// ---------------------------------------------------------------------------
VecSet adj_vec(pizza_ctx* ctx, bool& ok, bool checkpoint = false) {
    VecSet v{};
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    auto& list = checkpoint ? ctx->adj.ck_allocs : ctx->adj.allocs;
    v.psi = dalloc<double2>(ctx, vsz, list);
    v.th = dalloc<double2>(ctx, vsz, list);
    v.u = dalloc<double>(ctx, ctx->nc, list);
    if (!v.psi || !v.th || !v.u) {
        ok = false;
        return v;
    }
    ok = cudaMemset(v.psi, 0, vsz * 16) == cudaSuccess && cudaMemset(v.th, 0, vsz * 16) == cudaSuccess &&
         cudaMemset(v.u, 0, ctx->nc * 8) == cudaSuccess;
    return v;
}

int copy_vec(pizza_ctx* ctx, VecSet dst, VecSet src) {
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    CK(cudaMemcpyAsync(dst.psi, src.psi, vsz * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dst.th, src.th, vsz * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dst.u, src.u, ctx->nc * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return PIZZA_OK;
}

int zero_vec(pizza_ctx* ctx, VecSet v) {
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    CK(cudaMemsetAsync(v.psi, 0, vsz * 16, ctx->stream));
    CK(cudaMemsetAsync(v.th, 0, vsz * 16, ctx->stream));
    CK(cudaMemsetAsync(v.u, 0, ctx->nc * 8, ctx->stream));
    return PIZZA_OK;
}

// Dense P S^{-H} for gamma dt = dt/2 (the CNAB2 weight): S is the tau system of
// each field (tau rows on top), inverted by refined LU on the host; stored
// column-major without the tau rows of the output (host_ops.h, dense_inverse).
int build_adjoint_factors(pizza_ctx* ctx) {
    const int M = ctx->M, nc = ctx->nc, np = nc - 4, nt = nc - 2;
    const double gdt = 0.5 * ctx->dt;
    HostOps H = host_ops_of(ctx);
    const auto tauP = tau_rows_psi(ctx->n_r, nc);
    const auto tauD = tau_rows_dir(ctx->n_r, nc);
    auto get = [&](int id, int k, int n) -> double {
        const int h = op_h(id);
        const int d = n - k + h;
        if (d < 0 || d > 2 * h) return 0.0;
        return H.band[id][(size_t)k * (2 * h + 1) + d];
    };
    std::vector<double2> hW((size_t)M * nc * np, make_double2(0.0, 0.0));
    std::vector<double> hT((size_t)M * nc * nt), hU((size_t)nc * nt);
    std::vector<int> bad(M, 0);
    auto work = [&](int m) {
        const double mu = (double)m * m, dm = (double)m;
        if (m > 0) {
            std::vector<cplx> S((size_t)nc * nc), inv;
            for (int k = 0; k < nc; ++k)
                for (int n = 0; n < nc; ++n) {
                    cplx v;
                    if (k < 4) {
                        v = cplx(tauP[(size_t)k * nc + n], 0.0);
                    } else {
                        const double a = get(OP_A0, k, n) + mu * get(OP_A2, k, n);
                        const double b = get(OP_B0, k, n) + mu * (get(OP_B2, k, n) + mu * get(OP_B4, k, n));
                        v = cplx(a - gdt * b, -gdt * 2.0 * dm / ctx->E * get(OP_C, k, n));
                    }
                    S[(size_t)k * nc + n] = v;
                }
            if (!dense_inverse(nc, S, inv)) {
                bad[m] = 1;
                return;
            }
            // W = (S^{-1})^H rows >= 4, column-major: W[j][i-4] = conj(inv[j][i])
            for (int j = 0; j < nc; ++j)
                for (int i = 4; i < nc; ++i) {
                    const cplx c = std::conj(inv[(size_t)j * nc + i]);
                    hW[((size_t)m * nc + j) * np + (i - 4)] = make_double2(c.real(), c.imag());
                }
        }
        std::vector<double> S((size_t)nc * nc), inv;
        for (int k = 0; k < nc; ++k)
            for (int n = 0; n < nc; ++n)
                S[(size_t)k * nc + n] = (k < 2) ? tauD[(size_t)k * nc + n]
                                                : get(OP_D, k, n) - gdt * (get(OP_F0, k, n) + mu * get(OP_F2, k, n)) / ctx->Pr;
        if (!dense_inverse(nc, S, inv)) {
            bad[m] = 1;
            return;
        }
        for (int j = 0; j < nc; ++j)
            for (int i = 2; i < nc; ++i) hT[((size_t)m * nc + j) * nt + (i - 2)] = inv[(size_t)j * nc + i];
    };
    unsigned nthr = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nthr; ++t)
        th.emplace_back([&, t] {
            for (int m = (int)t; m < M; m += (int)nthr) work(m);
        });
    for (auto& t : th) t.join();
    for (int m = 0; m < M; ++m)
        if (bad[m]) return fail(ctx, PIZZA_EINVAL, "transposed tau system of mode m=%d is singular", m);
    {
        std::vector<double> S((size_t)nc * nc), inv;
        for (int k = 0; k < nc; ++k)
            for (int n = 0; n < nc; ++n)
                S[(size_t)k * nc + n] = (k < 2) ? tauD[(size_t)k * nc + n] : get(OP_D, k, n) - gdt * get(OP_EZ, k, n);
        if (!dense_inverse(nc, S, inv)) return fail(ctx, PIZZA_EINVAL, "zonal-flow tau system singular");
        for (int j = 0; j < nc; ++j)
            for (int i = 2; i < nc; ++i) hU[(size_t)j * nt + (i - 2)] = inv[(size_t)j * nc + i];
    }
    auto& al = ctx->adj.allocs;
    double2* wp = dalloc<double2>(ctx, hW.size(), al);
    double* wt = dalloc<double>(ctx, hT.size(), al);
    double* wu = dalloc<double>(ctx, hU.size(), al);
    if (!wp || !wt || !wu) return fail(ctx, PIZZA_ENOMEM, "allocation of the adjoint solves failed");
    CK(cudaMemcpy(wp, hW.data(), hW.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(wt, hT.data(), hT.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(wu, hU.data(), hU.size() * 8, cudaMemcpyHostToDevice));
    ctx->adj.A = AdjFactors{wp, wt, wu};
    return PIZZA_OK;
}

int ensure_adjoint(pizza_ctx* ctx) {
    auto& a = ctx->adj;
    if (a.ready) return PIZZA_OK;
    if (ctx->coll || ctx->P.fp32 || ctx->scheme != PIZZA_CNAB2)
        return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is implemented for CNAB2, integration, FP64");
    if (ctx->n_phi > 3072) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is limited to n_phi <= 3072");
    {
        int dev = 0, smax = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (smem_adj_grid_to_spec(ctx->P) > (size_t)smax || smem_adj_spec_to_grid(ctx->P) > (size_t)smax)
            return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint's radial kernels do not fit the device at n_r = %d",
                        ctx->n_r);
    }
    if (!ctx->dt_set) return fail(ctx, PIZZA_ESTATE, "dt is not set");
    int rc = build_adjoint_factors(ctx);
    if (rc) return rc;
    bool ok = true;
    a.lam = adj_vec(ctx, ok);
    a.rho[0] = adj_vec(ctx, ok);
    a.rho[1] = adj_vec(ctx, ok);
    a.w = adj_vec(ctx, ok);
    a.g = adj_vec(ctx, ok);
    const size_t gsz = (size_t)ctx->n_r * 4 * ctx->M;
    a.Gb1 = dalloc<double2>(ctx, gsz, a.allocs);
    a.Gb2 = dalloc<double2>(ctx, gsz, a.allocs);
    a.ra = dalloc<double>(ctx, ctx->M + 1, a.allocs);
    if (!ok || !a.Gb1 || !a.Gb2 || !a.ra) return fail(ctx, PIZZA_ENOMEM, "allocation of adjoint buffers failed");
    a.dRa_dev = a.ra + ctx->M;
    a.ready = true;
    return PIZZA_OK;
}

// after forward step number K (counted from the start of the tape): checkpoint
// y_K and E(y_{K-1}) every a.every steps
int tape_record(pizza_ctx* ctx) {
    auto& a = ctx->adj;
    a.K++;
    a.pos = a.K;
    if (a.K % a.every != 0) return PIZZA_OK;
    bool ok = true;
    VecSet y = adj_vec(ctx, ok, true), e = adj_vec(ctx, ok, true);
    if (!ok) return fail(ctx, PIZZA_ENOMEM, "allocation of a checkpoint failed");
    int rc = copy_vec(ctx, y, ctx->vec[ctx->ys[0]]);
    if (!rc) rc = copy_vec(ctx, e, ctx->vec[ctx->es[0]]);
    a.ck_y.push_back(y);
    a.ck_e.push_back(e);
    return rc;
}

// forward states y_{s*every + i} (i < every, up to K - 1) from checkpoint s
int load_segment(pizza_ctx* ctx, int s) {
    auto& a = ctx->adj;
    if (a.seg == s) return PIZZA_OK;
    bool ok = true;
    while ((int)a.seg_y.size() < a.every) {
        a.seg_y.push_back(adj_vec(ctx, ok));
        if (!ok) return fail(ctx, PIZZA_ENOMEM, "allocation of the segment states failed");
    }
    while ((int)a.seg_G1.size() < a.every - 1) {
        a.seg_G1.push_back(dalloc<double2>(ctx, (size_t)ctx->n_r * 4 * ctx->M, a.allocs));
        if (!a.seg_G1.back()) return fail(ctx, PIZZA_ENOMEM, "allocation of the segment grid fields failed");
    }
    a.seg_g1n = 0;
    const int n0 = s * a.every;
    const int n1 = std::min(n0 + a.every, a.K);  // states n0 .. n1-1
    const bool taping = a.taping;
    a.taping = false;
    reset_slots(ctx);
    int rc = copy_vec(ctx, ctx->vec[ctx->ys[0]], a.ck_y[s]);
    if (!rc && n0 > 0) rc = copy_vec(ctx, ctx->vec[ctx->es[0]], a.ck_e[s]);
    if (rc) return rc;
    ctx->n_done = n0;
    ctx->aux_valid = false;
    rc = ensure_aux(ctx);
    if (rc) return rc;
    rc = copy_vec(ctx, a.seg_y[0], ctx->vec[ctx->ys[0]]);
    double2* const g1 = ctx->G1;
    for (int n = n0 + 1; !rc && n < n1; ++n) {
        // the step's explicit stage synthesises y_{n-1}: into its slot
        ctx->G1 = a.seg_G1[n - 1 - n0];
        rc = step_multistep(ctx);
        ctx->G1 = g1;
        if (rc) break;
        ctx->n_done++;
        rc = copy_vec(ctx, a.seg_y[n - n0], ctx->vec[ctx->ys[0]]);
    }
    a.taping = taping;
    if (rc) return rc;
    a.seg_g1n = n1 - n0 - 1;
    a.seg = s;
    return PIZZA_OK;
}

// copy a caller's gradient (host or device, NULL = zero) into a.g
int load_gradient(pizza_ctx* ctx, const double* g_theta, const double* g_psi, const double* g_u) {
    auto& a = ctx->adj;
    int rc = zero_vec(ctx, a.g);
    if (rc) return rc;
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    if (g_theta) CK(cudaMemcpyAsync(a.g.th, g_theta, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (g_psi) CK(cudaMemcpyAsync(a.g.psi, g_psi, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (g_u) CK(cudaMemcpyAsync(a.g.u, g_u, ctx->nc * 8, cudaMemcpyDefault, ctx->stream));
    return PIZZA_OK;
}

}  // namespace

extern "C" {

int pizza_init(pizza_ctx** out, int n_r, int n_phi, double E, double Ra, double Pr, double radius_ratio,
               int scheme) {
    if (!out) return fail(nullptr, PIZZA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_r < 9 || !pow2(n_r - 1) || n_r > 2049)
        return fail(nullptr, PIZZA_EINVAL, "n_r must be 2^j + 1 with 9 <= n_r <= 2049 (got %d)", n_r);
    if (n_phi < 12 || n_phi % 3 != 0 || !pow2(n_phi / 3) || n_phi > 6144)
        return fail(nullptr, PIZZA_EINVAL, "n_phi must be 3*2^j with 12 <= n_phi <= 6144 (got %d)", n_phi);
    if (!(radius_ratio > 0.0 && radius_ratio < 1.0)) return fail(nullptr, PIZZA_EINVAL, "radius_ratio not in (0,1)");
    if (!(E > 0.0) || !(Pr > 0.0) || !std::isfinite(Ra)) return fail(nullptr, PIZZA_EINVAL, "E, Pr must be > 0");
    if (scheme < PIZZA_CNAB2 || scheme > PIZZA_BPR353) return fail(nullptr, PIZZA_EINVAL, "unknown scheme %d", scheme);

    pizza_ctx* ctx = new pizza_ctx();
    ctx->n_r = n_r;
    ctx->n_phi = n_phi;
    ctx->n_m = n_phi / 3;
    ctx->M = ctx->n_m + 1;
    ctx->K = n_r - 1;
    ctx->nc = (2 * (n_r - 1)) / 3;
    ctx->E = E;
    ctx->Ra = Ra;
    ctx->Pr = Pr;
    ctx->eta = radius_ratio;
    ctx->scheme = scheme;
    auto bail = [&](int rc) {
        g_init_error = ctx->err;
        pizza_free(ctx);
        return rc;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        ctx->err = "no CUDA device available";
        return bail(PIZZA_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ctx->err = "cudaStreamCreate failed";
        return bail(PIZZA_ECUDA);
    }
    ctx->stream = ctx->own_stream;

    Geom g = make_geom(radius_ratio);
    StepParams& P = ctx->P;
    P.n_r = n_r;
    P.n_phi = n_phi;
    P.n_m = ctx->n_m;
    P.M = ctx->M;
    P.nc = ctx->nc;
    P.K = ctx->K;
    P.E = E;
    P.Ra = Ra;
    P.Pr = Pr;
    P.s_o = g.s_o;
    P.inv_a = 1.0 / g.a;
    P.tc = tc_coefficient(radius_ratio);
    P.cnorm = std::sqrt(2.0 / (n_r - 1));
    P.inv_nphi = 1.0 / n_phi;

    std::vector<double> s(n_r), h2(n_r), is(n_r);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < n_r; ++k) {
        double x = (double)cosl(pi * (long double)k / (long double)(n_r - 1));
        s[k] = g.a * x + g.b;
        h2[k] = g.s_o * g.s_o - s[k] * s[k];
        is[k] = 1.0 / s[k];
    }
    h2[0] = 0.0;  // x_0 = 1 is the outer wall exactly
    ctx->s_host = s;
    ctx->ds_host.assign(n_r, 0.0);
    for (int k = 1; k + 1 < n_r; ++k) ctx->ds_host[k] = 0.5 * (s[k - 1] - s[k + 1]);
    ctx->ds_host[0] = s[0] - s[1];
    ctx->ds_host[n_r - 1] = s[n_r - 2] - s[n_r - 1];
    auto& al = ctx->allocs;
    double* ds = dalloc<double>(ctx, n_r, al);
    double* dh = dalloc<double>(ctx, n_r, al);
    double* di = dalloc<double>(ctx, n_r, al);
    if (!ds || !dh || !di) {
        ctx->err = "device allocation failed";
        return bail(PIZZA_ENOMEM);
    }
    int rc = PIZZA_OK;
    auto up = [&](void* d, const void* h, size_t bytes) {
        if (rc == PIZZA_OK && cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            ctx->err = "cudaMemcpy failed";
            rc = PIZZA_ECUDA;
        }
    };
    up(ds, s.data(), n_r * 8);
    up(dh, h2.data(), n_r * 8);
    up(di, is.data(), n_r * 8);
    P.s = ds;
    P.h2 = dh;
    P.inv_s = di;
    {
        std::vector<float> sf(n_r), hf(n_r), isf(n_r);
        for (int k = 0; k < n_r; ++k) {
            sf[k] = (float)s[k];
            hf[k] = (float)h2[k];
            isf[k] = (float)is[k];
        }
        float* fs = dalloc<float>(ctx, n_r, al);
        float* fh = dalloc<float>(ctx, n_r, al);
        float* fi = dalloc<float>(ctx, n_r, al);
        if (!fs || !fh || !fi) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(fs, sf.data(), n_r * 4);
        up(fh, hf.data(), n_r * 4);
        up(fi, isf.data(), n_r * 4);
        P.s_f = fs;
        P.h2_f = fh;
        P.inv_s_f = fi;
        // double-float copies: hi the nearest float, lo the float nearest the rest
        std::vector<float2> sd(n_r), hd(n_r), idd(n_r);
        auto split = [](double v) {
            const float h = (float)v;
            return make_float2(h, (float)(v - (double)h));
        };
        for (int k = 0; k < n_r; ++k) {
            sd[k] = split(s[k]);
            hd[k] = split(h2[k]);
            idd[k] = split(is[k]);
        }
        float2* ds2 = dalloc<float2>(ctx, n_r, al);
        float2* dh2 = dalloc<float2>(ctx, n_r, al);
        float2* di2 = dalloc<float2>(ctx, n_r, al);
        if (!ds2 || !dh2 || !di2) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(ds2, sd.data(), n_r * 8);
        up(dh2, hd.data(), n_r * 8);
        up(di2, idd.data(), n_r * 8);
        P.s_dd = ds2;
        P.h2_dd = dh2;
        P.inv_s_dd = di2;
    }

    if (!make_fft_plan(2 * ctx->K, P.plan_r) || !make_fft_plan(n_phi, P.plan_p)) {
        ctx->err = "unsupported transform length";
        return bail(PIZZA_EINVAL);
    }
    auto twr = fft_twiddles(2 * ctx->K), twp = fft_twiddles(n_phi);
    double2* dtwr = dalloc<double2>(ctx, twr.size(), al);
    double2* dtwp = dalloc<double2>(ctx, twp.size(), al);
    if (!dtwr || !dtwp) {
        ctx->err = "device allocation failed";
        return bail(PIZZA_ENOMEM);
    }
    up(dtwr, twr.data(), twr.size() * sizeof(double2));
    up(dtwp, twp.data(), twp.size() * sizeof(double2));
    P.plan_r.tw = dtwr;
    P.plan_p.tw = dtwp;
    {
        // the same twiddles rounded to FP32 for the mixed-precision explicit stage
        std::vector<float2> fr(twr.size()), fp(twp.size());
        for (size_t i = 0; i < twr.size(); ++i) fr[i] = make_float2((float)twr[i].x, (float)twr[i].y);
        for (size_t i = 0; i < twp.size(); ++i) fp[i] = make_float2((float)twp[i].x, (float)twp[i].y);
        float2* ftr = dalloc<float2>(ctx, fr.size(), al);
        float2* ftp = dalloc<float2>(ctx, fp.size(), al);
        if (!ftr || !ftp) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(ftr, fr.data(), fr.size() * sizeof(float2));
        up(ftp, fp.data(), fp.size() * sizeof(float2));
        P.plan_r.twf = ftr;
        P.plan_p.twf = ftp;
    }
    {
        // the azimuthal twiddles as double-float pairs for the double-float products
        std::vector<float4> dd(n_phi);
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int j = 0; j < n_phi; ++j) {
            const long double a = 2.0L * pi * (long double)j / (long double)n_phi;
            const long double c = cosl(a), sn = -sinl(a);
            const float ch = (float)c, sh = (float)sn;
            dd[j] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
        }
        float4* dtw = dalloc<float4>(ctx, dd.size(), al);
        if (!dtw) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(dtw, dd.data(), dd.size() * sizeof(float4));
        P.plan_p.twdd = dtw;
        P.phi_dd = 1;
    }
    P.solve_roles = -1;
    P.radial_lean = -1;
    P.psi_dd = -1;
    // half-length radial plan: its twiddles exp(-2 pi i j/K) are plan_r's at stride 2
    if (!make_fft_plan(ctx->K, P.plan_h)) {
        ctx->err = "unsupported transform length";
        return bail(PIZZA_EINVAL);
    }
    P.plan_h.tw = P.plan_r.tw;
    P.plan_h.twf = P.plan_r.twf;
    P.plan_h.tws = 2;
    {
        // the radial twiddles as double-float pairs (double-float lean transforms)
        const int L = 2 * ctx->K;
        std::vector<float4> dd(L);
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int j = 0; j < L; ++j) {
            const long double a = 2.0L * pi * (long double)j / (long double)L;
            const long double c = cosl(a), sn = -sinl(a);
            const float ch = (float)c, sh = (float)sn;
            dd[j] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
        }
        float4* dtw = dalloc<float4>(ctx, dd.size(), al);
        if (!dtw) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(dtw, dd.data(), dd.size() * sizeof(float4));
        P.plan_r.twdd = dtw;
        P.plan_h.twdd = dtw;
    }
    P.radial_dd = -1;

    // m-independent banded operators and tau rows
    HostOps H = host_ops_of(ctx);
    for (int id = 0; id < OP_COUNT; ++id) {
        double* d = dalloc<double>(ctx, H.band[id].size(), al);
        if (!d) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(d, H.band[id].data(), H.band[id].size() * 8);
        P.ops.band[id] = d;
        // the transposed operator in the same band storage: row n holds X[k][n],
        // k = n-h..n+h (used by the adjoint)
        const int h = op_h(id), W = 2 * h + 1, nc = ctx->nc;
        std::vector<double> bt((size_t)nc * W, 0.0);
        for (int n = 0; n < nc; ++n)
            for (int d2 = 0; d2 < W; ++d2) {
                const int k = n - h + d2;
                if (k >= 0 && k < nc) bt[(size_t)n * W + d2] = H.band[id][(size_t)k * W + (n - k + h)];
            }
        double* dt_ = dalloc<double>(ctx, bt.size(), al);
        if (!dt_) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(dt_, bt.data(), bt.size() * 8);
        P.ops.bandT[id] = dt_;
    }
    {
        const int nc = ctx->nc;
        auto tp = tau_rows_psi(n_r, nc), td = tau_rows_dir(n_r, nc);
        std::vector<double> bp((size_t)4 * (nc - 4)), bd((size_t)2 * (nc - 2));
        for (int r = 0; r < 4; ++r)
            for (int j = 0; j < nc - 4; ++j) bp[(size_t)r * (nc - 4) + j] = tp[(size_t)r * nc + 4 + j];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < nc - 2; ++j) bd[(size_t)r * (nc - 2) + j] = td[(size_t)r * nc + 2 + j];
        double* dp = dalloc<double>(ctx, bp.size(), al);
        double* dd = dalloc<double>(ctx, bd.size(), al);
        double* dfull = dalloc<double>(ctx, tp.size(), al);
        double* dfull2 = dalloc<double>(ctx, td.size(), al);
        if (!dp || !dd || !dfull || !dfull2) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(dp, bp.data(), bp.size() * 8);
        up(dd, bd.data(), bd.size() * 8);
        up(dfull, tp.data(), tp.size() * 8);
        up(dfull2, td.data(), td.size() * 8);
        std::vector<float> bd32(bd.begin(), bd.end());
        float* dd32 = dalloc<float>(ctx, bd32.size(), al);
        if (!dd32) {
            ctx->err = "device allocation failed";
            return bail(PIZZA_ENOMEM);
        }
        up(dd32, bd32.data(), bd32.size() * 4);
        P.ops.tau_dir_B32 = dd32;
        P.ops.tau_dir = dfull2;
        P.ops.tau_psi_B = dp;
        P.ops.tau_dir_B = dd;
        P.ops.tau_psi = dfull;
    }
    // work buffers and state vectors
    const size_t gsz = (size_t)n_r * 4 * ctx->M;
    ctx->G1 = dalloc<double2>(ctx, gsz, al);
    ctx->G2 = dalloc<double2>(ctx, gsz, al);
    if (!ctx->G1 || !ctx->G2) {
        ctx->err = "device allocation of grid buffers failed";
        return bail(PIZZA_ENOMEM);
    }
    if (rc == PIZZA_OK) rc = alloc_vecs(ctx);
    if (rc != PIZZA_OK) return bail(rc);
    reset_slots(ctx);
    *out = ctx;
    return PIZZA_OK;
}

}  // extern "C"
namespace {
int set_option_impl(pizza_ctx* ctx, const char* key, double value);
}  // namespace
extern "C" {

int pizza_set_option(pizza_ctx* ctx, const char* key, double value) {
    if (!ctx || !key) return fail(ctx, PIZZA_EINVAL, "NULL argument");
    const int rc = set_option_impl(ctx, key, value);
    if (rc == PIZZA_OK) ctx->epoch++;
    return rc;
}

}  // extern "C"

namespace {
int set_option_impl(pizza_ctx* ctx, const char* key, double value) {
    if (std::strcmp(key, "dt") == 0) {
        if (!(value > 0.0) || !std::isfinite(value)) return fail(ctx, PIZZA_EINVAL, "dt must be > 0");
        if (ctx->dt_set && value == ctx->dt) return PIZZA_OK;
        cudaStreamSynchronize(ctx->stream);
        free_factors(ctx);
        ctx->dt = value;
        ctx->dt_set = true;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "precision") == 0) {
        if (value != 0.0 && value != 1.0)
            return fail(ctx, PIZZA_EUNSUPPORTED, "precision must be 0 (FP64) or 1 (mixed: FP32 explicit stage)");
        if (value == 1.0 && ctx->coll)
            return fail(ctx, PIZZA_EUNSUPPORTED, "mixed precision is implemented for the integration formulation");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.fp32 = (value == 1.0) ? 1 : 0;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "radial") == 0) {
        if (value != 0.0 && value != 1.0 && value != 2.0)
            return fail(ctx, PIZZA_EUNSUPPORTED,
                        "radial must be 0 (collocation), 1 (integration, tau) or 2 (integration, Galerkin)");
        const bool coll = (value == 0.0), gal = (value == 2.0);
        if (coll == ctx->coll && gal == ctx->gal) return PIZZA_OK;
        if (coll && ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "slab contexts use the integration formulation");
        if (coll == ctx->coll) {  // tau <-> Galerkin: same unknowns, new factors
            cudaStreamSynchronize(ctx->stream);
            free_factors(ctx);
            ctx->gal = gal;
            return PIZZA_OK;
        }
        if (coll && ctx->P.fp32)
            return fail(ctx, PIZZA_EUNSUPPORTED, "mixed precision is implemented for the integration formulation");
        if (coll && ctx->n_r > PIZZA_COLL_MAX_NR)
            return fail(ctx, PIZZA_EUNSUPPORTED, "collocation is limited to n_r <= %d", PIZZA_COLL_MAX_NR);
        cudaStreamSynchronize(ctx->stream);
        free_factors(ctx);
        ctx->coll = coll;
        ctx->gal = gal;
        ctx->P.coll = coll ? 1 : 0;
        ctx->nc = coll ? ctx->n_r : (2 * (ctx->n_r - 1)) / 3;
        ctx->P.nc = ctx->nc;
        if (coll && !ctx->P.cD1) {
            int rc = enable_collocation(ctx);
            if (rc) return rc;
        }
        int rc = alloc_vecs(ctx);
        if (!rc) rc = set_pumping_tables(ctx);
        if (rc) return rc;
        reset_slots(ctx);
        return PIZZA_OK;
    }
    if (std::strcmp(key, "azimuthal_dd") == 0) {
        if (value != 0.0 && value != 1.0) return fail(ctx, PIZZA_EINVAL, "azimuthal_dd must be 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.phi_dd = (value == 1.0) ? 1 : 0;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "radial_lean") == 0) {
        if (value != 0.0 && value != 1.0 && value != -1.0)
            return fail(ctx, PIZZA_EINVAL, "radial_lean must be -1 (by size), 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.radial_lean = (int)value;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "solve_roles") == 0) {
        if (value != 0.0 && value != 1.0 && value != -1.0)
            return fail(ctx, PIZZA_EINVAL, "solve_roles must be -1 (by size), 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.solve_roles = (int)value;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "radial_dd") == 0) {
        if (value != 0.0 && value != 1.0 && value != -1.0)
            return fail(ctx, PIZZA_EINVAL, "radial_dd must be -1 (by size), 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.radial_dd = (int)value;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "theta_fp32") == 0) {
        if (value != 0.0 && value != 1.0 && value != -1.0)
            return fail(ctx, PIZZA_EINVAL, "theta_fp32 must be -1 (by size), 0 or 1");
        if ((int)value == ctx->theta32) return PIZZA_OK;
        cudaStreamSynchronize(ctx->stream);
        free_factors(ctx);  // the temperature factors change form
        ctx->theta32 = (int)value;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "psi_chain_dd") == 0) {
        if (value != 0.0 && value != 1.0 && value != -1.0)
            return fail(ctx, PIZZA_EINVAL, "psi_chain_dd must be -1 (by size), 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.psi_dd = (int)value;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "cfl_alpha") == 0) {
        if (!(value >= 0.0) || !std::isfinite(value)) return fail(ctx, PIZZA_EINVAL, "cfl_alpha must be >= 0");
        cudaStreamSynchronize(ctx->stream);
        if (value > 0.0 && !ctx->cfl_buf) {
            ctx->cfl_buf = dalloc<double>(ctx, 2 + ctx->n_r, ctx->allocs);
            if (!ctx->cfl_buf) return fail(ctx, PIZZA_ENOMEM, "device allocation failed");
            // local spacing of the Gauss-Lobatto grid (half the distance between
            // the two neighbours, one-sided at the walls), as the diagnostics use it
            CK(cudaMemcpy(ctx->cfl_buf + 2, ctx->ds_host.data(), ctx->n_r * sizeof(double), cudaMemcpyHostToDevice));
        }
        ctx->cfl_alpha = value;
        ctx->P.cfl_max = (value > 0.0) ? ctx->cfl_buf : nullptr;
        ctx->P.cfl_ds = ctx->cfl_buf ? ctx->cfl_buf + 2 : nullptr;
        ctx->P.cfl_dphi = 2.0 * 3.141592653589793238462643383279502884 / ctx->n_phi;
        if (ctx->cfl_buf) CK(cudaMemset(ctx->cfl_buf, 0, 2 * sizeof(double)));
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "check_finite") == 0) {
        if (value != 0.0 && value != 1.0) return fail(ctx, PIZZA_EINVAL, "check_finite must be 0 or 1");
        cudaStreamSynchronize(ctx->stream);
        if (value == 1.0 && !ctx->finite_flag) {
            ctx->finite_flag = dalloc<int>(ctx, 1, ctx->allocs);
            if (!ctx->finite_flag) return fail(ctx, PIZZA_ENOMEM, "device allocation failed");
            CK(cudaMemset(ctx->finite_flag, 0, sizeof(int)));
        }
        ctx->check_finite = (value == 1.0) ? 1 : 0;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "buoy_implicit") == 0) {
        if (value != 0.0 && value != 1.0) return fail(ctx, PIZZA_EINVAL, "buoy_implicit must be 0 or 1");
        if (ctx->adj.taping) return fail(ctx, PIZZA_ESTATE, "the buoyancy split cannot change while a tape is recorded");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.buoy_imp = (value == 1.0) ? 1 : 0;
        ctx->aux_valid = false;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "radial_batch") == 0) {
        if (value != 0.0 && value != 1.0 && value != 2.0 && value != 4.0)
            return fail(ctx, PIZZA_EINVAL, "radial_batch must be 0 (default rule), 1, 2 or 4");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.nb_r = (int)value;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "phi_threads") == 0) {
        if (value != 0.0 && value != 128.0 && value != 256.0 && value != 512.0)
            return fail(ctx, PIZZA_EINVAL, "phi_threads must be 0 (default rule), 128, 256 or 512");
        if (value > 0.0 && ctx->n_phi > 12 * (int)value)
            return fail(ctx, PIZZA_EINVAL, "phi_threads too small: at most 12 azimuthal points per thread");
        cudaStreamSynchronize(ctx->stream);
        ctx->P.phi_threads = (int)value;
        return PIZZA_OK;
    }
    if (std::strcmp(key, "pumping_eps") == 0) {
        if (!(value >= 0.0) || !std::isfinite(value) || value > 1.0)
            return fail(ctx, PIZZA_EINVAL, "pumping_eps must be in [0, 1] (0: Ekman pumping off)");
        if (ctx->adj.taping) return fail(ctx, PIZZA_ESTATE, "Ekman pumping cannot change while a tape is recorded");
        if (value == ctx->pump_eps) return PIZZA_OK;
        cudaStreamSynchronize(ctx->stream);
        free_factors(ctx);  // the collocation inverses hold the implicit pumping terms
        ctx->pump_eps = value;
        ctx->aux_valid = false;
        return set_pumping_tables(ctx);
    }
    return fail(ctx, PIZZA_EINVAL, "unknown option '%s'", key);
}
}  // namespace

extern "C" {

int pizza_set_slab(pizza_ctx* ctx, int m_lo, int m_hi, int k_lo, int k_hi, void* grid1, void* grid2,
                   pizza_exchange_fn exchange, void* user) {
    if (!ctx) return PIZZA_EINVAL;
    const bool full = (m_lo == 0 && m_hi == ctx->M && k_lo == 0 && k_hi == ctx->n_r);
    if (full && !exchange) {  // back to the whole step on this context
        cudaStreamSynchronize(ctx->stream);
        ctx->slab = pizza_ctx::Slab{};
        ctx->P.m_lo = ctx->P.m_n = ctx->P.k_lo = ctx->P.k_n = 0;
        ++ctx->epoch;
        return PIZZA_OK;
    }
    if (!(0 <= m_lo && m_lo < m_hi && m_hi <= ctx->M && 0 <= k_lo && k_lo < k_hi && k_hi <= ctx->n_r))
        return fail(ctx, PIZZA_EINVAL, "slab ranges must satisfy 0 <= m_lo < m_hi <= N_m+1, 0 <= k_lo < k_hi <= n_r");
    if (!grid1 || !grid2 || !exchange)
        return fail(ctx, PIZZA_EINVAL, "a slab needs two grid buffers and an exchange callback");
    if ((reinterpret_cast<uintptr_t>(grid1) | reinterpret_cast<uintptr_t>(grid2)) & 15)
        return fail(ctx, PIZZA_EINVAL, "grid buffers must be 16-byte aligned");
    if (ctx->coll) return fail(ctx, PIZZA_EUNSUPPORTED, "slab contexts use the integration formulation");
    if (ctx->adj.taping) return fail(ctx, PIZZA_ESTATE, "a tape is being recorded");
    cudaStreamSynchronize(ctx->stream);
    ctx->slab.on = true;
    ctx->slab.g1 = grid1;
    ctx->slab.g2 = grid2;
    ctx->slab.fn = exchange;
    ctx->slab.user = user;
    ctx->P.m_lo = m_lo;
    ctx->P.m_n = m_hi - m_lo;
    ctx->P.k_lo = k_lo;
    ctx->P.k_n = k_hi - k_lo;
    ++ctx->epoch;
    return PIZZA_OK;
}

int pizza_set_stream(pizza_ctx* ctx, void* stream) {
    if (!ctx) return PIZZA_EINVAL;
    ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own_stream;
    return PIZZA_OK;
}

int pizza_get_sizes(const pizza_ctx* ctx, int* n_r, int* n_phi, int* n_m, int* n_c) {
    if (!ctx) return PIZZA_EINVAL;
    if (n_r) *n_r = ctx->n_r;
    if (n_phi) *n_phi = ctx->n_phi;
    if (n_m) *n_m = ctx->n_m;
    if (n_c) *n_c = ctx->nc;
    return PIZZA_OK;
}

int pizza_set_state(pizza_ctx* ctx, const double* theta_hat, const double* psi_hat, const double* uphi0_hat,
                    int nc_in) {
    if (!ctx) return PIZZA_EINVAL;
    if (nc_in < 0 || nc_in > ctx->nc) return fail(ctx, PIZZA_EINVAL, "nc_in must be in [0, %d]", ctx->nc);
    reset_slots(ctx);
    if (ctx->finite_flag) CK(cudaMemsetAsync(ctx->finite_flag, 0, sizeof(int), ctx->stream));
    // collocation: coefficients go to the scratch slot, then to grid values
    VecSet y = ctx->coll ? ctx->vec[15] : ctx->vec[ctx->ys[0]];
    const size_t M = ctx->M, nc = ctx->nc;
    CK(cudaMemsetAsync(y.psi, 0, M * nc * 16, ctx->stream));
    CK(cudaMemsetAsync(y.th, 0, M * nc * 16, ctx->stream));
    CK(cudaMemsetAsync(y.u, 0, nc * 8, ctx->stream));
    if (nc_in > 0) {
        if (theta_hat)
            CK(cudaMemcpy2DAsync(y.th, nc * 16, theta_hat, (size_t)nc_in * 16, (size_t)nc_in * 16, M,
                                 cudaMemcpyDefault, ctx->stream));
        if (psi_hat && M > 1)
            CK(cudaMemcpy2DAsync(y.psi + nc, nc * 16, psi_hat + 2 * (size_t)nc_in, (size_t)nc_in * 16,
                                 (size_t)nc_in * 16, M - 1, cudaMemcpyDefault, ctx->stream));
        if (uphi0_hat) CK(cudaMemcpyAsync(y.u, uphi0_hat, (size_t)nc_in * 8, cudaMemcpyDefault, ctx->stream));
    }
    if (ctx->coll) CK(launch_coll_from_hat(ctx->P, y, ctx->vec[ctx->ys[0]], ctx->stream));
    // keep the host buffers valid only for the duration of the call
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_get_state(pizza_ctx* ctx, double* theta_hat, double* psi_hat, double* uphi0_hat) {
    if (!ctx) return PIZZA_EINVAL;
    VecSet y = ctx->vec[ctx->ys[0]];
    if (ctx->coll) {
        CK(launch_coll_to_hat(ctx->P, y, ctx->vec[15], ctx->stream));
        y = ctx->vec[15];
    }
    const size_t M = ctx->M, nc = ctx->nc;
    if (theta_hat) CK(cudaMemcpyAsync(theta_hat, y.th, M * nc * 16, cudaMemcpyDefault, ctx->stream));
    if (psi_hat) CK(cudaMemcpyAsync(psi_hat, y.psi, M * nc * 16, cudaMemcpyDefault, ctx->stream));
    if (uphi0_hat) CK(cudaMemcpyAsync(uphi0_hat, y.u, nc * 8, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_step(pizza_ctx* ctx, int nsteps) {
    if (!ctx) return PIZZA_EINVAL;
    if (nsteps < 0) return fail(ctx, PIZZA_EINVAL, "nsteps < 0");
    int rc = ensure_factors(ctx);
    if (rc) return rc;
    rc = ensure_aux(ctx);
    if (rc) return rc;
    for (int s = 0; s < nsteps; ++s) {
        if (ctx->coll)
            rc = is_multistep(ctx->scheme) ? step_multistep_coll(ctx) : step_dirk_coll(ctx);
        else
            rc = is_multistep(ctx->scheme) ? step_multistep(ctx) : step_dirk(ctx);
        if (rc) return rc;
        ctx->n_done++;
        if (ctx->check_finite) CK(launch_check_finite(ctx->P, ctx->vec[ctx->ys[0]], ctx->finite_flag, ctx->stream));
        if (ctx->nu_on) {
            CK(launch_nusselt_accumulate(ctx->P, ctx->vec[ctx->ys[0]], ctx->nu_buf + 1, ctx->nu_buf, ctx->stream));
            ctx->nu_steps++;
        }
        if (ctx->adj.taping) {
            rc = tape_record(ctx);
            if (rc) return rc;
        }
    }
    return PIZZA_OK;
}

int pizza_explicit_terms(pizza_ctx* ctx, double* e_psi, double* e_theta, double* e_uphi) {
    if (!ctx) return PIZZA_EINVAL;
    // scratch slot 15 is not used by either scheme
    VecSet e = ctx->vec[15];
    int rc = explicit_eval(ctx, ctx->vec[ctx->ys[0]], e);
    if (rc) return rc;
    const size_t M = ctx->M, nc = ctx->nc;
    if (e_psi) CK(cudaMemcpyAsync(e_psi, ctx->coll ? e.w : e.psi, M * nc * 16, cudaMemcpyDefault, ctx->stream));
    if (e_theta) CK(cudaMemcpyAsync(e_theta, e.th, M * nc * 16, cudaMemcpyDefault, ctx->stream));
    if (e_uphi) CK(cudaMemcpyAsync(e_uphi, e.u, nc * 8, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_profile_begin(pizza_ctx* ctx, unsigned mask) {
    if (!ctx) return PIZZA_EINVAL;
    ctx->prof_mask = mask & 0xFu;
    return PIZZA_OK;
}

int pizza_profile_end(pizza_ctx* ctx, double* total_ms, int* launches) {
    if (!ctx) return PIZZA_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    double t[4] = {0, 0, 0, 0};
    int n[4] = {0, 0, 0, 0};
    for (auto& r : ctx->prof) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        t[r.kernel] += ms;
        n[r.kernel] += 1;
        ctx->event_pool.push_back(r.a);
        ctx->event_pool.push_back(r.b);
    }
    ctx->prof.clear();
    ctx->prof_mask = 0;
    for (int k = 0; k < 4; ++k) {
        if (total_ms) total_ms[k] = t[k];
        if (launches) launches[k] = n[k];
    }
    return PIZZA_OK;
}

int pizza_diagnostics(pizza_ctx* ctx, pizza_diag* out) {
    if (!ctx || !out) return fail(ctx, PIZZA_EINVAL, "NULL argument");
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "diagnostics need every mode: not on a slab context");
    const int n_r = ctx->n_r, M = ctx->M, nc = ctx->nc;
    if (!ctx->diag_q) {
        // Clenshaw-Curtis weights on x_k = cos(pi k/K):
        //   w_k = (c_k/K) [1 - sum_{j=1}^{K/2} b_j cos(2 pi j k/K)/(4 j^2 - 1)],
        //   c_k = 1 at the ends, 2 inside; b_j = 1 for j = K/2, 2 otherwise;
        // times ds/dx = a and the s of the area element.
        const int K = n_r - 1;
        Geom g = make_geom(ctx->eta);
        std::vector<double> q(n_r);
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int k = 0; k <= K; ++k) {
            long double acc = 1.0L;
            for (int j = 1; j <= K / 2; ++j) {
                const long double b = (2 * j == K) ? 1.0L : 2.0L;
                acc -= b * cosl(2.0L * pi * j * k / K) / (4.0L * j * j - 1.0L);
            }
            const double c = (k == 0 || k == K) ? 1.0 : 2.0;
            q[k] = (double)(c / K * acc) * g.a * ctx->s_host[k];
        }
        ctx->diag_q = dalloc<double>(ctx, n_r, ctx->allocs);
        ctx->diag_modes = dalloc<double>(ctx, 2 * (size_t)M, ctx->allocs);
        ctx->diag_radii = dalloc<double>(ctx, 2 * (size_t)n_r, ctx->allocs);
        if (!ctx->diag_q || !ctx->diag_modes || !ctx->diag_radii)
            return fail(ctx, PIZZA_ENOMEM, "allocation of diagnostics buffers failed");
        CK(cudaMemcpy(ctx->diag_q, q.data(), n_r * sizeof(double), cudaMemcpyHostToDevice));
    }
    VecSet y = ctx->vec[ctx->ys[0]];
    StepParams P64 = ctx->P;  // diagnostics read FP64 grid fields in either precision mode
    P64.fp32 = 0;
    if (ctx->coll)
        CK(launch_coll_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    else
        CK(launch_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    CK(launch_diagnostics(P64, ctx->G1, ctx->diag_q, ctx->diag_modes, ctx->diag_radii, ctx->stream));
    std::vector<double> ms(2 * (size_t)M), rm(2 * (size_t)n_r);
    std::vector<double2> th0(nc);
    CK(cudaMemcpyAsync(ms.data(), ctx->diag_modes, ms.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(rm.data(), ctx->diag_radii, rm.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(th0.data(), y.th, nc * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double pi = 3.14159265358979323846;
    Geom g = make_geom(ctx->eta);
    double ez = pi * ms[0], ek = ez, z = 2 * pi * ms[1];
    for (int m = 1; m < M; ++m) {
        ek += 2 * pi * ms[2 * m];
        z += 4 * pi * ms[2 * m + 1];
    }
    double cs = 0.0, cp = 0.0;
    const double dphi = 2 * pi / ctx->n_phi;
    for (int k = 0; k < n_r; ++k) {
        cs = std::max(cs, rm[2 * k] / ctx->ds_host[k]);
        cp = std::max(cp, rm[2 * k + 1] / (ctx->s_host[k] * dphi));
    }
    // d theta_0/ds at s_o: (1/a) sum_n n^2 c_n, c_n = C w_n theta_hat_0n; on grid
    // values (collocation) the first row of the differentiation matrix
    double dth = 0.0;
    if (ctx->coll) {
        for (int j = 0; j < n_r; ++j) dth += ctx->coll_d1_row0[j] * th0[j].x;
    } else {
        const double C = std::sqrt(2.0 / (n_r - 1));
        for (int n = 0; n < nc; ++n) dth += (double)n * n * C * ((n == 0) ? 0.5 : 1.0) * th0[n].x;
        dth /= g.a;
    }
    const double dtc = std::log(ctx->eta) != 0.0 ? tc_coefficient(ctx->eta) / g.s_o : 0.0;
    out->E_K = ek;
    out->E_Z = ez;
    out->enstrophy = z;
    out->Nu = 1.0 + dth / dtc;
    out->Re = std::sqrt(2.0 * ek / (pi * (g.s_o * g.s_o - g.s_i * g.s_i)));
    out->Ro = out->Re * ctx->E;
    out->cfl_s = cs;
    out->cfl_phi = cp;
    bool finite = std::isfinite(ek) && std::isfinite(z) && std::isfinite(dth);
    for (double v : rm) finite = finite && std::isfinite(v);
    if (!finite) return fail(ctx, PIZZA_ENONFINITE, "the state holds NaN or infinite values");
    return PIZZA_OK;
}

int pizza_get_grid(pizza_ctx* ctx, double* us, double* uphi, double* omega, double* theta) {
    if (!ctx) return PIZZA_EINVAL;
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "the physical grid needs every mode: not on a slab context");
    const size_t n = (size_t)ctx->n_r * ctx->n_phi;
    if (!ctx->grid_out) {
        ctx->grid_out = dalloc<double>(ctx, 4 * n, ctx->allocs);
        if (!ctx->grid_out) return fail(ctx, PIZZA_ENOMEM, "allocation of the grid buffer failed");
    }
    VecSet y = ctx->vec[ctx->ys[0]];
    StepParams P64 = ctx->P;
    P64.fp32 = 0;
    if (ctx->coll)
        CK(launch_coll_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    else
        CK(launch_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    double* g = ctx->grid_out;
    CK(launch_phi_fields(P64, ctx->G1, g, g + n, g + 2 * n, g + 3 * n, ctx->stream));
    double* outs[4] = {us, uphi, omega, theta};
    for (int f = 0; f < 4; ++f)
        if (outs[f]) CK(cudaMemcpyAsync(outs[f], g + f * n, n * 8, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_tape_begin(pizza_ctx* ctx, int checkpoint_every) {
    if (!ctx) return PIZZA_EINVAL;
    if (checkpoint_every < 1) return fail(ctx, PIZZA_EINVAL, "checkpoint_every must be >= 1");
    if (ctx->n_done != 0) return fail(ctx, PIZZA_ESTATE, "the tape starts right after pizza_set_state");
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is not written for slab contexts");
    if (ctx->P.pump) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is written without Ekman pumping");
    if (ctx->P.buoy_imp) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is written for explicit buoyancy");
    int rc = ensure_factors(ctx);
    if (rc) return rc;
    rc = ensure_adjoint(ctx);
    if (rc) return rc;
    auto& a = ctx->adj;
    cudaStreamSynchronize(ctx->stream);
    for (void* p : a.ck_allocs) cudaFree(p);
    a.ck_allocs.clear();
    a.ck_y.clear();
    a.ck_e.clear();
    a.every = checkpoint_every;
    a.K = 0;
    a.pos = 0;
    a.seg = -1;
    a.seg_g1n = 0;
    CK(cudaMemsetAsync(a.dRa_dev, 0, sizeof(double), ctx->stream));
    a.rcur = 0;
    bool ok = true;
    VecSet y = adj_vec(ctx, ok, true), e = adj_vec(ctx, ok, true);
    if (!ok) return fail(ctx, PIZZA_ENOMEM, "allocation of a checkpoint failed");
    rc = copy_vec(ctx, y, ctx->vec[ctx->ys[0]]);
    if (rc) return rc;
    a.ck_y.push_back(y);
    a.ck_e.push_back(e);
    rc = zero_vec(ctx, a.lam);
    if (!rc) rc = zero_vec(ctx, a.rho[0]);
    if (!rc) rc = zero_vec(ctx, a.rho[1]);
    if (rc) return rc;
    a.taping = true;
    return PIZZA_OK;
}

int pizza_adjoint_step(pizza_ctx* ctx, const double* g_theta, const double* g_psi, const double* g_u,
                       double* dJ_dRa) {
    if (!ctx) return PIZZA_EINVAL;
    auto& a = ctx->adj;
    if (!a.ready || a.pos <= 0) return fail(ctx, PIZZA_ESTATE, "no recorded forward step left to reverse");
    a.taping = false;
    const int cur = a.pos, n = cur - 1;
    // lam <- lam + g_cur: the full adjoint of y_cur
    int rc = load_gradient(ctx, g_theta, g_psi, g_u);
    if (rc) return rc;
    CK(launch_vec_add(ctx->P, a.lam, a.g, ctx->stream));
    VecSet rho = a.rho[a.rcur], rho_next = a.rho[1 - a.rcur];
    if (cur == a.K) rc = zero_vec(ctx, rho_next);  // no step beyond y_K
    if (rc) return rc;
    // rho_n = P S^{-H} lam
    CK(launch_adj_solve(ctx->P, a.A, a.lam, rho, ctx->stream));
    // lam = (Mass + dt/2 Lin)^H rho_n,  w = dt (c rho_n - 1/2 rho_{n+1})
    const double c = (n == 0) ? 1.0 : 1.5;
    const double c2 = (cur < a.K) ? -0.5 : 0.0;
    VecSet none{};
    CK(launch_adj_apply(ctx->P, none, rho, rho_next, a.lam, a.w, ctx->dt, c, c2, ctx->stream));
    // lam += J_E(y_n)* w
    rc = load_segment(ctx, n / a.every);
    if (rc) return rc;
    const int i = n % a.every;
    VecSet y = a.seg_y[i];
    StepParams P64 = ctx->P;
    P64.fp32 = 0;
    const double2* g1 = ctx->G1;
    if (i < a.seg_g1n)
        g1 = a.seg_G1[i];  // recorded by the recomputation
    else
        CK(launch_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    CK(launch_adj_explicit(P64, a.w, y, a.lam, g1, a.Gb2, a.Gb1, a.ra, ctx->stream));
    CK(launch_ra_accumulate(a.ra, ctx->M, a.dRa_dev, ctx->stream));
    a.rcur = 1 - a.rcur;
    a.pos = n;
    if (dJ_dRa) {  // the only host synchronisation of the reverse step
        CK(cudaMemcpyAsync(dJ_dRa, a.dRa_dev, sizeof(double), cudaMemcpyDefault, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PIZZA_OK;
}

int pizza_get_adjoint(pizza_ctx* ctx, double* theta_bar, double* psi_bar, double* uphi0_bar) {
    if (!ctx) return PIZZA_EINVAL;
    auto& a = ctx->adj;
    if (!a.ready) return fail(ctx, PIZZA_ESTATE, "no adjoint has been computed");
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    if (theta_bar) CK(cudaMemcpyAsync(theta_bar, a.lam.th, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (psi_bar) CK(cudaMemcpyAsync(psi_bar, a.lam.psi, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (uphi0_bar) CK(cudaMemcpyAsync(uphi0_bar, a.lam.u, ctx->nc * 8, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_explicit_adjoint(pizza_ctx* ctx, const double* e_psi_bar, const double* e_theta_bar, const double* e_u_bar,
                           double* psi_bar, double* theta_bar, double* uphi0_bar) {
    if (!ctx) return PIZZA_EINVAL;
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is not written for slab contexts");
    if (ctx->P.pump) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is written without Ekman pumping");
    if (ctx->P.buoy_imp) return fail(ctx, PIZZA_EUNSUPPORTED, "the adjoint is written for explicit buoyancy");
    int rc = ensure_factors(ctx);
    if (rc) return rc;
    rc = ensure_adjoint(ctx);
    if (rc) return rc;
    auto& a = ctx->adj;
    rc = load_gradient(ctx, e_theta_bar, e_psi_bar, e_u_bar);
    if (!rc) rc = copy_vec(ctx, a.w, a.g);
    if (!rc) rc = zero_vec(ctx, a.g);
    if (rc) return rc;
    VecSet y = ctx->vec[ctx->ys[0]];
    StepParams P64 = ctx->P;
    P64.fp32 = 0;
    CK(launch_spec_to_grid(P64, y, ctx->G1, ctx->stream));
    CK(launch_adj_explicit(P64, a.w, y, a.g, ctx->G1, a.Gb2, a.Gb1, a.ra, ctx->stream));
    const size_t vsz = (size_t)ctx->M * ctx->nc;
    if (theta_bar) CK(cudaMemcpyAsync(theta_bar, a.g.th, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (psi_bar) CK(cudaMemcpyAsync(psi_bar, a.g.psi, vsz * 16, cudaMemcpyDefault, ctx->stream));
    if (uphi0_bar) CK(cudaMemcpyAsync(uphi0_bar, a.g.u, ctx->nc * 8, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIZZA_OK;
}

int pizza_nusselt_begin(pizza_ctx* ctx) {
    if (!ctx) return PIZZA_EINVAL;
    if (ctx->coll) return fail(ctx, PIZZA_EUNSUPPORTED, "the Nusselt weights are those of the integration state");
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "the sum needs the rank holding m = 0: not on a slab");
    if (!ctx->nu_buf) {
        ctx->nu_buf = dalloc<double>(ctx, 1 + ctx->nc, ctx->allocs);
        if (!ctx->nu_buf) return fail(ctx, PIZZA_ENOMEM, "device allocation failed");
        std::vector<double> w(1 + ctx->nc, 0.0);
        pizza_nusselt_weights(ctx, w.data() + 1);
        CK(cudaMemcpy(ctx->nu_buf, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMemsetAsync(ctx->nu_buf, 0, sizeof(double), ctx->stream));
    ctx->nu_on = true;
    ctx->nu_steps = 0;
    return PIZZA_OK;
}

int pizza_nusselt_end(pizza_ctx* ctx, double* sum, int* steps) {
    if (!ctx || !sum) return fail(ctx, PIZZA_EINVAL, "NULL argument");
    if (!ctx->nu_on) return fail(ctx, PIZZA_ESTATE, "pizza_nusselt_begin was not called");
    CK(cudaMemcpyAsync(sum, ctx->nu_buf, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (steps) *steps = ctx->nu_steps;
    ctx->nu_on = false;
    return PIZZA_OK;
}

int pizza_nusselt_weights(const pizza_ctx* ctx, double* w) {
    if (!ctx || !w) return PIZZA_EINVAL;
    if (ctx->coll) return PIZZA_EUNSUPPORTED;
    // Nu - 1 = (d theta_0/ds)(s_o)/(dT_c/ds)(s_o) = sum_n w_n Re theta_hat_0n with
    // w_n = C c_n n^2 / (a dT_c/ds(s_o)), c_0 = 1/2 (T_n'(1) = n^2, d/ds = (1/a) d/dx)
    Geom g = make_geom(ctx->eta);
    const double dtc = tc_coefficient(ctx->eta) / g.s_o;
    const double C = std::sqrt(2.0 / (ctx->n_r - 1));
    for (int n = 0; n < ctx->nc; ++n) w[n] = C * ((n == 0) ? 0.5 : 1.0) * (double)n * n / (g.a * dtc);
    return PIZZA_OK;
}

int pizza_autotune(pizza_ctx* ctx, int* nb_r, int* phi_thr) {
    if (!ctx) return PIZZA_EINVAL;
    if (ctx->coll) return fail(ctx, PIZZA_EUNSUPPORTED, "the autotuner covers the integration formulation");
    if (ctx->slab.on) return fail(ctx, PIZZA_EUNSUPPORTED, "the autotuner times whole contexts, not slabs");
    int dev = 0, smax = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int keep_nb = ctx->P.nb_r, keep_th = ctx->P.phi_threads;
    std::vector<std::pair<int, int>> cand;
    for (int nb : {1, 2, 4})
        for (int th : {128, 256, 512}) {
            if (ctx->n_phi > th * 12) continue;  // the azimuthal kernel holds 12 points per thread
            ctx->P.nb_r = nb;
            ctx->P.phi_threads = th;
            if (smem_spec_to_grid(ctx->P) > (size_t)smax || smem_grid_to_spec(ctx->P) > (size_t)smax) continue;
            cand.push_back({nb, th});
        }
    cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
    VecSet y = ctx->vec[ctx->ys[0]], e = ctx->vec[15];
    float best = 1e30f;
    std::pair<int, int> pick{keep_nb, keep_th};
    for (auto c : cand) {
        ctx->P.nb_r = c.first;
        ctx->P.phi_threads = c.second;
        int rc = explicit_eval(ctx, y, e);  // warm-up
        if (rc) return rc;
        CK(cudaEventRecord(a, ctx->stream));
        for (int r = 0; r < 5; ++r) {
            rc = explicit_eval(ctx, y, e);
            if (rc) return rc;
        }
        CK(cudaEventRecord(b, ctx->stream));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    ctx->P.nb_r = pick.first;
    ctx->P.phi_threads = pick.second;
    // the solve: one CTA per mode or one per system (explicit buoyancy, tau rows),
    // timed on a solve of the current state with the first implicit weight's
    // factors into the scratch vector
    if (!ctx->P.buoy_imp && !ctx->gal) {
        int rc = ensure_factors(ctx);
        if (rc) return rc;
        RhsSpec R{};
        R.t[R.nterms++] = {y, 1.0};
        const DevFactors& F = ctx->factors[0];
        const int keep_roles = ctx->P.solve_roles;
        float best_s = 1e30f;
        int pick_s = keep_roles;
        for (int roles : {0, 1}) {
            ctx->P.solve_roles = roles;
            CK(launch_solve(ctx->P, R, F, e, e, e, true, false, ctx->stream));  // warm-up
            CK(cudaEventRecord(a, ctx->stream));
            for (int r = 0; r < 3; ++r) CK(launch_solve(ctx->P, R, F, e, e, e, true, false, ctx->stream));
            CK(cudaEventRecord(b, ctx->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (ms < best_s) {
                best_s = ms;
                pick_s = roles;
            }
        }
        ctx->P.solve_roles = pick_s;
    }
    ctx->event_pool.push_back(a);
    ctx->event_pool.push_back(b);
    ctx->epoch++;  // launch shapes changed: batch graphs are captured anew
    if (nb_r) *nb_r = pick.first;
    if (phi_thr) *phi_thr = pick.second;
    return PIZZA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many contexts advanced by one CUDA graph.  The step sequences of all
// contexts are captured on their own streams, forked from and joined to the
// batch's stream, so independent runs execute concurrently on the GPU.  A graph
// is kept with the slot state (rings, step count) of every context at its start
// and end, and relaunched when the contexts are back in its start state.
// ---------------------------------------------------------------------------
namespace {
struct Snap {
    int ys[4], es[4], ms[3], is[3], n_done;
    bool aux_valid;
    unsigned epoch;
    bool same_start(const pizza_ctx* c) const {
        if (std::memcmp(ys, c->ys, sizeof ys) || std::memcmp(es, c->es, sizeof es) || std::memcmp(ms, c->ms, sizeof ms) ||
            std::memcmp(is, c->is, sizeof is) || aux_valid != c->aux_valid || epoch != c->epoch)
            return false;
        // the coefficients depend on the step count only during the start-up steps
        return n_done == c->n_done || (n_done >= 3 && c->n_done >= 3);
    }
};
Snap snap_of(const pizza_ctx* c) {
    Snap s;
    std::memcpy(s.ys, c->ys, sizeof s.ys);
    std::memcpy(s.es, c->es, sizeof s.es);
    std::memcpy(s.ms, c->ms, sizeof s.ms);
    std::memcpy(s.is, c->is, sizeof s.is);
    s.n_done = c->n_done;
    s.aux_valid = c->aux_valid;
    s.epoch = c->epoch;
    return s;
}
void restore_snap(pizza_ctx* c, const Snap& s, int n_done) {
    std::memcpy(c->ys, s.ys, sizeof s.ys);
    std::memcpy(c->es, s.es, sizeof s.es);
    std::memcpy(c->ms, s.ms, sizeof s.ms);
    std::memcpy(c->is, s.is, sizeof s.is);
    c->aux_valid = s.aux_valid;
    c->n_done = n_done;
}
}  // namespace

struct pizza_batch {
    std::vector<pizza_ctx*> ctxs;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = 0;
    std::vector<Snap> start, end;
};

namespace {
int batch_fail(int code, const char* msg) {
    set_global_error(msg);
    return code;
}
int step_one(pizza_ctx* ctx) {
    int rc;
    if (ctx->coll)
        rc = is_multistep(ctx->scheme) ? step_multistep_coll(ctx) : step_dirk_coll(ctx);
    else
        rc = is_multistep(ctx->scheme) ? step_multistep(ctx) : step_dirk(ctx);
    if (!rc) ctx->n_done++;
    if (!rc && ctx->check_finite &&
        launch_check_finite(ctx->P, ctx->vec[ctx->ys[0]], ctx->finite_flag, ctx->stream) != cudaSuccess)
        rc = PIZZA_ECUDA;
    return rc;
}
}  // namespace

extern "C" {

int pizza_batch_create(pizza_batch** out, pizza_ctx* const* ctxs, int n) {
    if (!out || !ctxs || n < 1) return batch_fail(PIZZA_EINVAL, "pizza_batch_create: invalid arguments");
    *out = nullptr;
    pizza_batch* b = new pizza_batch();
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) {
            delete b;
            return batch_fail(PIZZA_EINVAL, "pizza_batch_create: NULL context");
        }
        if (ctxs[i]->adj.taping) {
            delete b;
            return batch_fail(PIZZA_ESTATE, "pizza_batch_create: a context is recording a tape");
        }
        if (ctxs[i]->slab.on) {
            delete b;
            return batch_fail(PIZZA_EUNSUPPORTED, "pizza_batch_create: slab contexts exchange through callbacks");
        }
        b->ctxs.push_back(ctxs[i]);
    }
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        pizza_batch_free(b);
        return batch_fail(PIZZA_ECUDA, "pizza_batch_create: stream or event creation failed");
    }
    b->joins.resize(n);
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) != cudaSuccess) {
            pizza_batch_free(b);
            return batch_fail(PIZZA_ECUDA, "pizza_batch_create: event creation failed");
        }
    *out = b;
    return PIZZA_OK;
}

int pizza_batch_step(pizza_batch* b, int nsteps) {
    if (!b || nsteps < 0) return batch_fail(PIZZA_EINVAL, "pizza_batch_step: invalid arguments");
    if (nsteps == 0) return PIZZA_OK;
    const int n = (int)b->ctxs.size();
    // set-up outside the graph: factors, first mass/implicit terms; then order the
    // batch stream after everything already queued on the contexts' streams
    for (int i = 0; i < n; ++i) {
        pizza_ctx* c = b->ctxs[i];
        int rc = ensure_factors(c);
        if (!rc) rc = ensure_aux(c);
        if (rc) return batch_fail(rc, c->err.c_str());
        if (cudaEventRecord(b->joins[i], c->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->joins[i], 0) != cudaSuccess)
            return batch_fail(PIZZA_ECUDA, "pizza_batch_step: event ordering failed");
    }
    bool reuse = b->exec && b->graph_steps == nsteps;
    for (int i = 0; reuse && i < n; ++i) reuse = b->start[i].same_start(b->ctxs[i]);
    if (!reuse) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->start.assign(n, Snap{});
        b->end.assign(n, Snap{});
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return batch_fail(PIZZA_ECUDA, "pizza_batch_step: stream capture failed to start");
        int rc = PIZZA_OK;
        if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) rc = PIZZA_ECUDA;
        for (int i = 0; !rc && i < n; ++i) {
            pizza_ctx* c = b->ctxs[i];
            if (cudaStreamWaitEvent(c->stream, b->fork, 0) != cudaSuccess) {
                rc = PIZZA_ECUDA;
                break;
            }
            b->start[i] = snap_of(c);
            for (int s = 0; !rc && s < nsteps; ++s) rc = step_one(c);
            b->end[i] = snap_of(c);
            if (!rc && (cudaEventRecord(b->joins[i], c->stream) != cudaSuccess ||
                        cudaStreamWaitEvent(b->stream, b->joins[i], 0) != cudaSuccess))
                rc = PIZZA_ECUDA;
        }
        const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
        if (rc || ec != cudaSuccess || !graph) {
            // the captured sequence did not run: put the contexts back
            for (int i = 0; i < n; ++i)
                if (b->start.size() > (size_t)i) restore_snap(b->ctxs[i], b->start[i], b->start[i].n_done);
            if (graph) cudaGraphDestroy(graph);
            return batch_fail(rc ? rc : PIZZA_ECUDA, "pizza_batch_step: capture of the step sequence failed");
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            for (int i = 0; i < n; ++i) restore_snap(b->ctxs[i], b->start[i], b->start[i].n_done);
            b->exec = nullptr;
            return batch_fail(PIZZA_ECUDA, "pizza_batch_step: graph instantiation failed");
        }
        b->graph_steps = nsteps;
        // the capture advanced the host bookkeeping; undo it, the launch below redoes it
        for (int i = 0; i < n; ++i) restore_snap(b->ctxs[i], b->start[i], b->start[i].n_done);
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess)
        return batch_fail(PIZZA_ECUDA, "pizza_batch_step: graph launch failed");
    for (int i = 0; i < n; ++i) {
        pizza_ctx* c = b->ctxs[i];
        restore_snap(c, b->end[i], c->n_done + nsteps);
    }
    // later work on any context's stream waits for the graph
    if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return batch_fail(PIZZA_ECUDA, "event record failed");
    for (int i = 0; i < n; ++i)
        if (cudaStreamWaitEvent(b->ctxs[i]->stream, b->done, 0) != cudaSuccess)
            return batch_fail(PIZZA_ECUDA, "pizza_batch_step: event ordering failed");
    return PIZZA_OK;
}

void* pizza_batch_stream(pizza_batch* b) { return b ? b->stream : nullptr; }

void pizza_batch_free(pizza_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int pizza_synchronize(pizza_ctx* ctx) {
    if (!ctx) return PIZZA_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    if (ctx->finite_flag) {
        int f = 0;
        CK(cudaMemcpy(&f, ctx->finite_flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (f) return fail(ctx, PIZZA_ENONFINITE, "a NaN or infinite value appeared in the state");
    }
    if (ctx->cfl_alpha > 0.0) {
        double r[2] = {0.0, 0.0};
        CK(cudaMemcpy(r, ctx->cfl_buf, sizeof r, cudaMemcpyDeviceToHost));
        CK(cudaMemset(ctx->cfl_buf, 0, sizeof r));
        const double rate = std::max(r[0], r[1]);
        if (rate > 0.0 && ctx->dt * rate > ctx->cfl_alpha)
            return fail(ctx, PIZZA_ECFL,
                        "Courant criterion (Eq. cfl) exceeded: dt = %.6g > alpha / max(|u_s|/ds, |u_phi|/(s dphi)) = "
                        "%.6g (alpha %.3g, rates %.17g, %.17g)",
                        ctx->dt, ctx->cfl_alpha / rate, ctx->cfl_alpha, r[0], r[1]);
    }
    return PIZZA_OK;
}

int pizza_host_operator(int which, int n_r, int n_c, double radius_ratio, double* out) {
    if (which < 0 || which >= OP_COUNT || n_r < 3 || n_c < 5 || n_c > n_r || !out ||
        !(radius_ratio > 0 && radius_ratio < 1))
        return fail(nullptr, PIZZA_EINVAL, "invalid arguments to pizza_host_operator");
    auto M = build_operator(which, n_r, n_c, make_geom(radius_ratio));
    std::memcpy(out, M.data(), M.size() * sizeof(double));
    return PIZZA_OK;
}

int pizza_host_collocation(int which, int n_r, double radius_ratio, double E, double Pr, int m, double gdt,
                           double* out) {
    if (which < 0 || which > 4 || n_r < 5 || n_r > PIZZA_COLL_MAX_NR || !out || !(radius_ratio > 0 && radius_ratio < 1) ||
        m < 0 || (which == 0 && m < 1) || !(E > 0) || !(Pr > 0))
        return fail(nullptr, PIZZA_EINVAL, "invalid arguments to pizza_host_collocation");
    CollGrid cg = coll_grid(n_r, make_geom(radius_ratio));
    if (which == 0) {
        std::vector<cplx> G;
        if (!coll_inverse_wpsi(cg, E, m, gdt, G)) return fail(nullptr, PIZZA_EINVAL, "singular system");
        std::memcpy(out, G.data(), G.size() * sizeof(cplx));
    } else if (which <= 2) {
        std::vector<double> G;
        const bool ok = (which == 1) ? coll_inverse_dir(cg, 1.0 / Pr, (double)m * m, gdt, G)
                                     : coll_inverse_dir(cg, 1.0, 1.0, gdt, G);
        if (!ok) return fail(nullptr, PIZZA_EINVAL, "singular system");
        std::memcpy(out, G.data(), G.size() * sizeof(double));
    } else {
        const auto& D = (which == 3) ? cg.D1 : cg.D2;
        std::memcpy(out, D.data(), D.size() * sizeof(double));
    }
    return PIZZA_OK;
}

void pizza_free(pizza_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_factors(ctx);
    for (auto& r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFree(p);
    for (void* p : ctx->vec_allocs) cudaFree(p);
    for (void* p : ctx->adj.allocs) cudaFree(p);
    for (void* p : ctx->adj.ck_allocs) cudaFree(p);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

const char* pizza_last_error(const pizza_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

}  // extern "C"
