// pizza_explicit_terms_noalloc: the explicit stage of the time step for callers
// that cannot allocate device memory.  Everything the three explicit kernels
// need beyond the caller's input and output arrays lives in file-scope static
// device arrays of fixed size:
//   g_scratch  the two radius-major intermediate arrays (grid-space Fourier
//              coefficients of the four fields, and of the four products);
//   g_tables   radial grid, FFT twiddles and the banded integration operators.
// Size limit: n_r <= 257 and n_phi <= 768 (8.5 MB of scratch, 0.2 MB of tables,
// held by every device that loads the library until the process exits).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pizza.h"
#include "pizza_internal.h"

namespace pz {
namespace {

constexpr int NA_MAX_NR = PIZZA_NOALLOC_MAX_NR;
constexpr int NA_MAX_NPHI = PIZZA_NOALLOC_MAX_NPHI;
constexpr int NA_MAX_M = NA_MAX_NPHI / 3 + 1;
constexpr int NA_MAX_NC = (2 * (NA_MAX_NR - 1)) / 3;
constexpr size_t NA_GRID = (size_t)NA_MAX_NR * 4 * NA_MAX_M;  // one radius-major array (double2)

// band widths 2h+1 of the operators, in the order of enum OpId
constexpr int NA_WIDTH[OP_COUNT] = {17, 17, 13, 13, 13, 17, 9, 5, 5, 5, 9};
constexpr size_t na_band_total() {
    size_t t = 0;
    for (int i = 0; i < OP_COUNT; ++i) t += (size_t)NA_MAX_NC * NA_WIDTH[i];
    return t;
}
// tables, in doubles, each section starting on a 256-byte boundary (32 doubles):
// s, h2, 1/s (3 * NA_MAX_NR), twiddles for 2(n_r-1) and n_phi (double2), bands
constexpr size_t na_round(size_t n) { return (n + 31) / 32 * 32; }
constexpr size_t NA_TAB_GRID = na_round(3 * (size_t)NA_MAX_NR);
constexpr size_t NA_TAB_TWR = na_round(2 * 2 * (size_t)(NA_MAX_NR - 1));
constexpr size_t NA_TAB_TWP = na_round(2 * (size_t)NA_MAX_NPHI);
constexpr size_t NA_TAB_TW = NA_TAB_TWR + NA_TAB_TWP;
constexpr size_t NA_TABLES = NA_TAB_GRID + NA_TAB_TW + na_band_total();
static_assert(NA_TAB_GRID % 2 == 0 && NA_TAB_TWR % 2 == 0, "double2 tables must be 16-byte aligned");

static __device__ __align__(256) double2 g_scratch[2 * NA_GRID];
static __device__ __align__(256) double g_tables[NA_TABLES];

constexpr int NA_MAX_DEVICES = 64;

struct DeviceSlot {
    bool ready = false;       // symbol addresses resolved
    double2* scratch = nullptr;
    double* tables = nullptr;
    bool have_params = false;  // tables hold the parameters below
    int n_r = 0, n_phi = 0;
    double eta = 0;  // Ra and Pr enter the kernels by value, not through the tables
};

DeviceSlot g_slots[NA_MAX_DEVICES];
std::mutex g_lock;

int na_fail(int code, const char* msg) {
    set_global_error(msg);
    return code;
}

// Set-up on the current device: resolve the device addresses of the static
// arrays (once per device) and (re)write the tables when (n_r, n_phi, eta)
// change.  A rewrite first waits for the whole device, so that no call queued
// earlier (on this stream or another) still reads the old tables, then copies
// on the caller's stream and waits for that copy.
int na_setup(int dev, int n_r, int n_phi, double eta, cudaStream_t st, DeviceSlot*& out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(PIZZA_EINVAL, "device index beyond the supported range");
    DeviceSlot& sl = g_slots[dev];
    if (!sl.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return na_fail(PIZZA_ECUDA, "cudaGetSymbolAddress(scratch) failed");
        sl.scratch = static_cast<double2*>(p);
        e = cudaGetSymbolAddress(&p, g_tables);
        if (e != cudaSuccess) return na_fail(PIZZA_ECUDA, "cudaGetSymbolAddress(tables) failed");
        sl.tables = static_cast<double*>(p);
        sl.ready = true;
    }
    if (!(sl.have_params && sl.n_r == n_r && sl.n_phi == n_phi && sl.eta == eta)) {
        sl.have_params = false;  // stays false unless the whole upload succeeds
        const int nc = (2 * (n_r - 1)) / 3;
        std::vector<double> host(NA_TABLES, 0.0);
        Geom g = make_geom(eta);
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int k = 0; k < n_r; ++k) {
            double x = (double)cosl(pi * (long double)k / (long double)(n_r - 1));
            double s = g.a * x + g.b;
            host[k] = s;
            host[NA_MAX_NR + k] = (k == 0) ? 0.0 : g.s_o * g.s_o - s * s;
            host[2 * NA_MAX_NR + k] = 1.0 / s;
        }
        auto twr = fft_twiddles(2 * (n_r - 1));
        auto twp = fft_twiddles(n_phi);
        std::memcpy(&host[NA_TAB_GRID], twr.data(), twr.size() * sizeof(double2));
        std::memcpy(&host[NA_TAB_GRID + NA_TAB_TWR], twp.data(), twp.size() * sizeof(double2));
        size_t off = NA_TAB_GRID + NA_TAB_TW;
        for (int id = 0; id < OP_COUNT; ++id) {
            if (2 * op_h(id) + 1 != NA_WIDTH[id])
                return na_fail(PIZZA_EINVAL, "operator band width differs from the static table layout");
            auto b = to_band(build_operator(id, n_r, nc, g), nc, op_h(id));
            if (b.size() != (size_t)nc * NA_WIDTH[id])
                return na_fail(PIZZA_EINVAL, "operator band size differs from the static table layout");
            std::memcpy(&host[off], b.data(), b.size() * sizeof(double));
            off += (size_t)NA_MAX_NC * NA_WIDTH[id];
        }
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return na_fail(PIZZA_ECUDA, cudaGetErrorString(e));
        e = cudaMemcpyAsync(sl.tables, host.data(), NA_TABLES * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return na_fail(PIZZA_ECUDA, "copy of the tables into static device memory failed");
        sl.n_r = n_r;
        sl.n_phi = n_phi;
        sl.eta = eta;
        sl.have_params = true;
    }
    out = &sl;
    return PIZZA_OK;
}

}  // namespace
}  // namespace pz

using namespace pz;

extern "C" int pizza_explicit_terms_noalloc(int n_r, int n_phi, double Ra, double Pr, double radius_ratio,
                                            const double* psi_hat, const double* theta_hat,
                                            const double* uphi0_hat, double* e_psi, double* e_theta,
                                            double* e_uphi, void* stream) {
    if (n_r < 9 || ((n_r - 1) & (n_r - 2)) != 0 || n_phi < 12 || n_phi % 3 != 0 ||
        ((n_phi / 3) & (n_phi / 3 - 1)) != 0)
        return na_fail(PIZZA_EINVAL, "n_r must be 2^j + 1 >= 9 and n_phi 3*2^j >= 12");
    if (n_r > NA_MAX_NR || n_phi > NA_MAX_NPHI)
        return na_fail(PIZZA_EINVAL,
                       "sizes exceed the static scratch of pizza_explicit_terms_noalloc "
                       "(n_r <= PIZZA_NOALLOC_MAX_NR = 257, n_phi <= PIZZA_NOALLOC_MAX_NPHI = 768)");
    if (!(radius_ratio > 0.0 && radius_ratio < 1.0) || !(Pr > 0.0) || !std::isfinite(Ra))
        return na_fail(PIZZA_EINVAL, "invalid physical parameters");
    if (!psi_hat || !theta_hat || !uphi0_hat || !e_psi || !e_theta || !e_uphi)
        return na_fail(PIZZA_EINVAL, "NULL array argument");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(PIZZA_ECUDA, "no CUDA device available");

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> guard(g_lock);
    DeviceSlot* sl = nullptr;
    int rc = na_setup(dev, n_r, n_phi, radius_ratio, st, sl);
    if (rc != PIZZA_OK) return rc;

    Geom g = make_geom(radius_ratio);
    StepParams P{};
    P.n_r = n_r;
    P.n_phi = n_phi;
    P.n_m = n_phi / 3;
    P.M = P.n_m + 1;
    P.nc = (2 * (n_r - 1)) / 3;
    P.K = n_r - 1;
    P.E = 1.0;  // not used by the explicit stage
    P.Ra = Ra;
    P.Pr = Pr;
    P.s_o = g.s_o;
    P.inv_a = 1.0 / g.a;
    P.tc = tc_coefficient(radius_ratio);
    P.cnorm = std::sqrt(2.0 / (n_r - 1));
    P.inv_nphi = 1.0 / n_phi;
    P.s = sl->tables;
    P.h2 = sl->tables + NA_MAX_NR;
    P.inv_s = sl->tables + 2 * NA_MAX_NR;
    if (!make_fft_plan(2 * P.K, P.plan_r) || !make_fft_plan(n_phi, P.plan_p))
        return na_fail(PIZZA_EINVAL, "unsupported transform length");
    P.plan_r.tw = reinterpret_cast<const double2*>(sl->tables + NA_TAB_GRID);
    if (!make_fft_plan(P.K, P.plan_h)) return na_fail(PIZZA_EINVAL, "unsupported transform length");
    P.plan_h.tw = P.plan_r.tw;  // exp(-2 pi i j/K) = plan_r's twiddles at stride 2
    P.plan_h.tws = 2;
    P.plan_p.tw = reinterpret_cast<const double2*>(sl->tables + NA_TAB_GRID + NA_TAB_TWR);
    size_t off = NA_TAB_GRID + NA_TAB_TW;
    for (int id = 0; id < OP_COUNT; ++id) {
        P.ops.band[id] = sl->tables + off;
        off += (size_t)NA_MAX_NC * NA_WIDTH[id];
    }
    P.ops.tau_psi_B = nullptr;  // the explicit stage uses no tau rows
    P.ops.tau_dir_B = nullptr;

    // the grid arrays are sized for the actual problem inside the static scratch
    double2* G1 = sl->scratch;
    double2* G2 = sl->scratch + NA_GRID;
    VecSet y{const_cast<double2*>(reinterpret_cast<const double2*>(psi_hat)),
             const_cast<double2*>(reinterpret_cast<const double2*>(theta_hat)), const_cast<double*>(uphi0_hat)};
    VecSet e{reinterpret_cast<double2*>(e_psi), reinterpret_cast<double2*>(e_theta), e_uphi};
    cudaError_t err = launch_spec_to_grid(P, y, G1, st);
    if (err == cudaSuccess) err = launch_phi_products(P, G1, G2, st);
    if (err == cudaSuccess) err = launch_grid_to_spec(P, G2, y, e, st);
    if (err != cudaSuccess) return na_fail(PIZZA_ECUDA, cudaGetErrorString(err));
    return PIZZA_OK;
}
