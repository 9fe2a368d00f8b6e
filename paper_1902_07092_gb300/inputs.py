"""Seeded synthetic initial states.  Shared by the tests and the benchmark; holds
none of the method's arithmetic.

Random numbers come from the SplitMix64 output function (Steele, Lea & Flood
2014) applied to a counter: u(seed, stream, i) = mix(seed * G + stream * H + i * G)
mapped to [-1, 1) with the top 53 bits.

Initial temperature perturbation, per mode m in [m_min, N_m]:
    theta_m(x) = A sum_{n=0}^{min(N_c-3, 15)} (u1 + i u2)/(1+n)^2 (T_{n+2}(x) - T_n(x))
(the Dirichlet basis T_{n+2} - T_n vanishes at both walls), u1, u2 from the
counter above with stream = (cfg, m, n), imaginary part dropped for m = 0.
Returned in the coefficient convention of the C interface (Eq. cheb):
f_hat_n = c_n / (C w_n), C = sqrt(2/(n_r-1)), w_0 = 1/2 (and w_{n_r-1} = 1/2).
The streamfunction and zonal flow start at zero.
"""
import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_H = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed, stream, counter):
    """U[-1, 1) draws; broadcasting over integer arrays ``stream``/``counter``."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed) * _G
        z = s + np.asarray(stream, dtype=np.uint64) * _H + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _G
        r = _mix(z)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def n_c_integration(n_r):
    return (2 * (n_r - 1)) // 3


def theta_init(n_r, n_phi, amp, seed, cfg=0, m_min=1, n_c=None, n_terms=16):
    """Initial theta_hat, complex array [N_m + 1][n_c]."""
    if n_c is None:
        n_c = n_c_integration(n_r)
    n_m = n_phi // 3
    M = n_m + 1
    nt = min(n_c - 2, n_terms)
    m = np.arange(M)[:, None]
    n = np.arange(nt)[None, :]
    stream = (np.uint64(cfg) << np.uint64(40)) + (m.astype(np.uint64) << np.uint64(20)) + n.astype(np.uint64)
    u1 = uniform(seed, stream, 0)
    u2 = uniform(seed, stream, 1)
    a = amp * (u1 + 1j * u2) / (1.0 + n) ** 2
    a[0] = a[0].real
    a[:m_min] = 0.0
    c = np.zeros((M, n_c), np.complex128)
    c[:, 2:nt + 2] += a
    c[:, :nt] -= a
    w = np.ones(n_c)
    w[0] = 0.5
    if n_c >= n_r:
        w[n_r - 1] = 0.5
    return c / (np.sqrt(2.0 / (n_r - 1)) * w)[None, :]


def zero_state(n_r, n_phi, n_c=None):
    if n_c is None:
        n_c = n_c_integration(n_r)
    M = n_phi // 3 + 1
    return np.zeros((M, n_c), np.complex128), np.zeros(n_c)


# The workloads (sizes, physical parameters, schemes, radial formulation); Ra is
# given as a multiple of the critical Rayleigh number at (E, Pr = 1, eta = 0.35).
# "radial": "collocation" (Section 3.1, N_c = n_r), "integration" (Section 3.2,
# N_c = floor(2 (n_r - 1)/3), tau rows) or "galerkin" (the same with the Galerkin
# bases of Appendix B).
WORKLOADS = {
    "coll_n33_p96": dict(n_r=33, n_phi=96, E=1e-3, Pr=1.0, eta=0.35, ra_factor=2.0, scheme="CNAB2",
                         dt=1e-4, steps=100, amp=1e-4, seed=1, cfg=1, radial="collocation"),
    "int_n33_p96": dict(n_r=33, n_phi=96, E=1e-3, Pr=1.0, eta=0.35, ra_factor=2.0, scheme="CNAB2",
                        dt=1e-4, steps=100, amp=1e-4, seed=1, cfg=1, radial="integration"),
    "sparse_n257_p768": dict(n_r=257, n_phi=768, E=1e-5, Pr=1.0, eta=0.35, ra_factor=10.0, scheme="ARS443",
                             dt=1e-7, steps=1000, amp=1e-3, seed=2, cfg=2, radial="integration"),
    "galerkin_n257_p768": dict(n_r=257, n_phi=768, E=1e-5, Pr=1.0, eta=0.35, ra_factor=10.0, scheme="ARS443",
                               dt=1e-7, steps=1000, amp=1e-3, seed=2, cfg=2, radial="galerkin"),
    "coll_n257_p768": dict(n_r=257, n_phi=768, E=1e-5, Pr=1.0, eta=0.35, ra_factor=10.0, scheme="ARS443",
                           dt=1e-7, steps=1000, amp=1e-3, seed=2, cfg=2, radial="collocation"),
    "large_n2049_p6144": dict(n_r=2049, n_phi=6144, E=1e-8, Pr=1.0, eta=0.35, ra_factor=20.0, scheme="SBDF3",
                              dt=1e-10, steps=50, amp=1e-3, seed=3, cfg=3, radial="integration"),
    "batch64": dict(n_r=0, n_phi=0, E=0.0, Pr=1.0, eta=0.35, ra_factor=0.0, scheme="CNAB2", dt=0.0, steps=200,
                    amp=1e-3, seed=1000, cfg=4, radial="integration", batch=64),
    "adjoint_n257_p768": dict(n_r=257, n_phi=768, E=1e-5, Pr=1.0, eta=0.35, ra_factor=5.0, scheme="CNAB2",
                              dt=1e-7, steps=400, amp=1e-3, seed=5, cfg=5, radial="integration",
                              adjoint=True, checkpoint_every=20),
}


def batch_runs(n=64):
    """The batched workload: run r (seed 1000 + r) draws n_r and n_phi independently
    from {65, 129, 257, 513} x {192, 384, 768, 1536}, E log-uniform in [1e-6, 1e-4]
    and Ra/Ra_c uniform in [1.5, 20]; CNAB2 with dt = 0.01 E, integration/tau,
    perturbation amplitude 1e-3."""
    sizes_r = (65, 129, 257, 513)
    sizes_p = (192, 384, 768, 1536)
    runs = []
    for r in range(n):
        u = (uniform(1000 + r, 7, np.arange(4)) + 1.0) * 0.5      # U[0, 1)
        E = 10.0 ** (-6.0 + 2.0 * u[2])
        runs.append(dict(n_r=sizes_r[min(3, int(4 * u[0]))], n_phi=sizes_p[min(3, int(4 * u[1]))], E=float(E),
                         ra_factor=float(1.5 + 18.5 * u[3]), Pr=1.0, eta=0.35, scheme="CNAB2", dt=float(0.01 * E),
                         amp=1e-3, seed=1000 + r, cfg=4))
    return runs


def n_c_of(wl):
    """Coefficients per mode of a workload's formulation."""
    return wl["n_r"] if wl.get("radial") == "collocation" else n_c_integration(wl["n_r"])
