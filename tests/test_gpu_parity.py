"""GPU parity: the CUDA path, called through the C interface, against the
oracle on the same seeded inputs.

Tolerances (relative L2, FP64): explicit right-hand sides max(1e-12, 4 n_r^2 eps)
with eps = 2^-53 (the flux divergence differentiates the interpolant of rounded
grid products; the derivative of T_n is bounded by n^2, so rounding errors of the
two implementations are amplified by up to n_r^2); full time
steps 1e-12 at n_r <= 65 and 2e-12 at n_r = 257, where the unpivoted banded
solve and the oracle's dense LU each sit ~1e-12 from the exact solution of the
tau system (measured against iteratively refined solutions: the streamfunction
block has an effective condition number ~1e4)."""
import numpy as np
import pytest

from oracle.explicit import explicit_terms
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import assert_state_close, critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu


def make_pair(n_r, n_phi, E, ra_factor, scheme, dt, Pr=1.0, eta=0.35):
    from paper_1902_07092_gb300.binding import Solver
    Ra = ra_factor * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, Pr, eta, scheme, dt)
    ora = IntegrationStepper(n_r, n_phi, E, Ra, Pr, eta, scheme, dt)
    return gpu, ora


def random_state(n_r, n_phi, amp, seed, psi_amp=None, u_amp=None):
    th = inputs.theta_init(n_r, n_phi, amp, seed, cfg=7, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, psi_amp if psi_amp is not None else amp * 1e-2, seed + 1, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, u_amp if u_amp is not None else amp, seed + 2, cfg=9, m_min=0)[0].real
    return psi, th, u


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (65, 192), (129, 384), (257, 768)])
def test_explicit_terms_match_oracle(n_r, n_phi):
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    psi, th, u = random_state(n_r, n_phi, 1.0, 3, psi_amp=1.0, u_amp=1.0)
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    print("explicit terms n_r=%d: rel L2 psi %.2e theta %.2e u %.2e (tol %.1e)" % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_steps_match_oracle_tiny(scheme, amp):
    """configs: n_r = 33, n_phi = 96, E = 1e-3, Pr = 1, Ra = 2 Ra_c, dt = 1e-4;
    amp = 1e-4 is the tiny workload, amp = 1 the strongly nonlinear case."""
    n_r, n_phi = 33, 96
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4)
    th = inputs.theta_init(n_r, n_phi, amp, 1, cfg=1)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for k in range(5):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    gpu.close()


def test_steps_match_oracle_sparse_workload():
    """n_r = 257, n_phi = 768, E = 1e-5, Pr = 1, Ra = 10 Ra_c, ARS443, dt = 1e-7,
    seeded amplitude 1e-3; two steps."""
    n_r, n_phi = 257, 768
    gpu, ora = make_pair(n_r, n_phi, 1e-5, 10.0, "ARS443", 1e-7)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 2, cfg=2)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for k in range(2):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 2e-12, oracle=ora)
    gpu.close()


def test_multistep_history_across_calls():
    """pizza_step(ctx, 3) equals three pizza_step(ctx, 1) calls (history kept)."""
    n_r, n_phi = 33, 96
    from paper_1902_07092_gb300.binding import Solver
    Ra = 2.0 * critical_rayleigh(1e-3)
    a = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4)
    b = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4)
    th = inputs.theta_init(n_r, n_phi, 1e-2, 5, cfg=1)
    z, zu = inputs.zero_state(n_r, n_phi)
    a.set_state(th, z, zu)
    b.set_state(th, z, zu)
    a.step(3)
    for _ in range(3):
        b.step(1)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)


def test_edge_cases():
    n_r, n_phi = 33, 96
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    # zero state stays exactly zero
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(z, z, zu)
    gpu.step(3)
    for x in gpu.get_state():
        assert not np.any(x)
    # zonal-only state (m = 0 flow and temperature): matches the oracle
    th = inputs.theta_init(n_r, n_phi, 1e-2, 4, cfg=1, m_min=0)
    th[1:] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1e-2, 6, cfg=3, m_min=0)[0].real
    gpu.set_state(th, z, u)
    ora.set_state(z, th, u)
    for _ in range(3):
        gpu.step(1)
        ora.step()
    assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    # ragged input: fewer coefficients than N_c are zero-padded
    th = inputs.theta_init(n_r, n_phi, 1e-3, 8, cfg=1)
    thr = np.ascontiguousarray(th[:, :7])
    gpu.set_state(thr)
    ps, tt, uu = gpu.get_state()
    assert np.array_equal(tt[:, :7], thr) and not np.any(tt[:, 7:]) and not np.any(ps) and not np.any(uu)
    gpu.close()


def _refined_solve(L, f, iters=3):
    """Row-scaled dense LU, then iterative refinement with residuals evaluated in
    extended precision (numpy longdouble)."""
    import scipy.linalg as sl
    r = 1.0 / np.abs(L).max(axis=1)
    lu = sl.lu_factor(L * r[:, None])
    x = sl.lu_solve(lu, f * r)
    Ll = L.astype(np.clongdouble)
    for _ in range(iters):
        res = (f.astype(np.clongdouble) - Ll @ x.astype(np.clongdouble)).astype(complex)
        x = x + sl.lu_solve(lu, res * r)
    return x


def test_large_workload_sampled():
    """n_r = 2049, n_phi = 6144 (N_m = 2048, N_c = 1365), E = 1e-8, SBDF3 whose
    first step is SBDF1: the explicit right-hand sides are compared in full; the
    first step's new state is compared on sampled modes, the oracle solving only
    those modes' tau systems."""
    import scipy.linalg as sl
    n_r, n_phi, E, dt = 2049, 6144, 1e-8, 1e-10
    from paper_1902_07092_gb300.binding import Solver
    from oracle.explicit import Grid
    from oracle.operators import IntegrationOperators
    Ra = 2.0e11     # 3.2 Ra_c at E = 1e-8; the value does not affect parity
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt)
    nc = gpu.n_c
    th = inputs.theta_init(n_r, n_phi, 1e-3, 3, cfg=3)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    ep, et, eu = gpu.explicit_terms()
    ops = IntegrationOperators(n_r, nc, 0.35, E, 1.0, Ra)
    g = Grid(ops, n_phi)
    rp, rt, ru = explicit_terms(g, z, th, zu)
    tol = 4 * n_r * n_r * 2.0 ** -53
    assert rel_l2(ep, rp) <= tol and rel_l2(et, rt) <= tol
    gpu.step(1)
    ps, tt, uu = gpu.get_state()
    for m in (1, 2, 700, 2048):
        # SBDF1: (Mass - dt Lin) y = Mass y_n + dt e_n
        Lp = ops.lhs_psi(m, dt)
        fp = dt * rp[m]
        fp[:4] = 0
        ref_p = _refined_solve(Lp, fp)
        Lt = ops.lhs_theta(m, dt).astype(complex)
        ft = ops.D @ th[m] + dt * rt[m]
        ft[:2] = 0
        ref_t = _refined_solve(Lt, ft)
        assert rel_l2(tt[m], ref_t) <= 1e-12, m
        # reference: row-scaled dense LU refined with extended-precision residuals.
        # With FP64 residuals any refined solve is limited to ~cond * eps; at this
        # size the streamfunction system's effective condition number is ~2e5
        # (a second FP64 refinement step leaves the GPU result at 2.2e-11), so
        # the bound is 5e-11 = 2e5 * 2.2e-16 rounded up.
        assert rel_l2(ps[m], ref_p) <= 5e-11, m
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (257, 768)])
def test_diagnostics_match_oracle(n_r, n_phi):
    from oracle.diagnostics import diagnostics
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    psi, th, u = random_state(n_r, n_phi, 1.0, 21, psi_amp=1e-2, u_amp=1e-1)
    th[0] = th[0].real
    gpu.set_state(th, psi, u)
    d = gpu.diagnostics()
    r = diagnostics(ora.g, psi, th, u)
    for key in ("E_K", "E_Z", "enstrophy", "Nu", "Re", "Ro", "cfl_s", "cfl_phi"):
        assert abs(d[key] - r[key]) <= 1e-12 * max(abs(r[key]), 1e-300), (key, d[key], r[key])
    gpu.close()


@pytest.mark.parametrize("radial", ["integration", "collocation"])
def test_overlapping_contexts_match_a_context_run_alone(radial):
    """Two contexts stepping on their own streams with no synchronisation between
    them (their kernels share SMs) must give bitwise the results of a context
    stepped alone: every kernel's result depends only on its own inputs."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E = (257, 768, 1e-5) if radial == "integration" else (65, 192, 1e-4)
    Ra = 10.0 * critical_rayleigh(1e-5) if radial == "integration" else 2e6
    nc = n_r if radial == "collocation" else None
    th = inputs.theta_init(n_r, n_phi, 1e-3, 2, cfg=2, n_c=nc)
    z, zu = inputs.zero_state(n_r, n_phi, n_c=nc)
    alone = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", 1e-7, radial=radial)
    alone.set_state(th, z, zu)
    alone.step(6)
    ref = alone.get_state()
    alone.close()
    a = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", 1e-7, radial=radial)
    b = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", 1e-7, radial=radial)
    a.set_state(th, z, zu)
    b.set_state(th, z, zu)
    for _ in range(6):
        a.step(1)
        b.step(1)
    for s in (a, b):
        for x, y in zip(s.get_state(), ref):
            assert np.array_equal(x, y)
        s.close()


@pytest.mark.parametrize("n_r,n_phi", [(65, 192), (257, 768)])
def test_azimuthal_products_in_ddfloat_and_fp64_match_oracle(n_r, n_phi):
    """Option azimuthal_dd: the azimuthal transforms and products of the FP64
    stage in double-float arithmetic (default) or in FP64; both within the
    explicit-term tolerance of the oracle, on states with O(1) fields."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    psi, th, u = random_state(n_r, n_phi, 1.0, 5, psi_amp=1.0, u_amp=1.0)
    tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
    for dd in (1, 0):
        gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
        pizza_set_option(gpu.ctx, "azimuthal_dd", dd)
        gpu.set_state(th, psi, u)
        ep, et, eu = gpu.explicit_terms()
        rp, rt, ru = explicit_terms(ora.g, psi, th, u)
        errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
        print("azimuthal_dd=%d n_r=%d: psi %.2e theta %.2e u %.2e (tol %.1e)" % ((dd, n_r) + errs + (tol,)))
        assert max(errs) <= tol
        gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "ARS443"])
def test_steps_match_oracle_split_streamfunction_solve(scheme):
    """n_r = 513 (N_c = 341, 43 blocks of 8 rows): the streamfunction block is
    solved in two halves joined through spikes (from 40 blocks); explicit
    buoyancy, all fields nonzero, two steps.  5e-12, the bound of the n_r = 1025
    tests: the block's conditioning grows with N_c."""
    n_r, n_phi = 513, 24
    gpu, ora = make_pair(n_r, n_phi, 1e-5, 5.0, scheme, 1e-7)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 31, cfg=1)
    psi = inputs.theta_init(n_r, n_phi, 1e-5, 32, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1e-3, 33, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, 5e-12, oracle=ora)
        print("split solve n_r=513 %s step %d: state %.2e" % (scheme, k + 1, e["state"]))
    gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF3"])
def test_steps_match_oracle_fp32_refined_temperature_solve(scheme):
    """n_r = 1025 (N_c = 682): the temperature systems are solved by FP32 block
    chains with two FP64-residual corrections, the first beside the
    streamfunction refinement (explicit buoyancy); the streamfunction block is
    split in two halves; mode 0 refines its zonal flow in FP64.  All fields
    nonzero, two steps, against the FP64 oracle.  5e-12, the bound of the
    n_r = 1025 implicit-buoyancy test."""
    n_r, n_phi = 1025, 24
    gpu, ora = make_pair(n_r, n_phi, 1e-6, 5.0, scheme, 1e-9)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 41, cfg=1, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1e-5, 42, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1e-3, 43, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, 5e-12, oracle=ora)
        print("FP32-refined temperature n_r=1025 %s step %d: %s" % (
            scheme, k + 1, {a: "%.2e" % b for a, b in e.items() if a != "_norms"}))
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi,E,scheme,tol", [(1025, 768, 1e-6, "CNAB2", 5e-12), (1025, 768, 1e-6, "SBDF3", 5e-12),
                                                    (257, 768, 1e-5, "ARS443", 2e-12),
                                                    (65, 192, 1e-3, "BPR353", 1e-12)])
def test_solve_in_one_cta_per_system_equals_one_cta_per_mode(n_r, n_phi, E, scheme, tol):
    """Option solve_roles: with explicit buoyancy the solve runs one CTA per
    system (streamfunction; temperature, then the zonal flow for m = 0) instead of
    one per mode -- by default from N_c > 600 (FP32-refined temperature), on
    request below it (FP64 temperature blocks).  With FP64 streamfunction chains
    (option psi_chain_dd = 0) the two kernels differ only in the order of the
    Schur step's sums (the whole CTA against one warp), so three steps from a
    state with every field nonzero agree to the parity bar of the size, and
    each is that close to the oracle."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    psi, th, u = random_state(n_r, n_phi, 1e-2, 31, psi_amp=1e-4, u_amp=1e-3)
    out = []
    ora = None
    for roles in (1, 0):
        s, o = make_pair(n_r, n_phi, E, 5.0, scheme, 1e-3 * E)
        if ora is None:
            ora = o
            ora.set_state(psi, th, u)
            for _ in range(3):
                ora.step()
        pizza_set_option(s.ctx, "solve_roles", roles)
        pizza_set_option(s.ctx, "psi_chain_dd", 0)
        s.set_state(th, psi, u)
        s.step(3)
        e = assert_state_close(s.get_state(), ora.y, tol, oracle=ora)
        print("solve_roles=%d n_r=%d %s: state %.2e" % (roles, n_r, scheme, e["state"]))
        out.append(s.get_state())
        s.close()
    d = rel_l2(np.concatenate([np.ravel(x) for x in out[0]]), np.concatenate([np.ravel(x) for x in out[1]]))
    print("one CTA per system vs per mode n_r=%d: %.2e" % (n_r, d))
    assert d <= tol


@pytest.mark.parametrize("n_r,n_phi", [(129, 384), (257, 768), (513, 1536)])
def test_lean_radial_layout_matches_oracle(n_r, n_phi):
    """Option radial_lean = 1 below its default threshold: the three-array
    synthesis and analysis kernels give the oracle's explicit terms to the same
    bar as the batched layout."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    pizza_set_option(gpu.ctx, "radial_lean", 1)
    psi, th, u = random_state(n_r, n_phi, 1.0, 5, psi_amp=1.0, u_amp=1.0)
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    print("lean explicit terms n_r=%d: %.2e %.2e %.2e (tol %.1e)" % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi,E,scheme,tol", [(65, 192, 1e-3, "BPR353", 1e-12), (257, 24, 1e-5, "ARS443", 2e-12),
                                                    (513, 24, 1e-5, "CNAB2", 5e-12),
                                                    (1025, 24, 1e-6, "SBDF3", 5e-12)])
def test_double_float_streamfunction_chains_match_oracle(n_r, n_phi, E, scheme, tol):
    """Option psi_chain_dd: the block chains of the streamfunction solve in
    double-float arithmetic (48 bits; Schur step, residual and refinement in
    FP64), forced on below its default threshold (n_r = 65, 257: one chain pair;
    513: the split block) and the default at n_r = 1025.  Two steps against the
    oracle at the bars of the FP64-chain tests of the same sizes, and against the
    FP64 chains of the same kernel (option 0) to the same bar."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    th = inputs.theta_init(n_r, n_phi, 1e-3, 51, cfg=1, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1e-5, 52, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1e-3, 53, cfg=9, m_min=0)[0].real.copy()
    runs = {}
    for dd in (1, 0):
        gpu, ora = make_pair(n_r, n_phi, E, 5.0, scheme, 1e-3 * E)
        pizza_set_option(gpu.ctx, "solve_roles", 1)
        pizza_set_option(gpu.ctx, "psi_chain_dd", dd)
        gpu.set_state(th, psi, u)
        ora.set_state(psi, th, u)
        for k in range(2):
            gpu.step(1)
            ora.step()
            e = assert_state_close(gpu.get_state(), ora.y, tol, oracle=ora)
            print("psi_chain_dd=%d n_r=%d %s step %d: state %.2e psi %.2e" % (dd, n_r, scheme, k + 1, e["state"],
                                                                             e["psi"]))
        runs[dd] = gpu.get_state()
        gpu.close()
    d = rel_l2(np.concatenate([np.ravel(x) for x in runs[1]]), np.concatenate([np.ravel(x) for x in runs[0]]))
    print("double-float vs FP64 chains n_r=%d: %.2e" % (n_r, d))
    assert d <= tol


@pytest.mark.parametrize("dd,t32", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("n_r,n_phi,E,scheme,tol", [(129, 24, 1e-4, "CNAB2", 1e-12), (257, 24, 1e-5, "ARS443", 2e-12),
                                                    (513, 24, 1e-5, "SBDF3", 5e-12)])
def test_one_cta_per_mode_solve_options_match_oracle(n_r, n_phi, E, scheme, tol, dd, t32):
    """The solve with one CTA per mode below N_c = 600 with options
    psi_chain_dd = 1 (double-float streamfunction chains, the solution converted
    back before the Schur steps and the join) and theta_fp32 = 1 (temperature by
    FP32 chains and two FP64-residual corrections, the zonal flow refined in
    FP64), alone and together: two steps with every field nonzero against the
    oracle at the bars of the FP64 solve of the same sizes."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    th = inputs.theta_init(n_r, n_phi, 1e-3, 61, cfg=1, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1e-5, 62, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1e-3, 63, cfg=9, m_min=0)[0].real.copy()
    gpu, ora = make_pair(n_r, n_phi, E, 5.0, scheme, 1e-3 * E)
    pizza_set_option(gpu.ctx, "solve_roles", 0)
    pizza_set_option(gpu.ctx, "psi_chain_dd", dd)
    pizza_set_option(gpu.ctx, "theta_fp32", t32)
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, tol, oracle=ora)
        print("per-mode solve dd=%d t32=%d n_r=%d %s step %d: %s" % (
            dd, t32, n_r, scheme, k + 1, {a: "%.2e" % b for a, b in e.items() if a != "_norms"}))
    gpu.close()


def test_solve_with_one_cta_per_system_is_deterministic():
    """The double-float path of the solve with one CTA per system (n_r = 1025:
    split streamfunction block, the correction solved in place of its residual,
    shared-memory coefficient rings; FP32-refined temperature) has no
    nondeterministic reduction, so repeated runs from one state must agree bit
    for bit; a race between the warps of a pair (a row read after the other warp
    stored into it) shows up here as a mismatch."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E = 1025, 768, 1e-6
    Ra = 5.0 * critical_rayleigh(E)
    psi, th, u = random_state(n_r, n_phi, 1e-2, 71, psi_amp=1e-4, u_amp=1e-3)
    ref = None
    for rep in range(4):
        s = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", 1e-9)
        s.set_state(th, psi, u)
        s.step(3)
        got = s.get_state()
        s.close()
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), rep


@pytest.mark.parametrize("n_r,n_phi", [(129, 384), (257, 768), (513, 1536)])
def test_double_float_lean_radial_transforms_match_oracle(n_r, n_phi):
    """Option radial_dd = 1 with the lean layout forced: the DCT-I, the derivative
    scans and the field arithmetic at each radius of the synthesis and analysis
    kernels in double-float arithmetic (the banded applies and the stored values
    in FP64) give the oracle's explicit terms to the bar of the FP64 transforms,
    max(1e-12, 4 n_r^2 eps), on states with O(1) fields; and two steps to the
    step bars of the size."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    pizza_set_option(gpu.ctx, "radial_lean", 1)
    pizza_set_option(gpu.ctx, "radial_dd", 1)
    psi, th, u = random_state(n_r, n_phi, 1.0, 5, psi_amp=1.0, u_amp=1.0)
    gpu.set_state(th, psi, u)
    ep, et, eu = gpu.explicit_terms()
    rp, rt, ru = explicit_terms(ora.g, psi, th, u)
    tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
    errs = (rel_l2(ep, rp), rel_l2(et, rt), rel_l2(eu, ru))
    print("double-float lean explicit terms n_r=%d: %.2e %.2e %.2e (tol %.1e)" % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()
    # two steps from a small state, against the oracle
    gpu, ora = make_pair(n_r, 24, 1e-5, 5.0, "SBDF3", 1e-8)
    pizza_set_option(gpu.ctx, "radial_lean", 1)
    pizza_set_option(gpu.ctx, "radial_dd", 1)
    th = inputs.theta_init(n_r, 24, 1e-3, 81, cfg=1, m_min=0)
    psi = inputs.theta_init(n_r, 24, 1e-5, 82, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, 24, 1e-3, 83, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    ora.set_state(psi, th, u)
    bar = {129: 1e-12, 257: 2e-12, 513: 5e-12}[n_r]
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, bar, oracle=ora)
        print("double-float lean n_r=%d step %d: state %.2e" % (n_r, k + 1, e["state"]))
    gpu.close()
