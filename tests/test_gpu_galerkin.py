"""GPU Galerkin-basis solve (option "radial" = 2, Appendix B) against the oracle's
GalerkinStepper (itself pinned against the tau solve, numpy's Chebyshev boundary
values and the paper's bandwidths), and against the GPU tau path, which solves
the same discrete problem.

Tolerances: 1e-12 whole-state relative L2 per step as for the tau path up to
n_r = 129.  At n_r = 257 the row-scaled streamfunction Galerkin systems have
condition numbers 5e7 - 1e8 (oracle matrices, m = 1, 64, 256), where the tau
systems' are far lower; two unrefined FP64 solves of such a system with
different rounding (host-built versus numpy-built matrix, different elimination
order) differ by up to cond * eps componentwise, and the oracle's own Galerkin
and tau solves of one step differ by 5.3e-12 in Psi (one refinement step only
takes that to 3.3e-12).  The n_r = 257 bound is therefore 2e-11 per field and
for the state, against the Galerkin oracle and against the GPU tau path.  The
sampled n_r = 2049 modes are held within 4 cond(G) eps of an extended-precision
solve of the same Galerkin system (cond of the row-scaled matrix, computed here)."""
import numpy as np
import pytest

from oracle.explicit import explicit_terms
from oracle.galerkin import GalerkinStepper, galerkin_matrix, stencil_dir, stencil_psi
from oracle import chebyshev as ch
from paper_1902_07092_gb300 import inputs
from tests.parity_util import assert_state_close, critical_rayleigh, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.linalg.LinAlgWarning")]


def make_pair(n_r, n_phi, E, ra_factor, scheme, dt, buoy=False):
    from paper_1902_07092_gb300.binding import Solver
    Ra = ra_factor * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, radial="galerkin", buoy_implicit=buoy)
    ora = GalerkinStepper(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, buoy_implicit=buoy)
    return gpu, ora


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_galerkin_steps_match_oracle_tiny(scheme, amp):
    n_r, n_phi = 33, 96
    gpu, ora = make_pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4)
    th = inputs.theta_init(n_r, n_phi, amp, 1, cfg=1)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for _ in range(5):
        gpu.step(1)
        ora.step()
        assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi", [(9, 24), (17, 48), (65, 192), (129, 384)])
def test_galerkin_sizes_and_implicit_buoyancy(n_r, n_phi):
    """Ragged and small systems (n_r = 9, the smallest grid: one streamfunction
    unknown and three for temperature; n_r = 17: 6 streamfunction unknowns, fewer
    than the 8 subdiagonals) and the temperature-first ordering of implicit
    buoyancy."""
    for buoy in (False, True):
        gpu, ora = make_pair(n_r, n_phi, 1e-3, 3.0, "CNAB2", 1e-4, buoy=buoy)
        th = inputs.theta_init(n_r, n_phi, 1e-2, 11, cfg=1, m_min=0)
        u = inputs.theta_init(n_r, n_phi, 1e-2, 12, cfg=3, m_min=0)[0].real
        z, _ = inputs.zero_state(n_r, n_phi)
        gpu.set_state(th, z, u)
        ora.set_state(z, th, u)
        for _ in range(3):
            gpu.step(1)
            ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
        print("galerkin n_r=%d buoy=%d: state %.2e" % (n_r, buoy, e["state"]))
        gpu.close()


def test_galerkin_sparse_workload_matches_oracle_and_tau():
    """The n_r = 257, n_phi = 768 ARS443 workload, two steps: against the Galerkin
    oracle, and the GPU Galerkin and tau paths against each other."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E = 257, 768, 1e-5
    gpu, ora = make_pair(n_r, n_phi, E, 10.0, "ARS443", 1e-7)
    tau = Solver(n_r, n_phi, E, 10.0 * critical_rayleigh(E), 1.0, 0.35, "ARS443", 1e-7)
    th = inputs.theta_init(n_r, n_phi, 1e-3, 2, cfg=2)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    tau.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for _ in range(2):
        gpu.step(1)
        tau.step(1)
        ora.step()
        e = assert_state_close(gpu.get_state(), ora.y, 2e-11, oracle=ora)
        et = assert_state_close(gpu.get_state(), tau.get_state(), 2e-11, oracle=ora)
        print("galerkin n257: vs oracle %.2e, vs GPU tau %.2e" % (e["state"], et["state"]))
    gpu.close()
    tau.close()


def test_galerkin_switch_keeps_the_state():
    """radial 1 -> 2 keeps the state and the multistep history and rebuilds only
    the factors: two tau steps and a Galerkin step equal three Galerkin steps."""
    from paper_1902_07092_gb300.binding import Solver, pizza_set_option
    n_r, n_phi = 33, 96
    Ra = 2.0 * critical_rayleigh(1e-3)
    a = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4)
    th = inputs.theta_init(n_r, n_phi, 1e-2, 3, cfg=1)
    z, zu = inputs.zero_state(n_r, n_phi)
    a.set_state(th, z, zu)
    a.step(2)
    y = a.get_state()
    pizza_set_option(a.ctx, "radial", 2)
    for x0, x1 in zip(y, a.get_state()):
        assert np.array_equal(x0, x1)
    a.step(1)  # the third step in the Galerkin bases, with the history of the first two
    b = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4, radial="galerkin")
    b.set_state(th, z, zu)
    b.step(3)
    for x0, x1 in zip(a.get_state(), b.get_state()):
        assert rel_l2(x0, x1) <= 1e-12
    a.close()
    b.close()


def _extended_solve(G, f, iters=3):
    """Row-scaled dense LU refined with extended-precision residuals."""
    import scipy.linalg as sl
    r = 1.0 / np.abs(G).max(axis=1)
    lu = sl.lu_factor(G * r[:, None])
    x = sl.lu_solve(lu, f * r)
    Gl = G.astype(np.clongdouble)
    for _ in range(iters):
        res = (f.astype(np.clongdouble) - Gl @ x.astype(np.clongdouble)).astype(complex)
        x = x + sl.lu_solve(lu, res * r)
    return x, np.linalg.cond(G * r[:, None])


def test_galerkin_large_workload_sampled():
    """n_r = 2049, n_phi = 6144 (N_c = 1365), E = 1e-8, SBDF3 (first step SBDF1):
    sampled modes of the first step against an extended-precision solve of the
    oracle's Galerkin systems."""
    from paper_1902_07092_gb300.binding import Solver
    from oracle.explicit import Grid
    from oracle.operators import IntegrationOperators
    n_r, n_phi, E, dt = 2049, 6144, 1e-8, 1e-10
    Ra = 2.0e11
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", dt, radial="galerkin")
    nc = gpu.n_c
    th = inputs.theta_init(n_r, n_phi, 1e-3, 3, cfg=3)
    z, zu = inputs.zero_state(n_r, n_phi)
    gpu.set_state(th, z, zu)
    gpu.step(1)
    ps, tt, uu = gpu.get_state()
    ops = IntegrationOperators(n_r, nc, 0.35, E, 1.0, Ra)
    g = Grid(ops, n_phi)
    rp, rt, ru = explicit_terms(g, z, th, zu)
    hs = ch.hat_scale(n_r, nc)
    Sp, Sd = stencil_psi(nc), stencil_dir(nc)
    eps = 2.0 ** -53
    for m in (1, 700, 2048):
        Gp = galerkin_matrix(ops.A(m) - dt * ops.B(m), 4, Sp, n_r)
        xp, cp = _extended_solve(Gp, (dt * rp[m])[4:])
        Gt = galerkin_matrix(ops.D - dt * ops.F(m) / ops.Pr, 2, Sd, n_r).astype(complex)
        xt, ct = _extended_solve(Gt, (ops.D @ th[m] + dt * rt[m])[2:])
        ep, et = rel_l2(ps[m], (Sp @ xp) / hs), rel_l2(tt[m], (Sd @ xt) / hs)
        print("galerkin n2049 m=%d: psi %.2e (cond %.1e) theta %.2e (cond %.1e)" % (m, ep, cp, et, ct))
        assert ep <= max(1e-12, 4 * cp * eps), m
        assert et <= max(1e-12, 4 * ct * eps), m
    gpu.close()


def test_galerkin_with_pumping_mixed_precision_batch_and_adjoint():
    """The Galerkin solve combined with the other options: Ekman pumping (explicit
    in the integration formulation) against the Galerkin oracle with pumping;
    mixed precision against that oracle within the mixed-precision bar; one batch
    graph over a Galerkin and a tau context equal to each stepped alone, bit for
    bit; and a taped CNAB2 run reversed by the adjoint (the adjoint of the tau
    step, the same discrete map) against the oracle's adjoint."""
    from oracle.adjoint import adjoint_cnab2
    from oracle.stepper import IntegrationStepper
    from paper_1902_07092_gb300.binding import Batch, Solver, pizza_set_option
    n_r, n_phi, E = 33, 96, 1e-3
    Ra = 3.0 * critical_rayleigh(E)
    th = inputs.theta_init(n_r, n_phi, 1e-2, 21, cfg=1, m_min=0)
    z, zu = inputs.zero_state(n_r, n_phi)
    # pumping
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", 1e-4, radial="galerkin", pumping_eps=1e-2)
    ora = GalerkinStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "SBDF3", 1e-4, pumping_eps=1e-2)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for _ in range(3):
        gpu.step(1)
        ora.step()
    assert_state_close(gpu.get_state(), ora.y, 1e-12, oracle=ora)
    gpu.close()
    # mixed precision
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", 1e-4, radial="galerkin")
    pizza_set_option(gpu.ctx, "precision", 1)
    ora = GalerkinStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "ARS443", 1e-4)
    gpu.set_state(th, z, zu)
    ora.set_state(z, th, zu)
    for _ in range(5):
        gpu.step(1)
        ora.step()
    assert_state_close(gpu.get_state(), ora.y, 1e-6, oracle=ora)
    gpu.close()
    # one batch graph
    runs = [("galerkin", "CNAB2"), ("integration", "ARS443")]
    alone = []
    for radial, scheme in runs:
        a = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, 1e-4, radial=radial)
        a.set_state(th, z, zu)
        a.step(4)
        alone.append(a.get_state())
        a.close()
    sols = [Solver(n_r, n_phi, E, Ra, 1.0, 0.35, s, 1e-4, radial=r) for r, s in runs]
    for s in sols:
        s.set_state(th, z, zu)
    batch = Batch(sols)
    batch.step(4)
    for s, ref in zip(sols, alone):
        for x, y in zip(s.get_state(), ref):
            assert np.array_equal(x, y)
    batch.close()
    for s in sols:
        s.close()
    # adjoint of a Galerkin-stepped run, (17, 24), nine steps, checkpoints every 4
    n_r, n_phi, E, Ra, dt, K = 17, 24, 1e-3, 2e5, 2e-4, 9
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt, radial="galerkin")
    ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt)
    rng = np.random.default_rng(5)
    c = lambda: 0.5 * (rng.standard_normal((gpu.M, gpu.n_c)) + 1j * rng.standard_normal((gpu.M, gpu.n_c))) \
        / (1 + np.arange(gpu.n_c)) ** 2
    psi0, th0 = c(), c()
    psi0[0] = 0.0
    th0[0] = th0[0].real
    u0 = 0.5 * rng.standard_normal(gpu.n_c) / (1 + np.arange(gpu.n_c)) ** 2
    J_ref, lam_ref, dRa_ref = adjoint_cnab2(ora, (psi0, th0, u0), K)
    gpu.set_state(th0, psi0, u0)
    gpu.tape_begin(4)
    gpu.step(K)
    w = gpu.nusselt_weights()
    g = np.zeros((gpu.M, gpu.n_c), complex)
    g[0] = w / K
    for i in range(K):
        dRa = gpu.adjoint_step(g_theta=g, want_dRa=(i == K - 1))
    ps, tt, uu = gpu.get_adjoint()
    errs = (rel_l2(ps, lam_ref[0]), rel_l2(tt, lam_ref[1]), rel_l2(uu, lam_ref[2]))
    print("galerkin adjoint run: psi %.2e theta %.2e u %.2e dRa %.3e vs %.3e" % (errs + (dRa, dRa_ref)))
    assert max(errs) <= 1e-9
    assert abs(dRa - dRa_ref) <= 1e-9 * abs(dRa_ref)
    gpu.close()
