"""GPU discrete adjoint (pizza_tape_begin / pizza_adjoint_step) against the
oracle's adjoint (oracle/adjoint.py, itself pinned by the dot-product test and
finite differences) and against central finite differences of GPU runs.

Tolerances: the adjoint of the explicit stage 8 n_r^2 eps for theta and u_bar
and 8 n_r^4 eps for Psi (relative L2): Psi_bar passes the transposes of two radial
derivatives, whose rows grow like n^4 (T_n'' at the walls); whole-run gradients
1e-9 against the oracle at (17, 24) (dense transposed solves on both sides) and
1e-8 at (257, 768), the streamfunction adjoint there within the same 8 n_r^4 eps
as the explicit stage; finite differences with h = 1e-6 relative carry O(h^2)
truncation and ~eps J/h rounding: 1e-5 relative.  J depends on Ra only through
the nonlinear coupling, about 1e-9 of J over the 2.4e-6 time units of the test,
so its finite difference takes h = 1e-2 relative (smaller steps resolve
rounding, not the derivative; measured 5e-3 at h = 1e-6, 2e-6 at h = 1e-2)."""
import numpy as np
import pytest

from oracle.adjoint import adjoint_cnab2, explicit_adjoint
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _rand(rng, M, nc, amp):
    c = lambda: amp * (rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))) / (1 + np.arange(nc)) ** 2
    psi, th = c(), c()
    psi[0] = 0.0
    th[0] = th[0].real
    u = amp * rng.standard_normal(nc) / (1 + np.arange(nc)) ** 2
    return psi, th, u


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (257, 768)])
def test_explicit_adjoint_matches_oracle(n_r, n_phi):
    from paper_1902_07092_gb300.binding import Solver
    Ra = 3e5
    gpu = Solver(n_r, n_phi, 1e-3, Ra, 0.7, 0.35, "CNAB2", 1e-4)
    ora = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 0.7, 0.35, "CNAB2", 1e-4)
    rng = np.random.default_rng(21)
    y = _rand(rng, gpu.M, gpu.n_c, 1.0)
    eb = _rand(rng, gpu.M, gpu.n_c, 1.0)
    gpu.set_state(y[1], y[0], y[2])
    got = gpu.explicit_adjoint(*eb)
    ref, _ = explicit_adjoint(ora.g, *y, eb)
    tol = 8 * n_r * n_r * EPS
    tol_psi = 8 * float(n_r) ** 4 * EPS
    errs = [rel_l2(a, b) for a, b in zip(got, ref)]
    print("explicit adjoint n_r=%d: psi %.2e theta %.2e u %.2e (tol %.1e, psi %.1e)"
          % ((n_r,) + tuple(errs) + (tol, tol_psi)))
    assert errs[0] <= tol_psi
    assert max(errs[1:]) <= tol
    gpu.close()


@pytest.mark.parametrize("every", [1, 4])
def test_adjoint_run_matches_oracle(every):
    """J = (1/K) sum (Nu_n - 1), K = 9 CNAB2 steps at (17, 24), E = 1e-3, a strongly
    nonlinear state; checkpoints every 1 or 4 steps (segments recomputed)."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E, Ra, dt, K = 17, 24, 1e-3, 2e5, 2e-4, 9
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt)
    ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt)
    rng = np.random.default_rng(5)
    y0 = _rand(rng, gpu.M, gpu.n_c, 0.5)
    J_ref, lam_ref, dRa_ref = adjoint_cnab2(ora, y0, K)
    gpu.set_state(y0[1], y0[0], y0[2])
    gpu.tape_begin(every)
    w = gpu.nusselt_weights()
    J = 0.0
    for _ in range(K):
        gpu.step(1)
        J += float(np.dot(w, gpu.get_state()[1][0].real)) / K
    g = np.zeros((gpu.M, gpu.n_c), complex)
    g[0] = w / K
    for _ in range(K):
        dRa = gpu.adjoint_step(g_theta=g)
    ps, th, u = gpu.get_adjoint()
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    errs = (rel_l2(ps, lam_ref[0]), rel_l2(th, lam_ref[1]), rel_l2(u, lam_ref[2]))
    print("adjoint run every=%d: psi %.2e theta %.2e u %.2e dRa %.3e vs %.3e" % ((every,) + errs + (dRa, dRa_ref)))
    assert max(errs) <= 1e-9
    assert abs(dRa - dRa_ref) <= 1e-9 * abs(dRa_ref)
    gpu.close()


def test_adjoint_gradient_matches_finite_differences_n257():
    """The adjoint workload's grid (n_r = 257, n_phi = 768, E = 1e-5, Ra = 5 Ra_c,
    CNAB2, dt = 1e-7), 24 steps with checkpoints every 10 (a partial last
    segment), seeded initial perturbation 1e-3: dJ/dtheta_0 along a seeded
    direction and dJ/dRa against central differences (h = 1e-6 relative)."""
    from paper_1902_07092_gb300.autograd import NusseltAverage
    import torch
    E = 1e-5
    Ra = 5.0 * critical_rayleigh(E)
    cfg = dict(n_r=257, n_phi=768, E=E, Pr=1.0, radius_ratio=0.35, dt=1e-7, steps=24, checkpoint_every=10)
    th0 = inputs.theta_init(257, 768, 1e-3, 5, cfg=5, m_min=0)
    t = torch.tensor(th0, requires_grad=True)
    r = torch.tensor(Ra, dtype=torch.float64, requires_grad=True)
    J = NusseltAverage.apply(t, r, cfg)
    J.backward()
    d = inputs.theta_init(257, 768, 1.0, 55, cfg=5, m_min=0)
    h = 1e-6 * np.linalg.norm(th0) / np.linalg.norm(d)
    with torch.no_grad():
        Jp = float(NusseltAverage.apply(torch.tensor(th0 + h * d), r, cfg))
        Jm = float(NusseltAverage.apply(torch.tensor(th0 - h * d), r, cfg))
    fd = (Jp - Jm) / (2 * h)
    ad = float(np.real(np.vdot(t.grad.numpy(), d)))
    print("n257 gradient: fd %.9e adjoint %.9e" % (fd, ad))
    assert abs(fd - ad) <= 1e-5 * abs(ad)
    hR = 1e-2 * Ra
    with torch.no_grad():
        Jp = float(NusseltAverage.apply(torch.tensor(th0), torch.tensor(Ra + hR), cfg))
        Jm = float(NusseltAverage.apply(torch.tensor(th0), torch.tensor(Ra - hR), cfg))
    fdR = (Jp - Jm) / (2 * hR)
    print("n257 dJ/dRa: fd %.9e adjoint %.9e" % (fdR, float(r.grad)))
    assert abs(fdR - float(r.grad)) <= 1e-4 * abs(float(r.grad))


def test_adjoint_workload_400_steps_checkpoint_20():
    """The adjoint workload as specified: 400 CNAB2 steps at n_r = 257,
    n_phi = 768, E = 1e-5, Pr = 1, Ra = 5 Ra_c, dt = 1e-7, checkpoints every 20
    steps, seeded initial perturbation 1e-3 (seed 5): dJ/dtheta_0 along a seeded
    direction against central finite differences with h = 1e-6 relative to
    |theta_0|, and dJ/dRa with h = 1e-3 relative to Ra: J depends on Ra only
    weakly here (Ra dJ/dRa ~ 2e-3 J), so at h = 1e-6 the difference J(Ra + h) -
    J(Ra - h) is ~4e-9 J, a few thousand ulps of J, and the rounding differences
    of two separate 400-step runs are a visible fraction of it (measured: 4e-3
    off at h = 1e-6); at h = 1e-3 they are not, and the central difference's
    O(h^2) error stays far below the bar."""
    from paper_1902_07092_gb300.autograd import NusseltAverage
    import torch
    wl = inputs.WORKLOADS["adjoint_n257_p768"]
    E = wl["E"]
    Ra = wl["ra_factor"] * critical_rayleigh(E)
    cfg = dict(n_r=wl["n_r"], n_phi=wl["n_phi"], E=E, Pr=1.0, radius_ratio=0.35, dt=wl["dt"], steps=wl["steps"],
               checkpoint_every=wl["checkpoint_every"])
    th0 = inputs.theta_init(wl["n_r"], wl["n_phi"], wl["amp"], wl["seed"], cfg=wl["cfg"], m_min=0)
    t = torch.tensor(th0, requires_grad=True)
    r = torch.tensor(Ra, dtype=torch.float64, requires_grad=True)
    J = NusseltAverage.apply(t, r, cfg)
    J.backward()
    d = inputs.theta_init(wl["n_r"], wl["n_phi"], 1.0, 55, cfg=5, m_min=0)
    h = 1e-6 * np.linalg.norm(th0) / np.linalg.norm(d)
    with torch.no_grad():
        Jp = float(NusseltAverage.apply(torch.tensor(th0 + h * d), r, cfg))
        Jm = float(NusseltAverage.apply(torch.tensor(th0 - h * d), r, cfg))
        JRp = float(NusseltAverage.apply(torch.tensor(th0), torch.tensor(Ra * (1 + 1e-3)), cfg))
        JRm = float(NusseltAverage.apply(torch.tensor(th0), torch.tensor(Ra * (1 - 1e-3)), cfg))
    fd = (Jp - Jm) / (2 * h)
    ad = float(np.real(np.vdot(t.grad.numpy(), d)))
    fdR = (JRp - JRm) / (2e-3 * Ra)
    print("400-step adjoint: J %.12e  theta: fd %.12e adjoint %.12e (rel %.2e)  Ra: fd %.12e adjoint %.12e "
          "(rel %.2e)" % (float(J.detach()), fd, ad, abs(fd - ad) / abs(ad), fdR, float(r.grad),
                          abs(fdR - float(r.grad)) / abs(float(r.grad))))
    assert abs(fd - ad) <= 1e-5 * abs(ad)
    assert abs(fdR - float(r.grad)) <= 1e-4 * abs(float(r.grad))


@pytest.mark.parametrize("dd", [1, 0])
def test_adjoint_run_matches_oracle_n257(dd):
    """Three CNAB2 steps on the adjoint workload's grid (257, 768), E = 1e-5,
    Ra = 5 Ra_c, dt = 1e-7, from a state with all fields nonzero; the segments
    recomputed with either form of the forward azimuthal stage (option
    azimuthal_dd)."""
    from paper_1902_07092_gb300.binding import Solver, pizza_set_option
    n_r, n_phi, E, dt, K = 257, 768, 1e-5, 1e-7, 3
    Ra = 5.0 * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt)
    pizza_set_option(gpu.ctx, "azimuthal_dd", dd)
    ora = IntegrationStepper(n_r, n_phi, E, Ra, 1.0, 0.35, "CNAB2", dt)
    rng = np.random.default_rng(8)
    y0 = _rand(rng, gpu.M, gpu.n_c, 1e-3)
    J_ref, lam_ref, dRa_ref = adjoint_cnab2(ora, y0, K)
    gpu.set_state(y0[1], y0[0], y0[2])
    gpu.tape_begin(2)
    w = gpu.nusselt_weights()
    for _ in range(K):
        gpu.step(1)
    g = np.zeros((gpu.M, gpu.n_c), complex)
    g[0] = w / K
    for _ in range(K):
        dRa = gpu.adjoint_step(g_theta=g)
    ps, th, u = gpu.get_adjoint()
    errs = (rel_l2(ps, lam_ref[0]), rel_l2(th, lam_ref[1]), rel_l2(u, lam_ref[2]))
    print("adjoint run n257 dd=%d: psi %.2e theta %.2e u %.2e dRa %.6e vs %.6e" % ((dd,) + errs + (dRa, dRa_ref)))
    assert errs[0] <= 8 * float(n_r) ** 4 * EPS   # the Psi_bar bound of the explicit adjoint
    assert max(errs[1:]) <= 1e-8
    assert abs(dRa - dRa_ref) <= 1e-8 * abs(dRa_ref)
    gpu.close()
