"""GPU parity of the Chebyshev-collocation formulation (Section 3.1), called
through the C interface with option "radial" = 0, against the oracle's
CollocationStepper on the same seeded inputs.

Tolerances (relative L2, FP64): explicit rows max(1e-12, 4 n_r^2 eps) as for the
integration path (derivatives of interpolated grid products); the physical-grid
vorticity set from psi max(1e-12, n_r^4 eps / 4) (two derivatives); full steps
1e-12 at n_r = 33 and 2e-12 at n_r = 257, where the inverses of the dense systems
themselves carry ~3e-13 (the oracle solves by LU with one refinement step, the
device multiplies by inverse columns built on the host the same way).

Where the dynamics themselves amplify rounding-size differences (the strongly
nonlinear amp = 1 states: in the oracle alone a difference grows up to ~10x per
ARS443 step at dt = 1e-4), the step-k bar
is max(1e-12, 2^7 d_k), d_k the divergence after k steps of the oracle from
itself with the initial state perturbed by 2^-52 relative (rounding_growth): each
step of the device path differs from the oracle's by up to ~2^7 units of FP64
rounding (the double-float azimuthal transforms, 2^-48 per operation over
log2 n_phi levels), and those differences grow as d_k does."""
import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle import fourier as fo
from oracle.collocation import CollocationStepper
from oracle.explicit import radial_fields
from oracle.geometry import gauss_lobatto
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def coll_pair(n_r, n_phi, E, ra_factor, scheme, dt, Pr=1.0, eta=0.35):
    from paper_1902_07092_gb300.binding import Solver
    Ra = ra_factor * critical_rayleigh(E)
    gpu = Solver(n_r, n_phi, E, Ra, Pr, eta, scheme, dt, radial="collocation")
    ora = CollocationStepper(n_r, n_phi, E, Ra, Pr, eta, scheme, dt)
    return gpu, ora


def coll_state(n_r, n_phi, amp, seed, psi_amp=None, u_amp=None):
    """theta and u_bar in the Dirichlet basis; psi = (1 - x^2)^2 p(x) meets the four
    streamfunction conditions (coefficients of p from the same generator)."""
    x = gauss_lobatto(n_r)
    th = inputs.theta_init(n_r, n_phi, amp, seed, cfg=7, m_min=0, n_c=n_r)
    base = inputs.theta_init(n_r, n_phi, psi_amp if psi_amp is not None else amp * 1e-2, seed + 1, cfg=8,
                             n_c=n_r)
    psi = ch.analysis(((1 - x * x) ** 2)[:, None] * ch.synthesis(base.T, n_r), n_r).T.copy()
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, u_amp if u_amp is not None else amp, seed + 2, cfg=9, m_min=0,
                          n_c=n_r)[0].real.copy()
    return psi, th, u


def rounding_growth(make_oracle, psi, th, u, nsteps, seed=7):
    """d_k, k = 1..nsteps: relative L2 divergence (the larger of state and theta)
    of the oracle from itself when every initial coefficient is perturbed by a
    seeded relative 2^-52 (one FP64 rounding)."""
    a, b = make_oracle(), make_oracle()
    rng = np.random.default_rng(seed)

    def pert(x):
        return x * (1.0 + 2.0 ** -52 * rng.standard_normal(np.shape(x)))

    set_both_oracle = lambda o, p, t, v: o.set_state(o.vorticity_from_psi(p), p, t, v)
    set_both_oracle(a, psi, th, u)
    set_both_oracle(b, pert(psi), pert(th), pert(u))
    out = []
    for _ in range(nsteps):
        a.step()
        b.step()
        _, p1, t1, u1 = a.y
        _, p2, t2, u2 = b.y
        r = np.concatenate([p1.ravel(), t1.ravel(), u1.astype(complex)])
        g = np.concatenate([p2.ravel(), t2.ravel(), u2.astype(complex)])
        out.append(max(rel_l2(g, r), rel_l2(t2, t1)))
    return out


def set_both(gpu, ora, psi, th, u):
    gpu.set_state(th, psi, u)
    ora.set_state(ora.vorticity_from_psi(psi), psi, th, u)


def oracle_grid(ora):
    us, uphi, w, th = ora.grid_state()
    return tuple(fo.to_grid(f, ora.n_phi) for f in (us, uphi, w, th))


def compare_state(gpu, ora, tol, tol_w=None):
    ps, th, u = gpu.get_state()
    _, rps, rth, ru = ora.y
    ref = np.concatenate([rps.ravel(), rth.ravel(), ru.astype(complex)])
    got = np.concatenate([ps.ravel(), th.ravel(), u.astype(complex)])
    errs = dict(state=rel_l2(got, ref), psi=rel_l2(ps, rps), theta=rel_l2(th, rth), u=rel_l2(u, ru))
    gw = gpu.get_grid()[2]
    rw = oracle_grid(ora)[2]
    errs["omega_grid"] = rel_l2(gw, rw)
    assert errs["state"] <= tol, errs
    assert errs["theta"] <= tol, errs
    if np.linalg.norm(rps) > 1e-3 * np.linalg.norm(ref):
        assert errs["psi"] <= tol, errs
    assert errs["omega_grid"] <= (tol_w or tol), errs
    return errs


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (65, 192), (129, 384)])
def test_collocation_explicit_rows_match_oracle(n_r, n_phi):
    gpu, ora = coll_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    psi, th, u = coll_state(n_r, n_phi, 1.0, 3, psi_amp=1.0, u_amp=1.0)
    set_both(gpu, ora, psi, th, u)
    ew, et, eu = gpu.explicit_terms()
    rw, _, rt, ru = ora.explicit(ora.y)
    tol = max(1e-12, 4 * n_r * n_r * EPS)
    errs = (rel_l2(ew, rw), rel_l2(et, rt), rel_l2(eu, ru))
    print("collocation explicit rows n_r=%d: rel L2 omega %.2e theta %.2e u %.2e (tol %.1e)"
          % ((n_r,) + errs + (tol,)))
    assert max(errs) <= tol
    gpu.close()


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (129, 384)])
def test_collocation_set_state_grid_fields(n_r, n_phi):
    """pizza_set_state builds omega = -L_beta psi; pizza_get_grid returns the
    physical-grid fields, compared with the oracle's grid_state through Eq. fft."""
    gpu, ora = coll_pair(n_r, n_phi, 1e-3, 2.0, "CNAB2", 1e-4)
    psi, th, u = coll_state(n_r, n_phi, 1.0, 5, psi_amp=1.0, u_amp=1.0)
    set_both(gpu, ora, psi, th, u)
    got = gpu.get_grid()
    ref = oracle_grid(ora)
    errs = [rel_l2(a, b) for a, b in zip(got, ref)]
    print("collocation grid fields n_r=%d: us %.2e uphi %.2e omega %.2e theta %.2e" % ((n_r,) + tuple(errs)))
    assert max(errs[0], errs[1], errs[3]) <= max(1e-12, 4 * n_r * n_r * EPS)
    assert errs[2] <= max(1e-12, n_r ** 4 * EPS / 4)
    gpu.close()


@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF2", "SBDF3", "ARS443", "BPR353"])
@pytest.mark.parametrize("amp", [1e-4, 1.0])
def test_collocation_steps_match_oracle_tiny(scheme, amp):
    """n_r = 33 collocation points, n_phi = 96, E = 1e-3, Pr = 1, Ra = 2 Ra_c,
    dt = 1e-4; amp = 1e-4 is the tiny workload's perturbation, amp = 1 the
    strongly nonlinear case.  Compared after each of four steps."""
    n_r, n_phi = 33, 96
    gpu, ora = coll_pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4)
    psi, th, u = coll_state(n_r, n_phi, amp, 1, psi_amp=amp, u_amp=amp)
    d = rounding_growth(lambda: coll_pair(n_r, n_phi, 1e-3, 2.0, scheme, 1e-4)[1], psi, th, u, 4)
    set_both(gpu, ora, psi, th, u)
    for k in range(4):
        gpu.step(1)
        ora.step()
        tol = max(1e-12, 2.0 ** 7 * d[k])
        e = compare_state(gpu, ora, tol, tol_w=max(tol, n_r ** 4 * EPS / 4))
        print("collocation %s amp %g step %d: %s" % (scheme, amp, k + 1, {a: "%.2e" % b for a, b in e.items()}))
    gpu.close()


def test_collocation_history_is_kept_across_calls():
    n_r, n_phi = 33, 96
    from paper_1902_07092_gb300.binding import Solver
    Ra = 2.0 * critical_rayleigh(1e-3)
    psi, th, u = coll_state(n_r, n_phi, 1e-2, 2)
    a = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4, radial="collocation")
    b = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4, radial="collocation")
    a.set_state(th, psi, u)
    b.set_state(th, psi, u)
    a.step(5)
    for _ in range(5):
        b.step(1)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_collocation_steps_match_oracle_n257():
    """The n_r = 257, n_phi = 768 workload (E = 1e-5, Ra = 10 Ra_c, ARS443,
    dt = 1e-7) in the collocation formulation, two steps."""
    n_r, n_phi = 257, 768
    gpu, ora = coll_pair(n_r, n_phi, 1e-5, 10.0, "ARS443", 1e-7)
    psi, th, u = coll_state(n_r, n_phi, 1e-3, 2, psi_amp=1e-5, u_amp=1e-5)
    set_both(gpu, ora, psi, th, u)
    for k in range(2):
        gpu.step(1)
        ora.step()
        e = compare_state(gpu, ora, 2e-12, tol_w=max(2e-12, n_r ** 4 * EPS / 4))
        print("collocation n257 step %d: %s" % (k + 1, {a: "%.2e" % b for a, b in e.items()}))
    gpu.close()


def test_collocation_option_limits():
    from paper_1902_07092_gb300.binding import PizzaError, Solver, pizza_set_option
    s = Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    with pytest.raises(PizzaError) as ei:
        pizza_set_option(s.ctx, "radial", 3)
    assert ei.value.code == -8
    pizza_set_option(s.ctx, "radial", 2)   # Galerkin bases (Appendix B)
    pizza_set_option(s.ctx, "radial", 0)
    assert s.ctx is not None
    s.close()
    big = Solver(1025, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    with pytest.raises(PizzaError) as ei:
        pizza_set_option(big.ctx, "radial", 0)
    assert ei.value.code == -8
    big.close()


def test_integration_grid_fields_match_oracle():
    """pizza_get_grid of the integration formulation: u_s = (h^2/s) dPsi/dphi,
    u_phi, omega and theta on the physical grid."""
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi = 65, 192
    Ra = 2.0 * critical_rayleigh(1e-3)
    gpu = Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4)
    ora = IntegrationStepper(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "CNAB2", 1e-4)
    th = inputs.theta_init(n_r, n_phi, 1.0, 4, cfg=7, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1.0, 6, cfg=9, m_min=0)[0].real.copy()
    gpu.set_state(th, psi, u)
    v, uphi, w, t = radial_fields(ora.g, psi, th, u)
    us = (ora.g.h2 / ora.g.s)[:, None] * v
    ref = [fo.to_grid(f, n_phi) for f in (us, uphi, w, t)]
    got = gpu.get_grid()
    errs = [rel_l2(a, b) for a, b in zip(got, ref)]
    print("integration grid fields: us %.2e uphi %.2e omega %.2e theta %.2e" % tuple(errs))
    assert max(errs) <= max(1e-12, 4 * n_r * n_r * EPS)
    gpu.close()
