"""Batches in one CUDA graph and the autotuner's explicit-stage launch shapes:
both change the schedule, not the arithmetic, so the states must equal those of
contexts stepped one by one, bit for bit.  The autotuner's other choice, the
solve with one CTA per mode or per system, sums the Schur steps in another order:
there the states agree to the accuracy of the solve."""
import numpy as np
import pytest

from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh

pytestmark = pytest.mark.gpu

RUNS = [  # n_r, n_phi, E, Ra/Ra_c, scheme, dt, radial
    (33, 96, 1e-3, 2.0, "CNAB2", 1e-4, "integration"),
    (65, 192, 1e-4, 5.0, "SBDF3", 1e-6, "integration"),
    (33, 96, 1e-3, 3.0, "ARS443", 1e-4, "integration"),
    (33, 96, 1e-3, 2.0, "CNAB2", 1e-4, "collocation"),
    (129, 384, 1e-5, 10.0, "SBDF2", 1e-7, "integration"),
]


def _make(k, run):
    from paper_1902_07092_gb300.binding import Solver
    n_r, n_phi, E, rf, scheme, dt, radial = run
    s = Solver(n_r, n_phi, E, rf * critical_rayleigh(E), 1.0, 0.35, scheme, dt, radial=radial)
    nc = n_r if radial == "collocation" else None
    th = inputs.theta_init(n_r, n_phi, 1e-2, 100 + k, cfg=4, n_c=nc)
    z, zu = inputs.zero_state(n_r, n_phi, n_c=nc)
    s.set_state(th, z, zu)
    return s, (th, z, zu)


def test_batch_graph_equals_contexts_stepped_alone():
    from paper_1902_07092_gb300.binding import Batch
    alone, batched, states = [], [], []
    for k, run in enumerate(RUNS):
        a, st = _make(k, run)
        a.step(7)
        alone.append(a.get_state())
        a.close()
        b, st = _make(k, run)
        batched.append(b)
        states.append(st)
    batch = Batch(batched)
    batch.step(7)                        # capture, instantiate, launch
    for b, ref in zip(batched, alone):
        for x, y in zip(b.get_state(), ref):
            assert np.array_equal(x, y)
    for b, st in zip(batched, states):   # back to the graph's start state: relaunch
        b.set_state(*st)
    batch.step(7)
    for b, ref in zip(batched, alone):
        for x, y in zip(b.get_state(), ref):
            assert np.array_equal(x, y)
    batch.step(5)                        # another length: a new capture from the current state
    for b in batched:
        assert all(np.all(np.isfinite(x)) for x in b.get_state())
    batch.close()
    for b in batched:
        b.close()


def test_autotuned_launch_shapes_do_not_change_results():
    ref = []
    for k, run in enumerate(RUNS[:3] + RUNS[4:]):
        a, _ = _make(k, run)
        a.step(4)
        ref.append(a.get_state())
        a.close()
    from tests.parity_util import rel_l2
    for k, run in enumerate(RUNS[:3] + RUNS[4:]):
        a, st = _make(k, run)
        nb, th = a.autotune()
        assert nb in (1, 2, 4) and th in (128, 256, 512)
        a.set_state(*st)
        a.step(4)
        got = a.get_state()
        d = rel_l2(np.concatenate([np.ravel(x) for x in got]), np.concatenate([np.ravel(x) for x in ref[k]]))
        assert d <= 1e-13, (k, d)
        a.close()


def test_explicit_launch_shapes_give_the_same_states():
    """Options radial_batch (1, 2, 4) and phi_threads (256, 512): the same steps,
    bitwise, in FP64 and in mixed precision."""
    from paper_1902_07092_gb300.binding import pizza_set_option
    run = RUNS[4]
    for prec in (0, 1):
        ref = None
        for nb in (1, 2, 4):
            for th in (256, 512):
                a, st = _make(0, run)
                pizza_set_option(a.ctx, "precision", prec)
                pizza_set_option(a.ctx, "radial_batch", nb)
                pizza_set_option(a.ctx, "phi_threads", th)
                a.set_state(*st)
                a.step(3)
                got = a.get_state()
                if ref is None:
                    ref = got
                else:
                    for x, y in zip(got, ref):
                        assert np.array_equal(x, y), (prec, nb, th)
                a.close()


def test_option_change_forces_a_new_graph():
    """Two launches from the same start state with an option changed in between
    (precision: no buffer is freed, but the explicit kernels differ): the second
    launch is captured anew and matches a context stepped alone in the new mode.
    The same check guards option changes that rebuild the factors (dt)."""
    from paper_1902_07092_gb300.binding import Batch, pizza_set_option
    run = RUNS[0]
    a, st = _make(0, run)
    b = Batch([a])
    b.step(3)
    fp64 = a.get_state()
    pizza_set_option(a.ctx, "precision", 1)
    a.set_state(*st)
    b.step(3)
    got = a.get_state()
    b.close()
    ref, st2 = _make(0, run)
    pizza_set_option(ref.ctx, "precision", 1)
    ref.set_state(*st2)
    ref.step(3)
    for x, y in zip(got, ref.get_state()):
        assert np.array_equal(x, y)
    assert not all(np.array_equal(x, y) for x, y in zip(got, fp64))
    a.close()
    ref.close()


def test_batch64_members_in_the_graph_match_the_oracle():
    """Four members of the 64-run batched workload -- the first run of each n_r,
    and run 8, the n_r = 513 run with the smallest E (1.04e-6, where the
    streamfunction solve leans on its refinement most) -- stepped twice inside
    one batch graph, each against the oracle's banded Appendix A stepper.  Bars
    as the single-run tests: 1e-12 (n_r <= 129), 2e-12 (257), 5e-12 (513; the
    streamfunction systems' effective condition grows with N_c)."""
    from oracle.banded import BandedIntegrationStepper
    from paper_1902_07092_gb300.binding import Batch, Solver
    from tests.parity_util import assert_state_close, critical_rayleigh_interp
    runs = inputs.batch_runs(64)
    pick = {}
    for i, r in enumerate(runs):
        pick.setdefault(r["n_r"], i)
    idx = sorted(set(pick.values()) | {8})
    assert runs[8]["n_r"] == 513 and runs[8]["E"] == min(r["E"] for r in runs)
    sols, oras = [], []
    for i in idx:
        r = runs[i]
        Ra = r["ra_factor"] * critical_rayleigh_interp(r["E"])
        s = Solver(r["n_r"], r["n_phi"], r["E"], Ra, r["Pr"], r["eta"], r["scheme"], r["dt"])
        o = BandedIntegrationStepper(r["n_r"], r["n_phi"], r["E"], Ra, r["Pr"], r["eta"], r["scheme"], r["dt"])
        th = inputs.theta_init(r["n_r"], r["n_phi"], r["amp"], r["seed"], cfg=r["cfg"])
        z, zu = inputs.zero_state(r["n_r"], r["n_phi"])
        s.set_state(th, z, zu)
        o.set_state(z, th, zu)
        sols.append(s)
        oras.append(o)
    batch = Batch(sols)
    batch.step(2)
    tol = {65: 1e-12, 129: 1e-12, 257: 2e-12, 513: 5e-12}
    for i, s, o in zip(idx, sols, oras):
        o.step()
        o.step()
        e = assert_state_close(s.get_state(), o.y, tol[runs[i]["n_r"]], oracle=o)
        print("batch64 run %d (n_r %d, n_phi %d, E %.3g): state %.2e psi %.2e theta %.2e u %.2e" % (
            i, runs[i]["n_r"], runs[i]["n_phi"], runs[i]["E"], e["state"], e["psi"], e["theta"], e["u"]))
    batch.close()
    for s in sols:
        s.close()
