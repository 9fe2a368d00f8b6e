"""The m-slab decomposition (Section 5) through the library on one GPU: R
contexts, one per rank, each advancing its slab of modes and radii in its own
host thread, the transposes between their grid buffers done by the loopback
transport (host barriers and device copies; no kernel waits on another).  The
per-mode and per-radius kernels do the same arithmetic on a slab as on the whole
problem, so explicit terms and steps must equal the single context's bit for
bit."""
import threading

import numpy as np
import pytest

from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh

pytestmark = pytest.mark.gpu


def _run_ranks(world, n_r, n_phi, scheme, dt, steps, precision=0, radial="integration", E=1e-3, rf=3.0):
    import torch
    from paper_1902_07092_gb300 import binding as B
    from paper_1902_07092_gb300.slabs import LoopbackHub, LoopbackTransport, Plan, SlabSolver
    Ra = rf * critical_rayleigh(E)
    th = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=7, m_min=0)
    ps = inputs.theta_init(n_r, n_phi, 1e-2, 6, cfg=8)
    ps[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 0.3, 7, cfg=9, m_min=0)[0].real.copy()
    dev = torch.device("cuda", 0)

    def make():
        s = B.Solver(n_r, n_phi, E, Ra, 1.0, 0.35, scheme, dt, radial=radial)
        if precision:
            B.pizza_set_option(s.ctx, "precision", precision)
        s.set_state(th, ps, u)
        return s

    whole = make()
    e_whole = whole.explicit_terms()
    whole.step(steps)
    y_whole = whole.get_state()
    whole.close()

    hub = LoopbackHub(world)
    sols = [make() for _ in range(world)]
    slabs = [SlabSolver(sols[r], Plan(sols[r].M, n_r, world, r),
                        LoopbackTransport(hub, r, lambda: torch.cuda.current_stream().synchronize()), dev)
             for r in range(world)]
    out, errs = [None] * world, [None] * world

    def run(r):
        try:
            torch.cuda.set_device(0)
            e = sols[r].explicit_terms()
            sols[r].step(steps)
            out[r] = (e, sols[r].get_state())
        except Exception as ex:  # reported below
            errs[r] = "%r %s" % (ex, slabs[r].error)

    th_ = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th_:
        t.start()
    for t in th_:
        t.join()
    assert not any(errs), errs
    for r in range(world):
        m0, m1 = slabs[r].plan.m_range
        e, y = out[r]
        assert np.array_equal(e[0][m0:m1], e_whole[0][m0:m1])
        assert np.array_equal(e[1][m0:m1], e_whole[1][m0:m1])
        assert np.array_equal(y[0][m0:m1], y_whole[0][m0:m1])
        assert np.array_equal(y[1][m0:m1], y_whole[1][m0:m1])
        if m0 == 0:
            assert np.array_equal(e[2], e_whole[2])
            assert np.array_equal(y[2], y_whole[2])
        slabs[r].close()
        sols[r].close()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("scheme", ["CNAB2", "SBDF3", "BPR353"])
def test_slab_ranks_equal_the_whole_step(world, scheme):
    _run_ranks(world, 65, 192, scheme, 1e-4, 3)


def test_slab_ranks_sparse_workload_size():
    """n_r = 257, n_phi = 768, E = 1e-5, Ra = 10 Ra_c, ARS443, 4 ranks."""
    _run_ranks(4, 257, 768, "ARS443", 1e-7, 2, E=1e-5, rf=10.0)


def test_slab_ranks_mixed_precision_and_galerkin():
    _run_ranks(2, 129, 384, "SBDF3", 1e-4, 3, precision=1)
    _run_ranks(3, 65, 192, "CNAB2", 1e-4, 3, radial="galerkin")


def test_slab_option_limits():
    import torch
    from paper_1902_07092_gb300 import binding as B
    from paper_1902_07092_gb300.slabs import LoopbackHub, LoopbackTransport, Plan, SlabSolver
    s = B.Solver(33, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    sl = SlabSolver(s, Plan(s.M, 33, 2, 0), LoopbackTransport(LoopbackHub(2), 0), torch.device("cuda", 0))
    for call in (lambda: s.diagnostics(), lambda: s.tape_begin(5), lambda: B.pizza_set_option(s.ctx, "radial", 0)):
        with pytest.raises(B.PizzaError) as ei:
            call()
        assert ei.value.code == -8
    with pytest.raises(B.PizzaError) as ei:
        B.pizza_set_slab(s.ctx, 3, 2, 0, 33, sl.g1, sl.g2, sl._cb)
    assert ei.value.code == -1
    sl.close()
    s.diagnostics()                      # the whole step again
    s.close()


def test_slab_ranks_through_nccl_all_to_all():
    """The same exchange code over torch.distributed's NCCL backend (one rank on
    this GPU: the all-to-alls run, each rank's share being everything): the
    decomposed step equals the whole step bit for bit."""
    import socket

    import torch
    import torch.distributed as dist
    from paper_1902_07092_gb300 import binding as B
    from paper_1902_07092_gb300.slabs import DistTransport, Plan, SlabSolver
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        n_r, n_phi = 129, 384
        Ra = 3.0 * critical_rayleigh(1e-3)
        th = inputs.theta_init(n_r, n_phi, 1.0, 5, cfg=7, m_min=0)
        z, zu = inputs.zero_state(n_r, n_phi)
        whole = B.Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4)
        whole.set_state(th, z, zu)
        whole.step(3)
        ref = whole.get_state()
        whole.close()
        s = B.Solver(n_r, n_phi, 1e-3, Ra, 1.0, 0.35, "SBDF3", 1e-4)
        slab = SlabSolver(s, Plan(s.M, n_r, 1, 0), DistTransport(), torch.device("cuda", 0))
        s.set_state(th, z, zu)
        s.step(3)
        assert slab.error is None
        for a, b in zip(s.get_state(), ref):
            assert np.array_equal(a, b)
        slab.close()
        s.close()
    finally:
        dist.destroy_process_group()
