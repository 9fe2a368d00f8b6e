"""pizza_explicit_terms_noalloc, the entry point for callers that cannot allocate
device memory: called through the C interface with caller-owned device arrays,
it must give the explicit right-hand sides of the regular context path
(pizza_explicit_terms), on two calls in a row with different states.

This file is collected last so that a run stopping at the first failure has
run every other test first."""
import numpy as np
import pytest

from paper_1902_07092_gb300 import inputs
from tests.parity_util import critical_rayleigh, rel_l2

pytestmark = pytest.mark.gpu


def _state(n_r, n_phi, seed):
    th = inputs.theta_init(n_r, n_phi, 1.0, seed, cfg=7, m_min=0)
    psi = inputs.theta_init(n_r, n_phi, 1.0, seed + 1, cfg=8)
    psi[0] = 0.0
    u = inputs.theta_init(n_r, n_phi, 1.0, seed + 2, cfg=9, m_min=0)[0].real.copy()
    return psi, th, u


@pytest.mark.parametrize("n_r,n_phi", [(33, 96), (257, 768)])
def test_noalloc_matches_context_path_on_two_calls(n_r, n_phi):
    import torch
    from paper_1902_07092_gb300 import binding as B
    E, Pr, eta = 1e-3, 1.0, 0.35
    Ra = 2.0 * critical_rayleigh(E)
    ref_solver = B.Solver(n_r, n_phi, E, Ra, Pr, eta, "CNAB2", 1e-4)
    dev = torch.device("cuda", 0)
    tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
    for seed in (11, 23):                      # two calls in a row
        psi, th, u = _state(n_r, n_phi, seed)
        ref_solver.set_state(th, psi, u)
        rp, rt, ru = ref_solver.explicit_terms()
        d_psi = torch.from_numpy(psi).to(dev)
        d_th = torch.from_numpy(th).to(dev)
        d_u = torch.from_numpy(u).to(dev)
        e_psi = torch.full_like(d_psi, float("nan"))
        e_th = torch.full_like(d_th, float("nan"))
        e_u = torch.full_like(d_u, float("nan"))
        stream = torch.cuda.current_stream(dev)
        B.pizza_explicit_terms_noalloc(n_r, n_phi, Ra, Pr, eta, d_psi, d_th, d_u, e_psi, e_th, e_u,
                                       stream.cuda_stream)
        torch.cuda.synchronize()
        gp, gt, gu = (x.cpu().numpy() for x in (e_psi, e_th, e_u))
        assert np.all(np.isfinite(gp)) and np.all(np.isfinite(gt)) and np.all(np.isfinite(gu))
        assert rel_l2(gp, rp) <= tol
        assert rel_l2(gt, rt) <= tol
        assert rel_l2(gu, ru) <= tol
    ref_solver.close()


def test_noalloc_calls_ordered_on_one_stream_with_different_sizes():
    """Two calls queued back to back on one non-blocking stream, with no host
    synchronisation between them, whose sizes and radius ratios differ: the
    second call rewrites the shared tables, which must not disturb the first."""
    import torch
    from paper_1902_07092_gb300 import binding as B
    dev = torch.device("cuda", 0)
    cases = [(257, 768, 0.35, 1e-5, 11), (65, 192, 0.5, 1e-3, 29)]
    refs, outs, keep = [], [], []
    for n_r, n_phi, eta, E, seed in cases:
        Ra = 3.0 * critical_rayleigh(E)
        psi, th, u = _state(n_r, n_phi, seed)
        ref = B.Solver(n_r, n_phi, E, Ra, 1.0, eta, "CNAB2", 1e-4)
        ref.set_state(th, psi, u)
        refs.append(ref.explicit_terms())
        ref.close()
        keep.append((n_r, n_phi, eta, Ra, [torch.from_numpy(x).to(dev) for x in (psi, th, u)]))
    torch.cuda.synchronize()
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        for n_r, n_phi, eta, Ra, (d_psi, d_th, d_u) in keep:
            e = [torch.full_like(x, float("nan")) for x in (d_psi, d_th, d_u)]
            B.pizza_explicit_terms_noalloc(n_r, n_phi, Ra, 1.0, eta, d_psi, d_th, d_u, *e, side.cuda_stream)
            outs.append(e)
    side.synchronize()
    for (n_r, *_), e, r in zip(cases, outs, refs):
        tol = max(1e-12, 4 * n_r * n_r * 2.0 ** -53)
        for g, want in zip(e, r):
            got = g.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, want) <= tol


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    import torch
    from paper_1902_07092_gb300 import binding as B
    dev = torch.device("cuda", 0)
    n_r, n_phi = 513, 768
    M, nc = n_phi // 3 + 1, (2 * (n_r - 1)) // 3
    a = torch.zeros((M, nc), dtype=torch.complex128, device=dev)
    u = torch.zeros(nc, dtype=torch.float64, device=dev)
    with pytest.raises(B.PizzaError) as e:
        B.pizza_explicit_terms_noalloc(n_r, n_phi, 1e5, 1.0, 0.35, a, a, u, a, a, u, None)
    assert e.value.code == -1
    assert "static scratch" in B.pizza_last_error()
