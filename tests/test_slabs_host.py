"""The m-slab decomposition (Section 5) on the host: the partition, the two
transposes' index arithmetic, and the same exchange code run by gloo ranks
(world sizes 2 and 3) on CPU tensors, with the oracle's three explicit stages as
the per-mode and per-radius work.  Every stage is column- (mode) or row-
(radius) independent, so the distributed explicit terms and one step must equal
the single-rank ones bit for bit."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_1902_07092_gb300 import inputs
from paper_1902_07092_gb300.slabs import (LoopbackHub, Plan, balanced_slabs, pack1, pack2, transpose, unpack1,
                                          unpack2)


@pytest.mark.parametrize("n,parts", [(9, 1), (9, 2), (9, 4), (9, 9), (257, 3), (2049, 8), (2049, 7), (17, 5)])
def test_slabs_cover_contiguous_and_balanced(n, parts):
    s = balanced_slabs(np.ones(n), parts)
    assert s[0][0] == 0 and s[-1][1] == n
    assert all(a < b for a, b in s)
    assert all(s[i][1] == s[i + 1][0] for i in range(parts - 1))
    sizes = [b - a for a, b in s]
    assert max(sizes) - min(sizes) <= 1


def test_slabs_reject_more_parts_than_items():
    with pytest.raises(ValueError):
        balanced_slabs(np.ones(3), 4)


@pytest.mark.parametrize("M,n_r,world", [(9, 17, 2), (9, 17, 3), (33, 65, 4), (5, 9, 5)])
def test_transposes_rebuild_the_global_layouts(M, n_r, world):
    """Ranks as plain loops with numpy buffers: after transpose 1 every rank's
    radius rows hold every mode of the global array, after transpose 2 every
    rank's mode columns hold every radius."""
    rng = np.random.default_rng(M * n_r)
    glob = rng.standard_normal((n_r, 4, M)) + 1j * rng.standard_normal((n_r, 4, M))
    plans = [Plan(M, n_r, world, r) for r in range(world)]
    for which in (1, 2):
        G = []
        for p in plans:
            g = np.full((n_r, 4, M), np.nan, complex)
            m0, m1 = p.m_range
            k0, k1 = p.k_range
            if which == 1:
                g[:, :, m0:m1] = glob[:, :, m0:m1]       # a1 wrote this rank's modes
            else:
                g[k0:k1] = glob[k0:k1]                   # a2 wrote this rank's radii
            G.append(g)
        sends = [(pack1 if which == 1 else pack2)(G[r], plans[r]) for r in range(world)]
        for r, p in enumerate(plans):
            ss = [plans[q].send1 if which == 1 else plans[q].send2 for q in range(world)]
            chunks = []
            for q in range(world):
                off = int(np.sum(ss[q][:r]))
                chunks.append(sends[q][off:off + ss[q][r]])
            recv = np.concatenate(chunks)
            assert recv.size == sum(p.recv1 if which == 1 else p.recv2)
            (unpack1 if which == 1 else unpack2)(recv, G[r], p)
            m0, m1 = p.m_range
            k0, k1 = p.k_range
            if which == 1:
                assert np.array_equal(G[r][k0:k1], glob[k0:k1])
            else:
                assert np.array_equal(G[r][:, :, m0:m1], glob[:, :, m0:m1])


def test_loopback_transport_in_threads():
    import threading

    import torch

    from paper_1902_07092_gb300.slabs import LoopbackTransport
    M, n_r, world = 9, 17, 3
    glob = torch.randn(n_r, 4, M, dtype=torch.complex128)
    hub = LoopbackHub(world)
    out = [None] * world

    def run(r):
        p = Plan(M, n_r, world, r)
        G = torch.zeros(n_r, 4, M, dtype=torch.complex128)
        m0, m1 = p.m_range
        G[:, :, m0:m1] = glob[:, :, m0:m1]
        transpose(1, G, p, LoopbackTransport(hub, r))
        out[r] = (p, G)

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for p, G in out:
        k0, k1 = p.k_range
        assert torch.equal(G[k0:k1], glob[k0:k1])


# ---------------------------------------------- gloo ranks with oracle stages
N_R, N_PHI, E, RA, DT = 17, 24, 1e-3, 8e4, 1e-4


def _problem():
    from oracle.stepper import IntegrationStepper
    st = IntegrationStepper(N_R, N_PHI, E, RA, 1.0, 0.35, "CNAB2", DT)
    th = inputs.theta_init(N_R, N_PHI, 1.0, 9, cfg=7, m_min=0)
    ps = inputs.theta_init(N_R, N_PHI, 0.1, 10, cfg=8)
    ps[0] = 0.0
    u = inputs.theta_init(N_R, N_PHI, 0.5, 11, cfg=9, m_min=0)[0].real.copy()
    st.set_state(ps, th, u)
    return st


def _stage_a1(st, cols):
    """The oracle's radial synthesis (step 1 of its explicit terms) on the modes
    in ``cols`` (others zeroed; same array shapes for every caller)."""
    from oracle.explicit import radial_fields
    ps, th, u = (np.array(x) for x in st.y)
    keep = np.zeros(st.g.M, bool)
    keep[cols[0]:cols[1]] = True
    ps[~keep] = 0.0
    th[~keep] = 0.0
    if cols[0] > 0:
        u = np.zeros_like(u)
    return np.stack(radial_fields(st.g, ps, th, u), axis=1)          # [k][4][m]


def _stage_a2(st, G1, rows):
    """The oracle's azimuthal products (step 2) on the radii in ``rows``."""
    from oracle.explicit import products
    f = [np.where(np.arange(N_R)[:, None] < rows[1], G1[:, i], 0.0) for i in range(4)]
    f = [np.where(np.arange(N_R)[:, None] >= rows[0], x, 0.0) for x in f]
    return np.stack(products(st.g, *f), axis=1)


def _stage_a3(st, G2):
    """The oracle's flux divergences, analysis and integrated right-hand sides
    (steps 3 to 5) from the product spectra, for every mode."""
    from oracle import chebyshev as ch
    from oracle.explicit import nonlinear_grid
    g, ops = st.g, st.ops
    ps, th, _ = st.y
    Nw_g, Nt_g, Nu_g = nonlinear_grid(g, *(G2[:, i] for i in range(4)))
    nc = g.n_c
    Nw = ch.analysis(Nw_g, g.n_r)[:nc].T
    Nt = ch.analysis(Nt_g, g.n_r)[:nc].T
    Nu = ch.analysis(Nu_g, g.n_r)[:nc].real
    m = g.m[:, None]
    e_psi = (ops.C @ ((ops.Ra / ops.Pr) * (1j * m / ops.ann.s_o) * th + Nw).T).T
    e_psi[0] = 0.0
    e_th = -(ops.D @ Nt.T).T - ops.tc_coef * 1j * m * (ops.G @ ps.T).T
    e_u = -(ops.D @ Nu)
    return e_psi, e_th, e_u


def _explicit_and_step(rank, world, transport):
    """One explicit evaluation and one SBDF1-like step of the modes of ``rank``:
    a1 on its modes, transpose 1, a2 on its radii, transpose 2, a3, then the
    per-mode solves of (Mass - dt Lin) y = Mass y_n + dt e."""
    import torch
    st = _problem()
    p = Plan(st.g.M, N_R, world, rank)
    G1 = torch.from_numpy(_stage_a1(st, p.m_range))
    transpose(1, G1, p, transport)
    G2 = torch.from_numpy(_stage_a2(st, G1.numpy(), p.k_range))
    transpose(2, G2, p, transport)
    e = _stage_a3(st, G2.numpy())
    m0, m1 = p.m_range
    lp, lt, lu_ = st.lu(1.0)
    mp, mt, mu = st.mass(st.y)
    new_p = np.zeros((m1 - m0, st.n_c), complex)
    new_t = np.zeros((m1 - m0, st.n_c), complex)
    for i, m in enumerate(range(m0, m1)):
        rp = mp[m] + DT * e[0][m]
        rt = mt[m] + DT * e[1][m]
        rp[:4] = 0.0
        rt[:2] = 0.0
        if m > 0:
            new_p[i] = st._solve_refined(*lp[m], rp)
        new_t[i] = st._solve_refined(*lt[m], rt)
    new_u = None
    if m0 == 0:
        ru = mu + DT * e[2]
        ru[:2] = 0.0
        new_u = st._solve_refined(*lu_, ru)
    return (m0, m1), (e[0][m0:m1], e[1][m0:m1], e[2] if m0 == 0 else None), (new_p, new_t, new_u)


def _gloo_rank(rank, world, port, outdir):
    import torch.distributed as dist

    from paper_1902_07092_gb300.slabs import DistTransport
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng, e, y = _explicit_and_step(rank, world, DistTransport())
        np.savez(os.path.join(outdir, "r%d.npz" % rank), rng=np.array(rng), ep=e[0], et=e[1],
                 eu=e[2] if e[2] is not None else np.zeros(0), yp=y[0], yt=y[1],
                 yu=y[2] if y[2] is not None else np.zeros(0))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class _NoTransport:
    def all_to_all(self, send, ss, rs):
        return send


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_single_rank_bitwise(world):
    import torch.multiprocessing as mp
    (m0, m1), e1, y1 = _explicit_and_step(0, 1, _NoTransport())
    assert (m0, m1) == (0, N_PHI // 3 + 1)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_gloo_rank, args=(world, _free_port(), d), nprocs=world, join=True)
        got_ep = np.zeros_like(e1[0])
        got_et = np.zeros_like(e1[1])
        got_yp = np.zeros_like(y1[0])
        got_yt = np.zeros_like(y1[1])
        seen = np.zeros(m1, bool)
        for r in range(world):
            z = np.load(os.path.join(d, "r%d.npz" % r))
            a, b = z["rng"]
            seen[a:b] = True
            got_ep[a:b], got_et[a:b] = z["ep"], z["et"]
            got_yp[a:b], got_yt[a:b] = z["yp"], z["yt"]
            if a == 0:
                assert np.array_equal(z["eu"], e1[2])
                assert np.array_equal(z["yu"], y1[2])
        assert seen.all()
    assert np.array_equal(got_ep, e1[0]) and np.array_equal(got_et, e1[1])
    assert np.array_equal(got_yp, y1[0]) and np.array_equal(got_yt, y1[1])
    # and the single-rank pipeline is the oracle's explicit stage itself
    from oracle.explicit import explicit_terms
    st = _problem()
    ref = explicit_terms(st.g, *st.y)
    for a, b in zip(e1, ref):
        assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(b)
