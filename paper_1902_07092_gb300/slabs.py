"""m-slab decomposition of one time step over ranks (Section 5).

The paper distributes a run over MPI ranks with a one-dimensional decomposition:
the radial work -- Chebyshev transforms, flux divergences, right-hand sides and
the implicit solves -- is independent per azimuthal wavenumber m, the azimuthal
transforms and grid products are independent per radius, and two all-to-all
transposes with uneven counts join the two layouts in every evaluation of the
explicit terms.  Here a rank is one GPU (one process, torch.distributed with the
NCCL backend) or, in the host tests, one gloo process.

Partition.  Modes are cut into contiguous slabs of near-equal size: every mode
costs the same in a1, a3 and the solve (same transform lengths, same band
widths; m = 0 trades the streamfunction system for the zonal-flow one).  Radii
are cut the same way for a2.  The paper balances the same way (N_m/N_ranks modes
and N_r/N_ranks radii per rank).

Grids.  Both grid arrays are radius-major [k][field][m] (n_r x 4 x M complex),
the library's layout, held at full size on every rank.  After a1 rank r holds the
columns m of its slab for every k; transpose 1 sends the rows of rank q's radius
slab, restricted to r's columns, to q.  After a2 rank q holds the rows of its
radius slab for every m; transpose 2 sends the columns of rank r's mode slab,
restricted to q's rows, to r.  Each transpose is one ``all_to_all_single`` with
uneven split sizes: NCCL's grouped send/receive on GPUs, gloo on CPUs.

This module is plumbing: index arithmetic and data movement, no method
arithmetic.  ``SlabSolver`` plugs it into the library through pizza_set_slab.
"""
import ctypes
import threading
import traceback

import numpy as np


# ------------------------------------------------------------------ partition
def balanced_slabs(weights, parts):
    """Contiguous [lo, hi) ranges covering range(len(weights)), each non-empty,
    cut where the running weight crosses j / parts of the total."""
    w = np.asarray(weights, dtype=float)
    n = len(w)
    if not 1 <= parts <= n:
        raise ValueError("need 1 <= parts <= %d items" % n)
    c = np.concatenate([[0.0], np.cumsum(w)])
    cuts = [0]
    for j in range(1, parts):
        t = c[-1] * j / parts
        b = int(np.searchsorted(c, t, side="left"))
        if b > 0 and abs(c[b - 1] - t) <= abs(c[b] - t):
            b -= 1
        b = min(max(b, cuts[-1] + 1), n - (parts - j))   # keep every part non-empty
        cuts.append(b)
    cuts.append(n)
    return [(cuts[i], cuts[i + 1]) for i in range(parts)]


def mode_slabs(M, world):
    return balanced_slabs(np.ones(M), world)


def radius_slabs(n_r, world):
    return balanced_slabs(np.ones(n_r), world)


class Plan:
    """Slabs of every rank and the split sizes (in complex elements) of both
    transposes as seen from ``rank``."""

    def __init__(self, M, n_r, world, rank):
        self.M, self.n_r, self.world, self.rank = M, n_r, world, rank
        self.ms = mode_slabs(M, world)
        self.ks = radius_slabs(n_r, world)
        m0, m1 = self.ms[rank]
        k0, k1 = self.ks[rank]
        nm = [b - a for a, b in self.ms]
        nk = [b - a for a, b in self.ks]
        # transpose 1: to q, my columns of q's rows; from r, r's columns of my rows
        self.send1 = [nk[q] * 4 * (m1 - m0) for q in range(world)]
        self.recv1 = [(k1 - k0) * 4 * nm[r] for r in range(world)]
        # transpose 2: to r, r's columns of my rows; from q, my columns of q's rows
        self.send2 = [(k1 - k0) * 4 * nm[r] for r in range(world)]
        self.recv2 = [nk[q] * 4 * (m1 - m0) for q in range(world)]

    @property
    def m_range(self):
        return self.ms[self.rank]

    @property
    def k_range(self):
        return self.ks[self.rank]


# ------------------------------------------------------------- pack / unpack
def _cat(parts, like):
    flat = [p.reshape(-1) for p in parts]
    if hasattr(like, "new_empty"):          # torch
        import torch
        return torch.cat(flat) if flat else like.new_empty(0)
    return np.concatenate(flat)


def pack1(G, plan):
    """Send buffer of transpose 1: for q = 0..world-1, G[k in q's radii, :, my modes]."""
    m0, m1 = plan.m_range
    return _cat([G[a:b, :, m0:m1] for a, b in plan.ks], G)


def unpack1(buf, G, plan):
    k0, k1 = plan.k_range
    off = 0
    for (a, b), n in zip(plan.ms, plan.recv1):
        G[k0:k1, :, a:b] = buf[off:off + n].reshape(k1 - k0, 4, b - a)
        off += n


def pack2(G, plan):
    """Send buffer of transpose 2: for r = 0..world-1, G[my radii, :, r's modes]."""
    k0, k1 = plan.k_range
    return _cat([G[k0:k1, :, a:b] for a, b in plan.ms], G)


def unpack2(buf, G, plan):
    m0, m1 = plan.m_range
    off = 0
    for (a, b), n in zip(plan.ks, plan.recv2):
        G[a:b, :, m0:m1] = buf[off:off + n].reshape(b - a, 4, m1 - m0)
        off += n


def transpose(which, G, plan, transport):
    """Transpose 1 (which = 1, after a1) or 2 (after a2) of the grid G in place."""
    if which == 1:
        send, ssz, rsz, unpack = pack1(G, plan), plan.send1, plan.recv1, unpack1
    else:
        send, ssz, rsz, unpack = pack2(G, plan), plan.send2, plan.recv2, unpack2
    recv = transport.all_to_all(send, ssz, rsz)
    unpack(recv, G, plan)


# ----------------------------------------------------------------- transports
class DistTransport:
    """torch.distributed all-to-all with uneven splits (NCCL or gloo)."""

    def __init__(self, group=None):
        self.group = group

    def all_to_all(self, send, send_splits, recv_splits):
        import torch.distributed as dist
        recv = send.new_empty(int(sum(recv_splits)))
        dist.all_to_all_single(recv, send.contiguous(), list(map(int, recv_splits)), list(map(int, send_splits)),
                               group=self.group)
        return recv


class LoopbackHub:
    """Ranks that are threads of one process (several contexts on one device):
    each posts its send buffer, waits for the others, and copies its chunks."""

    def __init__(self, world, timeout=120.0):
        self.world = world
        # a rank that fails leaves the others a broken barrier, not a hang
        self.barrier = threading.Barrier(world, timeout=timeout)
        self.posted = [None] * world


class LoopbackTransport:
    def __init__(self, hub, rank, synchronize=None):
        self.hub, self.rank = hub, rank
        self.synchronize = synchronize or (lambda: None)

    def all_to_all(self, send, send_splits, recv_splits):
        h, r = self.hub, self.rank
        self.synchronize()                       # the packed buffer is complete
        h.posted[r] = (send, [0] + list(np.cumsum(send_splits)))
        h.barrier.wait()
        chunks = []
        for q in range(h.world):
            buf, offs = h.posted[q]
            chunks.append(buf[offs[r]:offs[r + 1]])
        recv = _cat(chunks, send)
        self.synchronize()                       # the copies are done before anyone moves on
        h.barrier.wait()
        return recv


# ------------------------------------------------------------ library binding
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_void_p)


class SlabSolver:
    """One rank's share of a run: a binding.Solver restricted to this rank's
    modes and radii, its grid arrays in torch buffers on ``device`` and the two
    transposes done by ``transport`` inside the step (the library calls back)."""

    def __init__(self, solver, plan, transport, device):
        import torch
        from . import binding as B
        self.solver, self.plan, self.transport = solver, plan, transport
        n = solver.n_r * 4 * solver.M
        self.g1 = torch.zeros(n, dtype=torch.complex128, device=device)
        self.g2 = torch.zeros(n, dtype=torch.complex128, device=device)
        self.error = None
        self._cb = EXCHANGE_FN(self._exchange)    # referenced for the context's lifetime
        m0, m1 = plan.m_range
        k0, k1 = plan.k_range
        B.pizza_set_slab(solver.ctx, m0, m1, k0, k1, self.g1, self.g2, self._cb)

    def _grid(self, which, elem_bytes):
        import torch
        buf = self.g1 if which == 1 else self.g2
        n = self.solver.n_r * 4 * self.solver.M
        if elem_bytes == 8:
            buf = buf.view(torch.complex64)[:n]
        return buf.view(self.solver.n_r, 4, self.solver.M)

    def _exchange(self, user, which, grid, elem_bytes, stream):
        try:
            import torch
            st = torch.cuda.ExternalStream(stream)
            with torch.cuda.stream(st):
                transpose(which, self._grid(which, elem_bytes), self.plan, self.transport)
            return 0
        except Exception:                       # reported to the library as a failed step
            self.error = traceback.format_exc()
            return 1

    def state(self):
        """This rank's modes of (Psi, theta, u_bar); u_bar only on the rank of m = 0."""
        ps, th, u = self.solver.get_state()
        m0, m1 = self.plan.m_range
        return ps[m0:m1], th[m0:m1], (u if m0 == 0 else None)

    def close(self):
        from . import binding as B
        B.pizza_set_slab(self.solver.ctx, 0, self.solver.M, 0, self.solver.n_r, None, None, None)
