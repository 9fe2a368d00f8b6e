"""The integration/tau step in band storage, solved by the bordered algorithm of
Appendix A with a banded LU of the block D (Sections 3.2 and 4; Appendix A).

Test infrastructure only (see the package docstring).

``IntegrationStepper`` (``stepper.py``) assembles every operator of one mode as a
dense N_c x N_c matrix and solves by dense LU: O(N_c^3) per mode, which is what
lets it serve as the brute-force check, and what keeps it from running at
n_r = 2049.  This module runs the same scheme with:

* the m-independent operators of Section 3.2 (A^I = A0 + m^2 A2, B^I = B0 + m^2 B2
  + m^4 B4 + (2/E) i m C^I, C^I, D^I, E^I, F^I = F0 + m^2 F2, G^I) kept as their
  diagonals (half bandwidths 8, 6, 8, 4, 2, 2, 4: exact zeros outside), and
  every mass and implicit operator applied diagonal by diagonal;
* each tau system L = [tau rows; banded rows k >= p] (p = 4 for Psi, 2 for theta
  and u_bar) scaled row by row to unit maximum, exactly as the dense oracle does,
  then split as in Appendix A:
        L = ( A  B )   A: p x p,  B: p x (N_c - p)  (the dense tau rows)
            ( C  D )   C: (N_c - p) x p,  D: banded (N_c - p) x (N_c - p)
  D x = h and D Y = C by LAPACK's banded LU with partial pivoting (gbtrf/gbtrs,
  a library primitive), the Schur complement S = A - B Y (p x p), then
        psi_1 = S^{-1} (g - B x),   psi_2 = x - Y psi_1;
* one refinement step with an FP64 residual of the unscaled system, as in the
  dense oracle.

Nothing is reordered or fused beyond that: the right-hand sides, start-up and
stage logic are those of ``stepper.ImexScheme``.
"""
import numpy as np
from scipy.linalg.lapack import dgbtrf, dgbtrs, zgbtrf, zgbtrs

from .stepper import IntegrationStepper


def diagonals(Mat, h, q):
    """Band of a dense operator whose rows < q are zero: out[h + d, k] = Mat[k, k + d]
    for |d| <= h (zero where k + d leaves the matrix).  Checks that nothing lies
    outside the band."""
    n = Mat.shape[0]
    out = np.zeros((2 * h + 1, n), Mat.dtype)
    k = np.arange(n)
    for d in range(-h, h + 1):
        ok = (k + d >= 0) & (k + d < n)
        out[h + d, ok] = Mat[k[ok], k[ok] + d]
    rest = Mat.copy()
    for d in range(-h, h + 1):
        ok = (k + d >= 0) & (k + d < n)
        rest[k[ok], k[ok] + d] = 0.0
    if np.any(rest[q:] != 0.0):
        raise ValueError("operator has entries outside its half bandwidth %d" % h)
    return out


def band_apply(band, x):
    """y[..., k] = sum_d band[h + d, k] x[..., k + d]; band (2h+1, n) or
    (..., 2h+1, n) with leading axes matching x's."""
    h = (band.shape[-2] - 1) // 2
    n = x.shape[-1]
    y = np.zeros(np.broadcast_shapes(x.shape, band.shape[:-2] + (n,)), np.result_type(band, x))
    for d in range(-h, h + 1):
        lo, hi = max(0, -d), min(n, n - d)
        y[..., lo:hi] += band[..., h + d, lo:hi] * x[..., lo + d:hi + d]
    return y


class BorderedBandSolver:
    """Appendix A solve of one tau system given as (tau rows, band of the rows
    k >= p) -- the factors of D, Y = D^{-1} C and S^{-1} kept for repeated
    right-hand sides."""

    def __init__(self, tau_rows, band, p):
        tau_rows = np.asarray(tau_rows)
        n = band.shape[1]
        h = (band.shape[0] - 1) // 2
        cplx = np.iscomplexobj(tau_rows) or np.iscomplexobj(band)
        dt = complex if cplx else float
        self.p, self.n, self.h = p, n, h
        self.tau = tau_rows.astype(dt)
        self.band = band.astype(dt)
        self.band[:, :p] = 0.0                     # rows < p are the tau rows
        # row scales: each row of the whole system to unit maximum
        r = np.empty(n)
        r[:p] = 1.0 / np.abs(self.tau).max(axis=1)
        r[p:] = 1.0 / np.abs(self.band[:, p:]).max(axis=0)
        self.r = r
        # dense pieces of the partition (scaled rows)
        self.A = self.tau[:, :p] * r[:p, None]
        self.B = self.tau[:, p:] * r[:p, None]
        C = np.zeros((n - p, p), dt)
        for d in range(-h, h + 1):
            for i in range(p, min(n, p + h + 1)):
                j = i + d
                if 0 <= j < p:
                    C[i - p, j] = self.band[h + d, i] * r[i]
        # D in LAPACK band storage: ab[kl + ku + i - j, j] = D[i, j], kl = ku = h
        m = n - p
        ab = np.zeros((3 * h + 1, m), dt)
        for d in range(-h, h + 1):
            # D[i, i + d] = band[h + d, p + i] * r[p + i]
            i = np.arange(max(0, -d), min(m, m - d))
            ab[2 * h - d, i + d] = self.band[h + d, p + i] * r[p + i]
        self.gbtrf, self.gbtrs = (zgbtrf, zgbtrs) if cplx else (dgbtrf, dgbtrs)
        lu, piv, info = self.gbtrf(ab, h, h)
        if info != 0:
            raise np.linalg.LinAlgError("banded LU of D failed (info %d)" % info)
        self.lu, self.piv = lu, piv
        self.Y = self._dsolve(C)
        S = self.A - self.B @ self.Y
        self.S_inv = np.linalg.inv(S)

    def _dsolve(self, h_rhs):
        if self.gbtrs is dgbtrs and np.iscomplexobj(h_rhs):   # real system, complex data
            return self._dsolve(h_rhs.real) + 1j * self._dsolve(h_rhs.imag)
        x, info = self.gbtrs(self.lu, self.h, self.h, h_rhs, self.piv)
        if info != 0:
            raise np.linalg.LinAlgError("banded solve failed (info %d)" % info)
        return x

    def matvec(self, x):
        """Unscaled system times x: tau rows, then the band rows."""
        y = band_apply(self.band, x)
        y[:self.p] = self.tau @ x
        return y

    def _bordered(self, b):
        bs = b * self.r
        g, hh = bs[:self.p], bs[self.p:]
        x = self._dsolve(hh)
        psi1 = self.S_inv @ (g - self.B @ x)
        psi2 = x - self.Y @ psi1
        return np.concatenate([psi1, psi2])

    def solve(self, b):
        x = self._bordered(b)
        return x + self._bordered(b - self.matvec(x))


class BandedIntegrationStepper(IntegrationStepper):
    """``IntegrationStepper`` with band-stored operators and Appendix A solves."""

    HALF = {"A0": 8, "A2": 8, "B0": 6, "B2": 6, "B4": 6, "C": 8, "D": 4, "F0": 2, "F2": 2, "Ez": 2, "G": 4}
    ROWS = {"A0": 4, "A2": 4, "B0": 4, "B2": 4, "B4": 4, "C": 4, "D": 2, "F0": 2, "F2": 2, "Ez": 2, "G": 2}

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        ops = self.ops
        self.bands = {k: diagonals(getattr(ops, k), h, self.ROWS[k]) for k, h in self.HALF.items()}
        self.mm = np.arange(self.g.M, dtype=float)

    @staticmethod
    def _widen(b, h):
        """A band of half width h' <= h padded to half width h."""
        hb = (b.shape[0] - 1) // 2
        if hb == h:
            return b
        out = np.zeros((2 * h + 1, b.shape[1]), b.dtype)
        out[h - hb:h + hb + 1] = b
        return out

    def _A(self):          # (M, 17, n_c): A^I_m for every m
        b = self.bands
        return b["A0"][None] + (self.mm ** 2)[:, None, None] * b["A2"][None]

    def _B(self):          # (M, 17, n_c): B^I_m for every m
        b, mm = self.bands, self.mm[:, None, None]
        w = lambda k: self._widen(b[k], 8)[None]
        return w("B0") + mm ** 2 * w("B2") + mm ** 4 * w("B4") + 1j * mm * (2.0 / self.ops.E) * b["C"][None]

    def _F(self):          # (M, 5, n_c)
        b = self.bands
        return b["F0"][None] + (self.mm ** 2)[:, None, None] * b["F2"][None]

    def mass(self, y):
        psi, th, u = y
        b = self.bands
        mp = band_apply(self._A(), psi)
        mp[0] = 0.0
        return mp, band_apply(b["D"], th), band_apply(b["D"], u)

    def imp(self, y):
        psi, th, u = y
        ops, b = self.ops, self.bands
        ip = band_apply(self._B(), psi)
        if self.buoy_implicit:
            ip = ip + (ops.Ra / ops.Pr) * (1j * self.mm[:, None] / ops.ann.s_o) * band_apply(b["C"], th)
        ip[0] = 0.0
        it = band_apply(self._F(), th) / ops.Pr
        return ip, it, band_apply(b["Ez"], u)

    def lu(self, gamma):
        if gamma not in self._lu:
            gdt = gamma * self.dt
            ops = self.ops
            Ab, Bb, Fb = self._A(), self._B(), self._F()
            lp = [None] + [BorderedBandSolver(ops.bc_psi, Ab[m] - gdt * Bb[m], 4) for m in range(1, self.g.M)]
            Db = self._widen(self.bands["D"], 4)
            lt = [BorderedBandSolver(ops.bc_dir, Db - gdt * self._widen(Fb[m], 4) / ops.Pr, 2)
                  for m in range(self.g.M)]
            lu_ = BorderedBandSolver(ops.bc_dir, Db - gdt * self._widen(self.bands["Ez"], 4), 2)
            self._lu[gamma] = (lp, lt, lu_)
        return self._lu[gamma]

    def solve(self, gamma, rhs):
        lp, lt, lu_ = self.lu(gamma)
        rp, rt, ru = (np.array(r) for r in rhs)
        rp[:, :4] = 0.0
        rt[:, :2] = 0.0
        ru[:2] = 0.0
        th = np.stack([lt[m].solve(rt[m]) for m in range(self.g.M)])
        if self.buoy_implicit:
            gdt = gamma * self.dt
            ops = self.ops
            rp = rp + gdt * (ops.Ra / ops.Pr) * (1j * self.mm[:, None] / ops.ann.s_o) * band_apply(self.bands["C"], th)
            rp[:, :4] = 0.0
        psi = np.zeros_like(rp)
        for m in range(1, self.g.M):
            psi[m] = lp[m].solve(rp[m])
        u = lu_.solve(ru)
        return psi, th, u
