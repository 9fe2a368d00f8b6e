"""Pins of the banded Appendix A path of the oracle (``oracle.banded``) against the
dense operators and the dense LU of ``oracle.stepper`` on small grids
(Section 3.2, Appendix A)."""
import numpy as np
import pytest

from oracle.banded import BandedIntegrationStepper, BorderedBandSolver, band_apply, diagonals
from oracle.operators import IntegrationOperators
from oracle.stepper import IntegrationStepper
from paper_1902_07092_gb300 import inputs

HALF = BandedIntegrationStepper.HALF
ROWS = BandedIntegrationStepper.ROWS


def test_bands_hold_the_dense_operators_exactly():
    """Every operator is exactly banded with the half bandwidth of Section 3.2
    (A^I, C^I 8; B^I parts 6; D^I, G^I 4; E^I, F^I 2): ``diagonals`` raises on any
    entry outside, and the diagonal-by-diagonal product equals the dense one."""
    n_r = 65
    nc = (2 * (n_r - 1)) // 3
    ops = IntegrationOperators(n_r, nc, 0.35, 1e-4, 1.0, 1e6)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, nc)) + 1j * rng.standard_normal((3, nc))
    for name, h in HALF.items():
        Mat = getattr(ops, name)
        b = diagonals(Mat, h, ROWS[name])
        want = (Mat @ x.T).T
        assert np.abs(band_apply(b, x) - want).max() <= 1e-14 * np.abs(want).max(), name
        with pytest.raises(ValueError):
            diagonals(Mat, h - 1, ROWS[name])          # the stated width is the smallest


@pytest.mark.parametrize("n_r", [17, 65, 129])
def test_bordered_band_solve_matches_dense_solve(n_r):
    """Appendix A with the banded LU of D against LAPACK's dense LU of the same
    row-scaled tau systems (Psi: p = 4, complex; theta and u_bar: p = 2, real
    operators), random right-hand sides: both backward stable, and equal to the
    accuracy the condition number allows."""
    nc = (2 * (n_r - 1)) // 3
    ops = IntegrationOperators(n_r, nc, 0.35, 1e-5, 1.0, 1e7)
    gdt = 0.5e-6
    rng = np.random.default_rng(n_r)
    cases = []
    for m in (1, 7, nc // 2):
        L = ops.lhs_psi(m, gdt)
        cases.append((L, ops.bc_psi, diagonals(ops.A(m) - gdt * ops.B(m), 8, 4), 4))
    Lt = ops.lhs_theta(5, gdt)
    cases.append((Lt, ops.bc_dir, diagonals(ops.D - gdt * ops.F(5), 4, 2), 2))
    Lu = ops.lhs_uphi(gdt)
    cases.append((Lu, ops.bc_dir, diagonals(ops.D - gdt * ops.Ez, 4, 2), 2))
    for L, tau, band, p in cases:
        b = rng.standard_normal(nc) + 1j * rng.standard_normal(nc)
        b[:p] = 0.0
        sol = BorderedBandSolver(tau, band, p)
        x = sol.solve(b)
        r = 1.0 / np.abs(L).max(axis=1)
        Ls = L * r[:, None]
        xd = np.linalg.solve(Ls, b * r)
        assert np.linalg.norm(Ls @ x - b * r) <= 1e-14 * np.linalg.norm(Ls, 2) * np.linalg.norm(x)
        kappa = np.linalg.cond(Ls)
        assert np.linalg.norm(x - xd) <= 8 * kappa * 2.0 ** -53 * np.linalg.norm(xd), kappa
        scale = np.abs(L) @ np.abs(x)                   # size of the summed terms, row by row
        assert np.all(np.abs(sol.matvec(x) - L @ x) <= 1e-14 * scale)


@pytest.mark.parametrize("n_r,scheme,buoy", [(33, "CNAB2", False), (33, "ARS443", True),
                                             (65, "SBDF3", False), (129, "ARS443", False)])
def test_banded_stepper_matches_dense_stepper(n_r, scheme, buoy):
    """Three steps of the banded oracle equal three steps of the dense oracle
    (same scheme, start-up and explicit terms; only the operator storage and the
    solve differ) to rounding in Psi and theta; the zonal flow, forced by the
    m = 0 mean of u_s omega that cancels to ~1e-4 of its terms, to rounding of
    those terms."""
    n_phi = 3 * (n_r - 1)
    th = inputs.theta_init(n_r, n_phi, 1.0, 4, cfg=2)
    z, zu = inputs.zero_state(n_r, n_phi)
    a = IntegrationStepper(n_r, n_phi, 1e-5, 1e7, 1.0, 0.35, scheme, 1e-7, buoy_implicit=buoy)
    b = BandedIntegrationStepper(n_r, n_phi, 1e-5, 1e7, 1.0, 0.35, scheme, 1e-7, buoy_implicit=buoy)
    a.set_state(z, th, zu)
    b.set_state(z, th, zu)
    for _ in range(3):
        a.step()
        b.step()
    for k, tol in ((0, 1e-13), (1, 1e-13)):
        assert np.linalg.norm(a.y[k] - b.y[k]) <= tol * np.linalg.norm(a.y[k])
    assert np.linalg.norm(a.y[2] - b.y[2]) <= 1e-9 * np.linalg.norm(a.y[2])
    whole = lambda y: np.concatenate([np.ravel(v) for v in y])
    assert np.linalg.norm(whole(a.y) - whole(b.y)) <= 1e-13 * np.linalg.norm(whole(a.y))
