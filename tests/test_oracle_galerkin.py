"""The oracle's Galerkin-basis solve (Appendix B) against what fixes it independently:
numpy's Chebyshev routines for the boundary values of the basis functions, the
half bandwidths the paper states for the streamfunction system, and the tau
solve of the same discrete problem (the stencil columns span exactly the
coefficient vectors meeting the boundary conditions, so both give one solution)."""
import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import chebyshev as ch
from oracle.galerkin import (GalerkinStepper, band_extent, galerkin_matrix, stencil_dir, stencil_psi)
from oracle.stepper import IntegrationStepper

pytestmark = pytest.mark.filterwarnings("ignore::scipy.linalg.LinAlgWarning")


def test_streamfunction_basis_meets_the_four_boundary_conditions():
    """phi_n(1) = phi_n(-1) = phi_n'(-1) = phi_n'''(1) = 0 for every column of S_Psi,
    evaluated with numpy's chebval/chebder (x = 1 is s_o, x = -1 is s_i)."""
    S = stencil_psi(40)
    for n in range(S.shape[1]):
        c = S[:, n]
        scale = np.abs(c).sum() * (n + 5) ** 6
        assert abs(npc.chebval(1.0, c)) <= 1e-13 * scale
        assert abs(npc.chebval(-1.0, c)) <= 1e-13 * scale
        assert abs(npc.chebval(-1.0, npc.chebder(c))) <= 1e-13 * scale
        assert abs(npc.chebval(1.0, npc.chebder(c, 3))) <= 1e-13 * scale


def test_dirichlet_basis_vanishes_at_both_walls():
    S = stencil_dir(30)
    for n in range(S.shape[1]):
        assert abs(npc.chebval(1.0, S[:, n])) < 1e-14
        assert abs(npc.chebval(-1.0, S[:, n])) < 1e-14


def test_stencils_span_the_null_space_of_the_tau_rows():
    """Full column rank and annihilated by the tau rows (in f_hat coefficients):
    the columns are a basis of the boundary-satisfying coefficient vectors."""
    st = IntegrationStepper(33, 48, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    ops, nc = st.ops, st.n_c
    hs = ch.hat_scale(33, nc)
    for S, bc, p in ((stencil_psi(nc), ops.bc_psi, 4), (stencil_dir(nc), ops.bc_dir, 2)):
        Sh = S / hs[:, None]
        assert np.linalg.matrix_rank(Sh) == nc - p
        assert np.abs(bc @ Sh).max() <= 1e-12 * np.abs(bc).max() * np.abs(Sh).max() * nc


def test_galerkin_systems_have_the_stated_bandwidths():
    """P_4 (A - g dt B) S_Psi: 8 diagonals below and 12 above (Appendix B); the
    Dirichlet systems 4 below and 6 above; the extreme diagonals are populated."""
    st = GalerkinStepper(65, 96, 1e-3, 1e5, 1.0, 0.35, "CNAB2", 1e-4)
    ops, gdt = st.ops, 0.5e-4
    for m in (1, 7):
        Gp = galerkin_matrix(ops.A(m) - gdt * ops.B(m), 4, st.S_psi, 65)
        assert band_extent(Gp) == (8, 12)
        Gt = galerkin_matrix(ops.D - gdt * ops.F(m) / ops.Pr, 2, st.S_dir, 65)
        assert band_extent(Gt) == (4, 6)
    Gu = galerkin_matrix(ops.D - gdt * ops.Ez, 2, st.S_dir, 65)
    assert band_extent(Gu) == (4, 6)


@pytest.mark.parametrize("n_r", [33, 65])
def test_galerkin_solve_equals_tau_solve(n_r):
    args = (n_r, 3 * (n_r - 1) // 2, 1e-3, 3e5, 0.7, 0.35, "CNAB2", 1e-4)
    gal, tau = GalerkinStepper(*args), IntegrationStepper(*args)
    rng = np.random.default_rng(n_r)
    M, nc = gal.g.M, gal.n_c
    c = lambda: rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))
    rhs = (c(), c(), rng.standard_normal(nc))
    for gamma in (0.5, 0.25):
        a, b = gal.solve(gamma, rhs), tau.solve(gamma, rhs)
        for x, y in zip(a, b):
            assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


@pytest.mark.parametrize("scheme,buoy", [("CNAB2", False), ("ARS443", False), ("SBDF3", True)])
def test_galerkin_steps_equal_tau_steps(scheme, buoy):
    args = (33, 48, 1e-3, 2e5, 1.0, 0.35, scheme, 2e-4)
    gal = GalerkinStepper(*args, buoy_implicit=buoy)
    tau = IntegrationStepper(*args, buoy_implicit=buoy)
    rng = np.random.default_rng(4)
    M, nc = gal.g.M, gal.n_c
    c = lambda: 0.3 * (rng.standard_normal((M, nc)) + 1j * rng.standard_normal((M, nc))) / (1 + np.arange(nc)) ** 2
    psi, th = c(), c()
    th[0] = th[0].real
    u = 0.3 * rng.standard_normal(nc) / (1 + np.arange(nc)) ** 2
    # start from a state meeting the boundary conditions (one tau step)
    tau.set_state(psi, th, u)
    tau.step()
    y0 = tau.y
    gal.set_state(*y0)
    tau.set_state(*y0)
    for _ in range(5):
        gal.step()
        tau.step()
    for x, y in zip(gal.y, tau.y):
        assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)
