"""Plain FP64 CPU oracle of one IMEX time step of the spherical quasi-geostrophic
convection model of Gastine (pizza, GJI 2019).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
anything in this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is written to be read against the paper, not to be fast:

* transforms are the defining sums (Eqs. fft/ifft of Section 3, Eqs. cheb/icheb of
  Section 3) evaluated as dense matrix products; ``numpy.fft`` is used only as a
  library primitive for the azimuthal sums and is pinned against the direct sum;
* radial derivatives use the dense Chebyshev differentiation matrix, not a
  recurrence;
* the Chebyshev-integration operators (Section 3.2, Eqs. psi_int, uphi_int,
  temp_int) are built by writing each term as a polynomial times a derivative and
  integrating by parts until no derivative remains, exactly as the paper states;
* the implicit systems are solved by dense LU (LAPACK through numpy/scipy); the
  bordered solve of Appendix A is provided separately and pinned against it;
* the time schemes follow Section 4 (Eqs. multistep1 and dirks) term by term.

Shares no code with the CUDA path.
"""
