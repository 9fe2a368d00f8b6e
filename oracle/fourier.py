"""Azimuthal Fourier transforms (Section 3, Eqs. fft and ifft).

Test infrastructure only (see the package docstring).

  grid:      f(phi_j) = 2 sum'_{m=0}^{N_m} Re{ f_m exp(i m phi_j) }   (m = 0 halved)
  spectral:  f_m = (1/N_phi) sum_j f(phi_j) exp(-i m phi_j),  m = 0..N_m
  phi_j = 2 pi j/N_phi, j = 0..N_phi-1; modes N_m < m are dropped / zero-padded.

``to_grid``/``to_spec`` use numpy's real FFT as the library primitive for these
sums; ``to_grid_direct``/``to_spec_direct`` evaluate the sums literally and pin it.
The azimuthal index is the LAST axis.
"""
import numpy as np


def to_grid(fm, n_phi):
    fm = np.asarray(fm)
    M = fm.shape[-1]
    pad = np.zeros(fm.shape[:-1] + (n_phi // 2 + 1,), dtype=complex)
    pad[..., :M] = fm
    return n_phi * np.fft.irfft(pad, n=n_phi, axis=-1)


def to_spec(f, n_m):
    f = np.asarray(f)
    n_phi = f.shape[-1]
    return np.fft.rfft(f, axis=-1)[..., :n_m + 1] / n_phi


def to_grid_direct(fm, n_phi):
    fm = np.asarray(fm)
    M = fm.shape[-1]
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    E = np.exp(1j * np.outer(np.arange(M), phi))        # (M, n_phi)
    w = np.full(M, 2.0)
    w[0] = 1.0
    return np.real(np.tensordot(fm * w, E, axes=(-1, 0)))


def to_spec_direct(f, n_m):
    f = np.asarray(f)
    n_phi = f.shape[-1]
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    E = np.exp(-1j * np.outer(phi, np.arange(n_m + 1)))   # (n_phi, M)
    return np.tensordot(f, E, axes=(-1, 0)) / n_phi
