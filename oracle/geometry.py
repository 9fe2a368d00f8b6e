"""Annulus geometry and conduction background of the QG model (Section 2).

Test infrastructure only (see the package docstring).

Definitions followed:
* gap d = s_o - s_i = 1, s_o = 1/(1-eta), s_i = eta/(1-eta)   (Section 2, units)
* h = (s_o^2 - s^2)^(1/2), beta = -s/h^2                       (Eq. cont)
* T_c = alpha ln[(1-eta) s]/ln eta, dT_c/ds = alpha/(s ln eta)
  alpha = eta/(1-eta) { arcsinh[(1-eta^2)^(1/2)/eta]/(1-eta^2)^(1/2) - 1 }
                                                              (Eq. temp and below)
* Gauss-Lobatto points x_k = cos(pi k/(N_r-1)), k = 0..N_r-1 (0-based), mapped
  affinely to s_k = (d/2) x_k + (s_o+s_i)/2                   (Section 3)
"""
import numpy as np


class Annulus:
    def __init__(self, eta):
        if not 0.0 < eta < 1.0:
            raise ValueError("radius ratio must lie in (0, 1)")
        self.eta = float(eta)
        self.s_o = 1.0 / (1.0 - eta)
        self.s_i = eta / (1.0 - eta)
        self.d = self.s_o - self.s_i
        self.a = self.d / 2.0            # ds/dx of the affine map
        self.b = (self.s_o + self.s_i) / 2.0

    def s_of_x(self, x):
        return self.a * np.asarray(x) + self.b

    def h2(self, s):
        return self.s_o ** 2 - np.asarray(s) ** 2

    def beta(self, s):
        s = np.asarray(s, dtype=float)
        return -s / self.h2(s)

    @property
    def alpha(self):
        eta = self.eta
        r = np.sqrt(1.0 - eta * eta)
        return eta / (1.0 - eta) * (np.arcsinh(r / eta) / r - 1.0)

    def Tc(self, s):
        return self.alpha * np.log((1.0 - self.eta) * np.asarray(s)) / np.log(self.eta)

    def dTc_ds(self, s):
        return self.alpha / (np.asarray(s) * np.log(self.eta))


def gauss_lobatto(n_r):
    k = np.arange(n_r)
    return np.cos(np.pi * k / (n_r - 1))
