"""Shared helpers of the GPU parity tests (no method arithmetic)."""
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")

# Ra_c fallback (Pr = 1, eta = 0.35) used only if the golden table is missing.
_RA_C_FALLBACK = {"0.001": 5.48836399e4, "1e-05": 9.95658291e6}


def critical_rayleigh(E):
    path = os.path.join(GOLDEN, "critical_rayleigh.json")
    key = "%g" % E
    if os.path.exists(path):
        t = json.load(open(path))
        if key in t:
            return t[key]["Ra_c"]
    return _RA_C_FALLBACK[key]


def critical_rayleigh_interp(E):
    """Ra_c from the golden table; between tabulated E, log-log interpolation
    (the batched runs draw E in [1e-6, 1e-4])."""
    import math
    t = json.load(open(os.path.join(GOLDEN, "critical_rayleigh.json")))
    key = "%g" % E
    if key in t:
        return t[key]["Ra_c"]
    pts = sorted((float(k), v["Ra_c"]) for k, v in t.items())
    for (e0, r0), (e1, r1) in zip(pts, pts[1:]):
        if e0 <= E <= e1:
            f = (math.log(E) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return math.exp(math.log(r0) + f * (math.log(r1) - math.log(r0)))
    raise KeyError("no critical Rayleigh number for E = %g" % E)


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def state_errors(gpu, ref):
    """Relative L2 of (Psi, theta, u_bar) and of the concatenated state."""
    out = {}
    for name, a, b in zip(("psi", "theta", "u"), gpu, ref):
        out[name] = rel_l2(a, b)
    ga = np.concatenate([np.asarray(x).ravel() for x in gpu])
    ra = np.concatenate([np.asarray(x).ravel() for x in ref])
    out["state"] = rel_l2(ga, ra)
    out["_norms"] = tuple(float(np.linalg.norm(x)) for x in ref)
    return out


# The zonal flow is forced only by the azimuthal mean of u_s omega,
# [v omega]_0 = sum_{m >= 1} 2 Re(v_m conj(omega_m)), a sum of terms of size
# |v_m||omega_m| that cancels to a small fraction 1/c_u of them (c_u ~ 1e2 .. 6e2
# at n_r = 33, ~4e3 on the n_r = 257 workload, ~2e3 at n_r = 2049).  Any error of
# the state (checked against its own bar) therefore reaches the forcing of
# u_bar amplified by c_u -- and by the derivatives in omega, which weight the
# high Chebyshev coefficients -- and u_bar, which integrates the forcing, cannot
# be more accurate than it.  So u_bar's own relative error is held to
#   max(U_FACTOR * tol, 4 * delta_F),
# delta_F the relative difference of the forcing evaluated (by the oracle's
# explicit stage) on the compared state and on the reference state: u_bar may
# carry the error its forcing explains, and no more.
U_FACTOR = 20.0


def zonal_forcing(oracle, y):
    """(h^2/s) [v omega]_0 on the radial grid for the state y = (Psi, theta, u_bar),
    and the size of its terms, (h^2/s) sum_m 2 |v_m||omega_m|."""
    from oracle.explicit import radial_fields
    v, _, omega, _ = radial_fields(oracle.g, *y)
    f = oracle.g.h2 / oracle.g.s
    mean = f * 2.0 * np.sum((v[:, 1:] * np.conj(omega[:, 1:])).real, axis=1)
    terms = f * 2.0 * np.sum(np.abs(v[:, 1:]) * np.abs(omega[:, 1:]), axis=1)
    return mean, terms


def zonal_cancellation(oracle):
    """c_u of the oracle's current state (integration and Galerkin steppers)."""
    mean, terms = zonal_forcing(oracle, oracle.y)
    nm = np.linalg.norm(mean)
    return float(np.linalg.norm(terms) / nm) if nm > 0 else 1.0


def assert_state_close(gpu, ref, tol, floor=1e-9, oracle=None):
    """Whole-state relative L2 <= tol; per field <= tol (u_bar: the forcing bar
    above, with ``oracle`` the reference stepper) for fields carrying more than
    ``floor`` of the state norm (a smaller field's error is bounded, relative to
    the state, by the whole-state check)."""
    e = state_errors(gpu, ref)
    total = np.sqrt(sum(n * n for n in e["_norms"]))
    assert e["state"] <= tol, e
    for name, n in zip(("psi", "theta", "u"), e["_norms"]):
        if n > floor * total:
            if name != "u":
                assert e[name] <= tol, (name, e)
            elif e["u"] > U_FACTOR * tol:
                assert oracle is not None, ("u", e)
                f_ref, _ = zonal_forcing(oracle, tuple(np.asarray(x) for x in ref))
                f_gpu, _ = zonal_forcing(oracle, tuple(np.asarray(x) for x in gpu))
                dF = rel_l2(f_gpu, f_ref)
                assert e["u"] <= max(U_FACTOR * tol, 4.0 * dF), ("u", dF, zonal_cancellation(oracle), e)
    return e

