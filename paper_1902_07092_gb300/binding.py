"""ctypes binding of libpizza (include/pizza.h).  Argument marshalling only:
every step of the time step runs in the CUDA library.  Functions carry the C
names; arrays may be numpy arrays (host) or torch CUDA tensors (device).

Loading fails loudly if the library is missing; there is no fallback path.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpizza.so")

PIZZA_CNAB2, PIZZA_SBDF2, PIZZA_SBDF3, PIZZA_ARS443, PIZZA_BPR353 = 0, 1, 2, 3, 4
SCHEMES = {"CNAB2": 0, "SBDF2": 1, "SBDF3": 2, "ARS443": 3, "BPR353": 4}

STATUS = {0: "PIZZA_OK", -1: "PIZZA_EINVAL", -2: "PIZZA_ENOMEM", -3: "PIZZA_ECUDA", -4: "PIZZA_ENONFINITE",
          -5: "PIZZA_ECFL", -6: "PIZZA_ETIMEOUT", -7: "PIZZA_ESTATE", -8: "PIZZA_EUNSUPPORTED"}

# every symbol include/pizza.h declares
EXPORTS = ("pizza_init", "pizza_set_option", "pizza_set_stream", "pizza_get_sizes", "pizza_set_state",
           "pizza_get_state", "pizza_step", "pizza_explicit_terms", "pizza_diagnostics", "pizza_get_grid",
           "pizza_profile_begin", "pizza_profile_end", "pizza_synchronize",
           "pizza_host_operator", "pizza_host_collocation", "pizza_explicit_terms_noalloc", "pizza_free",
           "pizza_last_error", "pizza_tape_begin", "pizza_adjoint_step", "pizza_get_adjoint",
           "pizza_explicit_adjoint", "pizza_nusselt_weights", "pizza_autotune", "pizza_batch_create",
           "pizza_batch_step", "pizza_batch_stream", "pizza_batch_free", "pizza_fp64_fma_rate",
           "pizza_set_slab", "pizza_nusselt_begin", "pizza_nusselt_end")

_lib = None


class PizzaDiag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("E_K", "E_Z", "enstrophy", "Nu", "Re", "Ro", "cfl_s", "cfl_phi")]


class PizzaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpizza.so is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, d, i = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int
    lib.pizza_init.argtypes = [ctypes.POINTER(vp), i, i, d, d, d, d, i]
    lib.pizza_set_option.argtypes = [vp, ctypes.c_char_p, d]
    lib.pizza_set_stream.argtypes = [vp, vp]
    lib.pizza_get_sizes.argtypes = [vp, ip, ip, ip, ip]
    lib.pizza_set_state.argtypes = [vp, dp, dp, dp, i]
    lib.pizza_get_state.argtypes = [vp, dp, dp, dp]
    lib.pizza_step.argtypes = [vp, i]
    lib.pizza_explicit_terms.argtypes = [vp, dp, dp, dp]
    lib.pizza_diagnostics.argtypes = [vp, ctypes.POINTER(PizzaDiag)]
    lib.pizza_get_grid.argtypes = [vp, dp, dp, dp, dp]
    lib.pizza_profile_begin.argtypes = [vp, ctypes.c_uint]
    lib.pizza_profile_end.argtypes = [vp, dp, dp]
    lib.pizza_synchronize.argtypes = [vp]
    lib.pizza_host_operator.argtypes = [i, i, i, d, dp]
    lib.pizza_host_collocation.argtypes = [i, i, d, d, d, i, d, dp]
    lib.pizza_tape_begin.argtypes = [vp, i]
    lib.pizza_adjoint_step.argtypes = [vp, dp, dp, dp, ctypes.POINTER(d)]
    lib.pizza_get_adjoint.argtypes = [vp, dp, dp, dp]
    lib.pizza_explicit_adjoint.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.pizza_nusselt_weights.argtypes = [vp, dp]
    lib.pizza_autotune.argtypes = [vp, ip, ip]
    lib.pizza_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i]
    lib.pizza_batch_step.argtypes = [vp, i]
    lib.pizza_batch_stream.argtypes = [vp]
    lib.pizza_batch_stream.restype = vp
    lib.pizza_batch_free.argtypes = [vp]
    lib.pizza_batch_free.restype = None
    lib.pizza_explicit_terms_noalloc.argtypes = [i, i, d, d, d, dp, dp, dp, dp, dp, dp, vp]
    lib.pizza_fp64_fma_rate.argtypes = [i, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.pizza_set_slab.argtypes = [vp, i, i, i, i, vp, vp, vp, vp]
    lib.pizza_nusselt_begin.argtypes = [vp]
    lib.pizza_nusselt_end.argtypes = [vp, ctypes.POINTER(d), ip]
    lib.pizza_free.argtypes = [vp]
    lib.pizza_free.restype = None
    lib.pizza_last_error.argtypes = [vp]
    lib.pizza_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("pizza_free", "pizza_last_error", "pizza_batch_free", "pizza_batch_stream"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


def _check(rc, ctx=None):
    if rc != 0:
        raise PizzaError(rc, load().pizza_last_error(ctx).decode())
    return rc


def pizza_init(n_r, n_phi, E, Ra, Pr, radius_ratio, scheme):
    lib = load()
    h = ctypes.c_void_p()
    if isinstance(scheme, str):
        scheme = SCHEMES[scheme]
    _check(lib.pizza_init(ctypes.byref(h), n_r, n_phi, E, Ra, Pr, radius_ratio, scheme))
    return h


def pizza_set_option(ctx, key, value):
    return _check(load().pizza_set_option(ctx, key.encode(), float(value)), ctx)


def pizza_set_stream(ctx, stream):
    return _check(load().pizza_set_stream(ctx, stream), ctx)


def pizza_get_sizes(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().pizza_get_sizes(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def pizza_set_state(ctx, theta_hat, psi_hat, uphi0_hat, nc_in):
    return _check(load().pizza_set_state(ctx, _ptr(theta_hat), _ptr(psi_hat), _ptr(uphi0_hat), nc_in), ctx)


def pizza_get_state(ctx, theta_hat, psi_hat, uphi0_hat):
    return _check(load().pizza_get_state(ctx, _ptr(theta_hat), _ptr(psi_hat), _ptr(uphi0_hat)), ctx)


def pizza_step(ctx, nsteps):
    return _check(load().pizza_step(ctx, nsteps), ctx)


def pizza_explicit_terms(ctx, e_psi, e_theta, e_uphi):
    return _check(load().pizza_explicit_terms(ctx, _ptr(e_psi), _ptr(e_theta), _ptr(e_uphi)), ctx)


def pizza_diagnostics(ctx):
    d = PizzaDiag()
    _check(load().pizza_diagnostics(ctx, ctypes.byref(d)), ctx)
    return {n: getattr(d, n) for n, _ in PizzaDiag._fields_}


def pizza_get_grid(ctx, us, uphi, omega, theta):
    return _check(load().pizza_get_grid(ctx, _ptr(us), _ptr(uphi), _ptr(omega), _ptr(theta)), ctx)


KERNELS = ("spec_to_grid", "phi_products", "grid_to_spec", "solve")


def pizza_profile_begin(ctx, mask=0xF):
    return _check(load().pizza_profile_begin(ctx, mask), ctx)


def pizza_profile_end(ctx):
    t = np.zeros(4)
    n = np.zeros(4, np.int32)
    _check(load().pizza_profile_end(ctx, _ptr(t), _ptr(n)), ctx)
    return t, n


def pizza_synchronize(ctx):
    return _check(load().pizza_synchronize(ctx), ctx)


def pizza_host_operator(which, n_r, n_c, radius_ratio):
    out = np.zeros((n_c, n_c))
    _check(load().pizza_host_operator(which, n_r, n_c, radius_ratio, _ptr(out)))
    return out


def pizza_tape_begin(ctx, checkpoint_every=20):
    return _check(load().pizza_tape_begin(ctx, checkpoint_every), ctx)


def pizza_adjoint_step(ctx, g_theta=None, g_psi=None, g_u=None, want_dRa=True):
    """Reverse one recorded step; returns the running dJ/dRa (None, without
    waiting for the GPU, when want_dRa is false)."""
    if not want_dRa:
        _check(load().pizza_adjoint_step(ctx, _ptr(g_theta), _ptr(g_psi), _ptr(g_u), None), ctx)
        return None
    r = ctypes.c_double(0.0)
    _check(load().pizza_adjoint_step(ctx, _ptr(g_theta), _ptr(g_psi), _ptr(g_u), ctypes.byref(r)), ctx)
    return r.value


def pizza_get_adjoint(ctx, theta_bar, psi_bar, uphi0_bar):
    return _check(load().pizza_get_adjoint(ctx, _ptr(theta_bar), _ptr(psi_bar), _ptr(uphi0_bar)), ctx)


def pizza_explicit_adjoint(ctx, e_psi_bar, e_theta_bar, e_u_bar, psi_bar, theta_bar, uphi0_bar):
    return _check(load().pizza_explicit_adjoint(ctx, _ptr(e_psi_bar), _ptr(e_theta_bar), _ptr(e_u_bar),
                                                _ptr(psi_bar), _ptr(theta_bar), _ptr(uphi0_bar)), ctx)


def pizza_nusselt_weights(ctx, n_c):
    w = np.zeros(n_c)
    _check(load().pizza_nusselt_weights(ctx, _ptr(w)), ctx)
    return w


def pizza_autotune(ctx):
    nb, th = ctypes.c_int(), ctypes.c_int()
    _check(load().pizza_autotune(ctx, ctypes.byref(nb), ctypes.byref(th)), ctx)
    return nb.value, th.value


class Batch:
    """Several contexts advanced together by one CUDA graph (pizza_batch_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        h = ctypes.c_void_p()
        _check(load().pizza_batch_create(ctypes.byref(h), arr, len(self.solvers)))
        self.h = h

    def step(self, nsteps):
        _check(load().pizza_batch_step(self.h, nsteps))

    @property
    def stream(self):
        return load().pizza_batch_stream(self.h)

    def close(self):
        if self.h is not None:
            load().pizza_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pizza_host_collocation(which, n_r, radius_ratio, E=1.0, Pr=1.0, m=1, gdt=0.0):
    shape = {0: (2 * n_r, n_r - 2), 1: (n_r, n_r - 2), 2: (n_r, n_r - 2), 3: (n_r, n_r), 4: (n_r, n_r)}[which]
    out = np.zeros(shape, np.complex128 if which == 0 else np.float64)
    _check(load().pizza_host_collocation(which, n_r, radius_ratio, E, Pr, m, gdt, _ptr(out)))
    return out


def pizza_explicit_terms_noalloc(n_r, n_phi, Ra, Pr, radius_ratio, psi_hat, theta_hat, uphi0_hat,
                                 e_psi, e_theta, e_uphi, stream=None):
    """Device arrays only (e.g. torch CUDA tensors); queued on ``stream``."""
    return _check(load().pizza_explicit_terms_noalloc(n_r, n_phi, Ra, Pr, radius_ratio, _ptr(psi_hat),
                                                      _ptr(theta_hat), _ptr(uphi0_hat), _ptr(e_psi),
                                                      _ptr(e_theta), _ptr(e_uphi), stream))


def pizza_set_slab(ctx, m_lo, m_hi, k_lo, k_hi, grid1, grid2, exchange, user=None):
    """exchange: a ctypes callback of slabs.EXCHANGE_FN (or None with the full
    ranges, which returns the context to the whole step)."""
    fn = ctypes.cast(exchange, ctypes.c_void_p) if exchange is not None else None
    return _check(load().pizza_set_slab(ctx, m_lo, m_hi, k_lo, k_hi, _ptr(grid1), _ptr(grid2), fn, user), ctx)


def pizza_fp64_fma_rate(iters=20000):
    """Measured FP64 FMA rate of the current device: (TFLOP/s, ms of the launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().pizza_fp64_fma_rate(iters, ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def pizza_free(ctx):
    load().pizza_free(ctx)


def pizza_last_error(ctx=None):
    return load().pizza_last_error(ctx).decode()


class Solver:
    """Convenience owner of one context with numpy host arrays in the C layouts
    (complex128 [N_m+1][N_c] for theta and Psi, float64 [N_c] for u_bar).
    ``radial`` selects the formulation: "integration" (Section 3.2, default; tau
    rows), "galerkin" (the same unknowns solved in the Galerkin bases of Appendix
    B) or "collocation" (Section 3.1; psi instead of Psi, N_c = n_r).  ``pumping_eps``
    turns Ekman pumping on: the approximate F_eps of Eq. approx_pump with that eps
    (integration) or the exact term, implicit (collocation)."""

    def __init__(self, n_r, n_phi, E, Ra, Pr, radius_ratio, scheme, dt=None, radial="integration",
                 pumping_eps=None, buoy_implicit=False):
        self.ctx = pizza_init(n_r, n_phi, E, Ra, Pr, radius_ratio, scheme)
        if radial not in ("integration", "collocation", "galerkin"):
            raise ValueError(radial)
        if radial != "integration":
            pizza_set_option(self.ctx, "radial", 0 if radial == "collocation" else 2)
        if pumping_eps is not None:
            pizza_set_option(self.ctx, "pumping_eps", pumping_eps)
        if buoy_implicit:
            pizza_set_option(self.ctx, "buoy_implicit", 1)
        self.n_r, self.n_phi, self.n_m, self.n_c = pizza_get_sizes(self.ctx)
        self.M = self.n_m + 1
        if dt is not None:
            pizza_set_option(self.ctx, "dt", dt)

    def set_state(self, theta_hat, psi_hat=None, uphi0_hat=None):
        th = np.ascontiguousarray(theta_hat, dtype=np.complex128)
        nc_in = th.shape[1]
        ps = None if psi_hat is None else np.ascontiguousarray(psi_hat, dtype=np.complex128)
        up = None if uphi0_hat is None else np.ascontiguousarray(uphi0_hat, dtype=np.float64)
        pizza_set_state(self.ctx, th, ps, up, nc_in)

    def get_state(self):
        th = np.zeros((self.M, self.n_c), np.complex128)
        ps = np.zeros((self.M, self.n_c), np.complex128)
        up = np.zeros(self.n_c)
        pizza_get_state(self.ctx, th, ps, up)
        return ps, th, up

    def step(self, n=1):
        pizza_step(self.ctx, n)

    def explicit_terms(self):
        ep = np.zeros((self.M, self.n_c), np.complex128)
        et = np.zeros((self.M, self.n_c), np.complex128)
        eu = np.zeros(self.n_c)
        pizza_explicit_terms(self.ctx, ep, et, eu)
        return ep, et, eu

    def diagnostics(self):
        return pizza_diagnostics(self.ctx)

    def nusselt_begin(self):
        _check(load().pizza_nusselt_begin(self.ctx), self.ctx)

    def nusselt_end(self):
        """(sum of Nu_n - 1 over the steps since nusselt_begin, number of steps)"""
        v, n = ctypes.c_double(), ctypes.c_int()
        _check(load().pizza_nusselt_end(self.ctx, ctypes.byref(v), ctypes.byref(n)), self.ctx)
        return v.value, n.value

    def tape_begin(self, checkpoint_every=20):
        pizza_tape_begin(self.ctx, checkpoint_every)

    def adjoint_step(self, g_theta=None, g_psi=None, g_u=None, want_dRa=True):
        """g_*: numpy arrays or contiguous tensors (host or device) of the step's
        objective gradient; returns the running dJ/dRa, or None when want_dRa is
        false (the step is then only enqueued)."""
        def c(a, dt):
            if a is None or isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
                return None if a is None else np.ascontiguousarray(a, dtype=dt)
            if str(a.dtype) != "torch." + np.dtype(dt).name:
                raise TypeError("expected a %s tensor" % np.dtype(dt).name)
            return a
        return pizza_adjoint_step(self.ctx, c(g_theta, np.complex128), c(g_psi, np.complex128), c(g_u, np.float64),
                                  want_dRa)

    def get_adjoint(self):
        th = np.zeros((self.M, self.n_c), np.complex128)
        ps = np.zeros((self.M, self.n_c), np.complex128)
        up = np.zeros(self.n_c)
        pizza_get_adjoint(self.ctx, th, ps, up)
        return ps, th, up

    def explicit_adjoint(self, e_psi_bar, e_theta_bar, e_u_bar):
        c = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        ps = np.zeros((self.M, self.n_c), np.complex128)
        th = np.zeros((self.M, self.n_c), np.complex128)
        up = np.zeros(self.n_c)
        pizza_explicit_adjoint(self.ctx, c(e_psi_bar, np.complex128), c(e_theta_bar, np.complex128),
                               c(e_u_bar, np.float64), ps, th, up)
        return ps, th, up

    def autotune(self):
        return pizza_autotune(self.ctx)

    def nusselt_weights(self):
        return pizza_nusselt_weights(self.ctx, self.n_c)

    def get_grid(self):
        """(u_s, u_phi, omega, theta) on the physical grid, each [n_r][n_phi]."""
        out = [np.zeros((self.n_r, self.n_phi)) for _ in range(4)]
        pizza_get_grid(self.ctx, *out)
        return tuple(out)

    def close(self):
        if self.ctx is not None:
            pizza_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
