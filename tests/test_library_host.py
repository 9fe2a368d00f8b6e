"""Host-side checks of the C library that need no GPU: it loads, exports every
symbol include/pizza.h declares, builds the same integration operators as the
oracle, and fails cleanly (status code, message) when no device is present."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.operators import IntegrationOperators

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pizza.h")).read()
    return sorted(set(re.findall(r"\b(pizza_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(libpizza):
    from paper_1902_07092_gb300 import binding
    decl = declared_symbols()
    assert set(decl) == set(binding.EXPORTS)
    for name in decl:
        assert hasattr(libpizza, name), name


@pytest.mark.parametrize("n_r", [33, 129])
def test_host_collocation_setup_equals_oracle(libpizza, n_r):
    """The library's grid-valued collocation inverses and differentiation matrices
    against the oracle's coefficient-space operators (T the synthesis matrix, an
    involution): D1 = T' T, D2 = T'' T, and G r = T x with x the oracle's refined
    solution of the same system for interior right-hand-side rows r."""
    import scipy.linalg as sl
    from paper_1902_07092_gb300 import binding
    from oracle.collocation import CollocationOperators
    E, Pr, m, gdt = 1e-4, 0.7, 5, 3e-5
    o = CollocationOperators(n_r, 0.35, E, Pr, 1.0)
    D1 = binding.pizza_host_collocation(3, n_r, 0.35)
    D2 = binding.pizza_host_collocation(4, n_r, 0.35)
    assert np.abs(D1 - o.T1 @ o.T).max() <= 1e-12 * np.abs(o.T1 @ o.T).max()
    assert np.abs(D2 - o.T2 @ o.T).max() <= 1e-11 * np.abs(o.T2 @ o.T).max()
    rng = np.random.default_rng(7)

    def refined(L, b):
        r = 1.0 / np.abs(L).max(axis=1)
        lu = sl.lu_factor(L * r[:, None])
        x = sl.lu_solve(lu, b * r)
        for _ in range(2):
            x = x + sl.lu_solve(lu, (b - L @ x) * r)
        return x

    N = n_r
    G = binding.pizza_host_collocation(0, n_r, 0.35, E, Pr, m, gdt)
    b = np.zeros(2 * N, complex)
    b[1:N - 1] = rng.standard_normal(N - 2) + 1j * rng.standard_normal(N - 2)
    x = refined(o.lhs_wpsi(m, gdt), b)
    ref = np.concatenate([o.T @ x[:N], o.T @ x[N:]])
    assert np.linalg.norm(G @ b[1:N - 1] - ref) <= 1e-12 * np.linalg.norm(ref)
    for which, Lin in ((1, o.Lt(m)), (2, o.Lu())):
        Gt = binding.pizza_host_collocation(which, n_r, 0.35, E, Pr, m, gdt)
        bt = np.zeros(N, complex)
        bt[1:N - 1] = rng.standard_normal(N - 2) + 1j * rng.standard_normal(N - 2)
        xt = refined(o.lhs_dir(Lin, gdt), bt)
        assert np.linalg.norm(Gt @ bt[1:N - 1] - o.T @ xt) <= 1e-13 * np.linalg.norm(o.T @ xt)


@pytest.mark.parametrize("n_r", [33, 65, 257])
def test_host_operators_equal_oracle(libpizza, n_r):
    from paper_1902_07092_gb300 import binding
    n_c = (2 * (n_r - 1)) // 3
    ops = IntegrationOperators(n_r, n_c, 0.35, 1e-3, 1.0, 1.0)
    names = ["A0", "A2", "B0", "B2", "B4", "C", "D", "F0", "F2", "Ez", "G"]
    for i, nm in enumerate(names):
        H = binding.pizza_host_operator(i, n_r, n_c, 0.35)
        O = getattr(ops, nm)
        assert np.abs(H - O).max() <= 1e-14 * np.abs(O).max() * 8, nm


def test_host_operator_rejects_bad_arguments(libpizza):
    from paper_1902_07092_gb300 import binding
    with pytest.raises(binding.PizzaError) as e:
        binding.pizza_host_operator(99, 33, 21, 0.35)
    assert e.value.code == -1


def test_init_validates_sizes(libpizza):
    from paper_1902_07092_gb300 import binding
    for args in [(32, 96), (33, 100), (33, 6), (4097, 96)]:
        with pytest.raises(binding.PizzaError) as e:
            binding.pizza_init(args[0], args[1], 1e-3, 1e5, 1.0, 0.35, 0)
        assert e.value.code == -1
    with pytest.raises(binding.PizzaError):
        binding.pizza_init(33, 96, -1.0, 1e5, 1.0, 0.35, 0)
    with pytest.raises(binding.PizzaError):
        binding.pizza_init(33, 96, 1e-3, 1e5, 1.0, 1.5, 0)
    with pytest.raises(binding.PizzaError):
        binding.pizza_init(33, 96, 1e-3, 1e5, 1.0, 0.35, 7)


def test_init_without_device_returns_status(libpizza):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_1902_07092_gb300 import binding
    with pytest.raises(binding.PizzaError) as e:
        binding.pizza_init(33, 96, 1e-3, 1e5, 1.0, 0.35, 0)
    assert e.value.code in (-2, -3)
    assert len(binding.pizza_last_error()) > 0
