"""torch.autograd.Function for the time-averaged Nusselt number of a CNAB2 run,
J = (1/K) sum_{n=1..K} (Nu_n - 1), as a function of the initial temperature
coefficients and of Ra, J summed on the device by the library (one read at the
end); the backward pass is the library's discrete adjoint
(pizza_tape_begin / pizza_adjoint_step), with checkpoints every
``checkpoint_every`` steps.  Argument marshalling only: the forward steps and the
adjoint run in the CUDA library.

Complex gradients follow PyTorch's convention for a real loss, dJ/dRe + i dJ/dIm,
which is the adjoint in the inner product Re sum conj(a) b used by the library.
"""
import numpy as np
import torch

from .binding import Solver


class NusseltAverage(torch.autograd.Function):
    """J = NusseltAverage.apply(theta0, Ra, cfg) with theta0 a complex128 tensor
    [N_m+1][N_c] (the initial temperature coefficients; Psi = u_bar = 0), Ra a
    0-d float64 tensor and cfg a dict with n_r, n_phi, E, Pr, radius_ratio, dt,
    steps and (optionally) checkpoint_every."""

    @staticmethod
    def forward(ctx, theta0, Ra, cfg):
        s = Solver(cfg["n_r"], cfg["n_phi"], cfg["E"], float(Ra), cfg["Pr"], cfg["radius_ratio"], "CNAB2",
                   cfg["dt"])
        th = theta0.detach().cpu().numpy().astype(np.complex128)
        z = np.zeros_like(th)
        s.set_state(th, z, np.zeros(th.shape[1]))
        s.tape_begin(int(cfg.get("checkpoint_every", 20)))
        w = s.nusselt_weights()
        K = int(cfg["steps"])
        s.nusselt_begin()          # Nu_n - 1 summed on the device after every step
        s.step(K)
        total, n = s.nusselt_end()
        if n != K:
            raise RuntimeError("the Nusselt sum covers %d of %d steps" % (n, K))
        ctx.solver, ctx.K, ctx.w = s, K, w
        return torch.tensor(total / K, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_J):
        s, K = ctx.solver, ctx.K
        gJ = float(grad_J)
        g = np.zeros((s.M, s.n_c), np.complex128)
        g[0] = ctx.w * (gJ / K)
        dRa = 0.0
        for k in range(K):
            dRa = s.adjoint_step(g_theta=g)
        _, th_bar, _ = s.get_adjoint()
        s.close()
        return torch.from_numpy(th_bar), torch.tensor(dRa * gJ, dtype=torch.float64), None
