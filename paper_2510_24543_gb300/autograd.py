"""torch.autograd binding of the energy functional (Eq. 1).

`EnergyModel` holds a handle for one grid and precision; `energy(psi, theta)`
returns E[psi; theta] as a differentiable 0-dim tensor.  theta is a float64
tensor of the parameters in `egpe.PARAM_NAMES` order (g11, g12, g22, gdd11,
gdd12, gdd22, kappa, eta_s, trap_x, trap_y, trap_z).

Forward runs `egpe_energy_grad` (which yields H_i psi_i) and `egpe_param_grad`;
backward is the hand-written adjoint:

* psi: for a real loss PyTorch stores the conjugate Wirtinger gradient times
  two, dL/dRe psi + i dL/dIm psi.  E is a sum over grid points weighted by dV
  and dE/dpsi*(x) = dV (H psi)(x), so the gradient is 2 dV H psi.
* theta: the partial derivatives of E at fixed psi.  At a normalised ground
  state psi*(theta) they are also the derivatives of the ground-state energy
  (Hellmann-Feynman), so `ground_state_energy` returns dE0/dtheta without
  differentiating through the solver.

Every step runs in the library's kernels; this module only marshals arguments.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import egpe as E


def params_vector(g, gdd, kappa, eta_s, trap) -> torch.Tensor:
    """theta in PARAM_NAMES order from symmetric couplings and the trap."""
    return torch.tensor([g[0][0], g[0][1], g[1][1], gdd[0][0], gdd[0][1], gdd[1][1], kappa, eta_s,
                         trap[0], trap[1], trap[2]], dtype=torch.float64)


class EnergyModel:
    """One grid, one precision, parameters settable from a theta vector."""

    def __init__(self, n: Sequence[int], L: Sequence[float], theta: torch.Tensor, nodes: int = 32,
                 prec: int = E.EGPE_FP64, stream: Optional[int] = None):
        E.load()
        self.n, self.L, self.nodes, self.prec = tuple(n), tuple(L), int(nodes), prec
        self.dV = (2.0 * L[0] / n[0]) * (2.0 * L[1] / n[1]) * (2.0 * L[2] / n[2])
        self.h = E.egpe_create([E.make_grid(n, L)], [self._params(theta)], prec, stream or 0)
        self._theta = theta.detach().to("cpu", torch.float64).clone()

    def _params(self, theta: torch.Tensor):
        t = [float(x) for x in theta.detach().to("cpu", torch.float64)]
        g = ((t[0], t[1]), (t[1], t[2]))
        gdd = ((t[3], t[4]), (t[4], t[5]))
        return E.make_params(g, gdd, t[6], t[7], self.nodes, (t[8], t[9], t[10]))

    def set_theta(self, theta: torch.Tensor) -> None:
        th = theta.detach().to("cpu", torch.float64)
        if not torch.equal(th, self._theta):
            E.egpe_set_params(self.h, 0, self._params(th))
            self._theta = th.clone()

    def close(self) -> None:
        if getattr(self, "h", None):
            E.egpe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, psi: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
        return EnergyFn.apply(psi, theta, self)

    def ground_state_energy(self, psi0: torch.Tensor, theta: torch.Tensor, opts=None) -> torch.Tensor:
        """E0(theta): solves for the ground state from psi0 (not modified) and
        returns its energy, differentiable in theta by Hellmann-Feynman."""
        return GroundStateEnergyFn.apply(psi0, theta, self, opts)


def _dtheta(model: EnergyModel, psi: torch.Tensor, device) -> torch.Tensor:
    d = E.egpe_param_grad(model.h, 0, psi)
    return torch.tensor([d[k] for k in E.PARAM_NAMES], dtype=torch.float64, device=device)


class EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi: torch.Tensor, theta: torch.Tensor, model: EnergyModel):
        model.set_theta(theta)
        psi_c = psi.detach().contiguous()
        hpsi = torch.empty_like(psi_c)
        Ev, _ = E.egpe_energy_grad(model.h, 0, psi_c, hpsi)
        ctx.save_for_backward(hpsi, _dtheta(model, psi_c, theta.device))
        ctx.dV = model.dV
        return torch.tensor(Ev, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        hpsi, dtheta = ctx.saved_tensors
        g_psi = g_theta = None
        if ctx.needs_input_grad[0]:
            g_psi = (2.0 * ctx.dV) * gE.to(hpsi.real.dtype) * hpsi
        if ctx.needs_input_grad[1]:
            g_theta = gE.to(torch.float64).to(dtheta.device) * dtheta
        return g_psi, g_theta, None


class GroundStateEnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0: torch.Tensor, theta: torch.Tensor, model: EnergyModel, opts):
        model.set_theta(theta)
        o = opts if opts is not None else E.egpe_default_solve_opts()
        x = psi0.detach().clone().contiguous()
        st, reps, _ = E.egpe_ncg_solve(model.h, [x], o, 1)
        if reps[0]["status"] != 0:
            raise RuntimeError(f"ground state not converged: {reps[0]}")
        ctx.save_for_backward(_dtheta(model, x, theta.device))
        return torch.tensor(reps[0]["E"], dtype=torch.float64, device=psi0.device)

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        (dtheta,) = ctx.saved_tensors
        g_theta = gE.to(torch.float64).to(dtheta.device) * dtheta if ctx.needs_input_grad[1] else None
        return None, g_theta, None, None
