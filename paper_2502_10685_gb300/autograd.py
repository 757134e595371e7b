"""torch.autograd.Function over the library's expectation and adjoint gradient.

Forward:  <0^n| U(theta)^dagger O U(theta) |0^n>  (stab_set_params from the
          device tensor, then stab_expect_async).
Backward: all d<O>/d theta_j from one adjoint reverse sweep (stab_grad_async),
          scaled by the incoming gradient.
Angles and results stay on the device; nothing is computed in Python.
"""
from __future__ import annotations

import torch

from .stab import Stab


class PauliExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, thetas: torch.Tensor, stab: Stab) -> torch.Tensor:
        if thetas.dtype != torch.float64 or not thetas.is_cuda:
            raise TypeError("thetas must be a CUDA float64 tensor")
        th = thetas.detach().contiguous()
        stab.set_params(th)
        out = torch.empty(1, dtype=torch.float64, device=thetas.device)
        stab.expect_async(out)
        ctx.stab = stab
        ctx.save_for_backward(th)
        return out[0]

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (th,) = ctx.saved_tensors
        stab: Stab = ctx.stab
        stab.set_params(th)          # another forward may have changed the angles
        grads = torch.empty(max(stab.n_params, 1), dtype=torch.float64, device=th.device)
        e = torch.empty(1, dtype=torch.float64, device=th.device)
        stab.grad_async(e, grads)
        return grads[: stab.n_params] * grad_out, None


class ExpectationLayer(torch.nn.Module):
    """A fixed circuit and observable with trainable angles."""

    def __init__(self, circuit, observable, device: int = 0, thetas=None):
        super().__init__()
        self.stab = Stab(circuit.n, device=device)
        self.stab.load_circuit(circuit.gates, circuit.thetas)
        self.stab.set_observable(observable)
        init = circuit.thetas if thetas is None else thetas
        self.thetas = torch.nn.Parameter(
            torch.tensor(init, dtype=torch.float64, device=torch.device("cuda", device)))

    def forward(self) -> torch.Tensor:
        return PauliExpectation.apply(self.thetas, self.stab)
