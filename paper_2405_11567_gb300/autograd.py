"""Energy with its exact adjoint gradient as a ``torch.autograd.Function``.

forward(theta) calls ``sv_energy_grad`` once: the library runs the forward sweep,
lambda = (H - c) psi and the reverse (adjoint) sweep on the GPU and returns E and
dE/dtheta in float64; backward scales the stored gradient by the incoming dE.
The angles live on the host (float64), like the C-ABI's.
"""
import numpy as np
import torch

from .sv import Hamiltonian, StateVector


class EnergyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, state: StateVector, ham: Hamiltonian, ops):
        th = theta.detach().to("cpu", torch.float64).numpy()
        E, g = state.energy_grad(ham, ops, th)
        ctx.save_for_backward(torch.from_numpy(np.array(g, dtype=np.float64)))
        return torch.tensor(E, dtype=torch.float64)

    @staticmethod
    def backward(ctx, dE):
        (g,) = ctx.saved_tensors
        return dE.to(torch.float64) * g, None, None, None


def energy(theta: torch.Tensor, state: StateVector, ham: Hamiltonian, ops) -> torch.Tensor:
    """E(theta) for the ansatz ``ops`` applied to the reference recorded on ``state``."""
    return EnergyFunction.apply(theta, state, ham, ops)
