"""The potential U(X, Y) of Eq. Lang as a differentiable PyTorch function.

``PotentialEnergy.apply(pos, evaluator)`` returns the total potential energy
(Lennard-Jones + reaction field + bonds + angles, FP64 totals of the CUDA
kernels) of one configuration; its backward is the force kernel's output,
dU/dX = -F, times the incoming gradient.  PyTorch supplies the autograd
plumbing only: the energy and the forces come from the C ABI
(``sim_set_state`` + ``energy_forces``), nothing is computed in Python.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Evaluator:
    """A one-trial handle used to evaluate U and -grad U at given positions
    (no bias: z_m is reset so that the ratchet force is zero)."""

    def __init__(self, system, params, seed: int = 0):
        self.system = system
        self.batch = B.TrialBatch(system, params, [1], trial_seeds=[seed])
        self.n = system.n_atoms
        self._vel = np.zeros((self.n, 3))

    def energy_and_forces(self, pos: np.ndarray):
        self.batch.set_state(0, pos, self._vel)  # restarts the ratchet: a = 0
        e, F = self.batch.energy_forces(0)
        return float(e[0] + e[1] + e[2] + e[3]), F

    def close(self):
        self.batch.close()


class PotentialEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, evaluator: Evaluator):
        x = pos.detach().to("cpu", torch.float64).numpy().reshape(-1, 3)
        U, F = evaluator.energy_and_forces(x)
        ctx.save_for_backward(torch.from_numpy(-F).reshape(pos.shape).to(pos.device, pos.dtype))
        return pos.new_tensor(U)

    @staticmethod
    def backward(ctx, grad_out):
        (dU,) = ctx.saved_tensors
        return grad_out * dU, None


def potential_energy(pos: torch.Tensor, evaluator: Evaluator) -> torch.Tensor:
    return PotentialEnergy.apply(pos, evaluator)
