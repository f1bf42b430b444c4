"""The potential U(X, Y) of Eq. Lang as a differentiable PyTorch function.

``PotentialEnergy.apply(pos, evaluator)`` returns the total potential energy
(Lennard-Jones + reaction field + bonds + angles, FP64 totals of the CUDA
kernels); its backward is the force kernel's output, dU/dX = -F, times the
incoming gradient.  PyTorch supplies the autograd plumbing and the device
memory only: the energy and the forces come from the C ABI, nothing is
computed in Python.

* CUDA tensors (``(n_atoms, 3)`` or a batch ``(n_conf, n_atoms, 3)``, FP64)
  go through ``sim_potential_device``: device pointers in and out on the
  tensor's current stream, one configuration per trial of the evaluator's
  handle, no host round trip; a trial's list is rebuilt only when the new
  configuration has moved an atom beyond the list buffer.
* Host tensors take the host path (``sim_set_state`` + ``energy_forces``).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Evaluator:
    """A handle used to evaluate U and -grad U at given positions: n_conf
    trials of the system, one configuration each (no bias: on the host path
    z_m is reset so that the ratchet force is zero; the device path leaves the
    bias out)."""

    def __init__(self, system, params, seed: int = 0, n_conf: int = 1):
        self.system = system
        self.n_conf = int(n_conf)
        self.batch = B.TrialBatch(system, params, [self.n_conf], trial_seeds=[seed + k for k in range(self.n_conf)])
        self.n = system.n_atoms
        self._vel = np.zeros((self.n, 3))

    def energy_and_forces(self, pos: np.ndarray):
        """Host path: one configuration (trial 0)."""
        self.batch.set_state(0, pos, self._vel)  # restarts the ratchet: a = 0
        e, F = self.batch.energy_forces(0)
        return float(e[0] + e[1] + e[2] + e[3]), F

    def device_energy_and_forces(self, pos: torch.Tensor):
        """Device path: pos (n_conf, n_atoms, 3) FP64 CUDA tensor; returns
        (energies (n_conf,), forces like pos), both CUDA tensors, ordered on
        the current stream."""
        if pos.shape != (self.n_conf, self.n, 3) or pos.dtype != torch.float64 or not pos.is_cuda:
            raise ValueError(f"expected a CUDA float64 tensor of shape {(self.n_conf, self.n, 3)}")
        x = pos.contiguous()
        energy = torch.empty(self.n_conf, dtype=torch.float64, device=x.device)
        forces = torch.empty_like(x)
        B.sim_potential_device(self.batch.h, x.data_ptr(), energy.data_ptr(), forces.data_ptr(),
                               torch.cuda.current_stream(x.device).cuda_stream)
        return energy, forces

    def close(self):
        self.batch.close()


class PotentialEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, evaluator: Evaluator):
        if pos.is_cuda:
            batched = pos.dim() == 3
            x = pos.detach().to(torch.float64).reshape(evaluator.n_conf, -1, 3)
            U, F = evaluator.device_energy_and_forces(x)
            ctx.save_for_backward((-F).reshape(pos.shape).to(pos.dtype))
            return (U if batched else U[0]).to(pos.dtype)
        x = pos.detach().to("cpu", torch.float64).numpy().reshape(-1, 3)
        U, F = evaluator.energy_and_forces(x)
        ctx.save_for_backward(torch.from_numpy(-F).reshape(pos.shape).to(pos.device, pos.dtype))
        return pos.new_tensor(U)

    @staticmethod
    def backward(ctx, grad_out):
        (dU,) = ctx.saved_tensors
        if dU.dim() == 3:  # a batch: one energy per configuration
            return grad_out.reshape(-1, 1, 1) * dU, None
        return grad_out * dU, None


def potential_energy(pos: torch.Tensor, evaluator: Evaluator) -> torch.Tensor:
    return PotentialEnergy.apply(pos, evaluator)
