"""torch.autograd front end of the learned surrogate: the energy of a configuration as a
differentiable function of the atom positions.

forward: the positions (a float64 CUDA tensor [N][3], caller order) are handed to the library
(md_set_state, device to device), whose kernels evaluate the descriptors, the network and the
force gather (md_eam_forces); the total energy comes back as a float64 scalar tensor and the
forces F = -dU/dr (the library's backward-for-forces kernels) are kept on the device.
backward: dU/dr = -F, scaled by the incoming gradient of the energy.

The library does every step of the evaluation; this module only moves pointers and applies the
chain rule to the one scalar.  There is no CPU path: without libmd.so the first call raises.

    sys = md.SurrogateSystem(w, theta, gmu, ginv, net="fp32")
    pos = torch.tensor(w.pos, device="cuda", requires_grad=True)
    U = SurrogateEnergy.apply(pos, sys)
    U.backward()              # pos.grad = -forces
"""
from __future__ import annotations

import torch

from . import md


class SurrogateEnergy(torch.autograd.Function):
    """U(r) of a surrogate context (md.SurrogateSystem); forward and backward on the GPU."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, system: "md.SurrogateSystem") -> torch.Tensor:
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2 and pos.shape[1] == 3):
            raise ValueError("pos must be a float64 CUDA tensor of shape [N, 3]")
        if pos.shape[0] != system.n:
            raise ValueError(f"pos has {pos.shape[0]} atoms, the system {system.n}")
        p = pos.detach().contiguous()
        torch.cuda.current_stream().synchronize()   # the library works on its own stream
        md.md_set_state(system.ctx, pos=p)
        energy = md.md_eam_forces(system.ctx)
        force = torch.empty_like(p)
        md.md_get(system.ctx, md.MD_GET_FORCE, force)
        ctx.save_for_backward(force)
        return torch.tensor(energy, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, grad_energy: torch.Tensor):
        (force,) = ctx.saved_tensors
        return -grad_energy * force, None


class SurrogatePotential(torch.nn.Module):
    """nn.Module view of a surrogate context: forward(pos) -> U, forces(pos) -> -dU/dr."""

    def __init__(self, system: "md.SurrogateSystem"):
        super().__init__()
        self.system = system

    def forward(self, pos: torch.Tensor) -> torch.Tensor:
        return SurrogateEnergy.apply(pos, self.system)

    def forces(self, pos: torch.Tensor) -> torch.Tensor:
        p = pos.detach().requires_grad_(True)
        (g,) = torch.autograd.grad(self.forward(p), p)
        return -g
