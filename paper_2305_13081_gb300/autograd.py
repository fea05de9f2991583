"""The staggered solve's objective as a differentiable function of the
eigenstrain field: a torch.autograd.Function over fftmech_adjoint_eigenstrain
(the library's discrete adjoint with checkpointed recomputation of load
steps). The forward call computes the objective and its gradient in one
library call; backward scales the stored gradient by the incoming one.
Argument marshalling only: every step runs in the CUDA library.
"""

import torch

from . import fftmech as fm

OBJECTIVES = {"energy": fm.FFTMECH_OBJ_ENERGY, "damage": fm.FFTMECH_OBJ_DAMAGE}


class EigenstrainObjective(torch.autograd.Function):
    """J(e): total elastic energy or summed damage after len(ramp) staggered
    steps with the eigenstrain ramp[s] e(x)."""

    @staticmethod
    def forward(ctx, e_field, handle, phase, ramp, eps_mac, objective, checkpoint_every):
        e = e_field.detach().contiguous()
        grad = torch.empty(e.numel(), dtype=torch.float64, device=e.device)
        J, _ = fm.fftmech_adjoint_eigenstrain(handle, phase, e, ramp, eps_mac, OBJECTIVES[objective],
                                              checkpoint_every, grad)
        ctx.save_for_backward(grad)
        ctx.shape, ctx.dtype = e_field.shape, e_field.dtype
        return torch.tensor(J, dtype=torch.float64, device=e.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        g = (gJ * grad).to(ctx.dtype).view(ctx.shape)
        return g, None, None, None, None, None, None


def eigenstrain_objective(e_field, context, phase, ramp, eps_mac=None, objective="energy", checkpoint_every=5):
    """Differentiable J(e_field) on a fftmech Context (one problem);
    e_field: a CUDA tensor of the context's field type, phase: uint8 CUDA
    tensor."""
    return EigenstrainObjective.apply(e_field, context.handle, phase, list(ramp), eps_mac, objective,
                                      int(checkpoint_every))
