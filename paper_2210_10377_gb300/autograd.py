"""torch.autograd.Function over the library's discrete adjoint.

force_objective(f0, tau, u_in, mask, steps, window, wx, wy, storage) returns
J = the window-averaged wx Fx + wy Fy of the algorithm-B force after `steps`
channel steps from the pre-collision state f0; its backward pass hands out the
gradients the adjoint computed (dJ/df0, dJ/dtau, dJ/du_in).  The forward and
the adjoint both run in the library's CUDA kernels (lbm_adjoint).
"""
import numpy as np
import torch

from . import binding


class ForceObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, tau, u_in, mask, steps, window, wx, wy, storage):
        m = np.ascontiguousarray(mask, np.uint8)
        u = u_in.detach().to("cpu", torch.float64).numpy()
        lat = binding.Lattice(m, float(tau), u, storage=storage)
        lat.set_populations(f0.detach().to("cpu", torch.float64).numpy())
        # a CUDA f0 gets its gradient straight from device memory
        J, dtau, du, df0 = lat.adjoint(int(steps), int(window), float(wx), float(wy), df0_device=f0.is_cuda)
        lat.close()
        df0 = df0 if f0.is_cuda else torch.from_numpy(df0)
        ctx.save_for_backward(df0.to(f0.device, f0.dtype),
                              torch.tensor(dtau, dtype=tau.dtype, device=tau.device),
                              torch.from_numpy(du).to(u_in.device, u_in.dtype))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        df0, dtau, du = ctx.saved_tensors
        g = gJ.to(torch.float64)
        return (g.to(df0.dtype) * df0, g.to(dtau.dtype) * dtau, g.to(du.dtype) * du, None, None,
                None, None, None, None)


def force_objective(f0, tau, u_in, mask, steps, window, wx=1.0, wy=0.0, storage="f32"):
    return ForceObjective.apply(f0, tau, u_in, mask, steps, window, wx, wy, storage)
