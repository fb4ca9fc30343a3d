"""torch.autograd binding of si_grad.

``relaxed_energy(J, zeta, dt, k, q_init, ...)`` returns the relaxed Ising
energy at the final step, L = sum_r (-1/2 q_r^T J q_r - h^T q_r), as a scalar
tensor that is differentiable with respect to the schedules ``zeta``, ``dt``
and the spring constant ``k``.  Forward and backward both come from one call
of the library's adjoint sweep (si_grad); nothing is computed in PyTorch.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as b


def _np(x):
    if isinstance(x, torch.Tensor):
        return x.detach().cpu().numpy()
    return np.asarray(x)


class RelaxedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, zeta, dt, k, J, h, q_init, p_init, prec, ckpt_every, extra):
        steps = int(zeta.numel())
        Jn = _np(J).astype(np.float32)
        n = Jn.shape[0]
        R = int(_np(q_init).size // n)
        with b.Context(Jn, None if h is None else _np(h).astype(np.float32), replicas=R, steps=steps,
                       prec=prec, k=float(k), ckpt_every=int(ckpt_every), **(extra or {})) as c:
            obj, gz, gd, gk = c.grad(_np(zeta).astype(np.float32), _np(dt).astype(np.float32),
                                     _np(q_init).astype(np.float32),
                                     None if p_init is None else _np(p_init).astype(np.float32))
        dev = zeta.device
        ctx.save_for_backward(torch.from_numpy(np.array(gz)).to(dev), torch.from_numpy(np.array(gd)).to(dev),
                              torch.tensor(gk, dtype=torch.float32, device=dev))
        return torch.tensor(obj, dtype=torch.float32, device=dev)

    @staticmethod
    def backward(ctx, gout):
        gz, gd, gk = ctx.saved_tensors
        return (gout * gz, gout * gd, gout * gk, None, None, None, None, None, None, None)


def relaxed_energy(J, zeta, dt, k, q_init, p_init=None, h=None, prec="fp32", ckpt_every=50, **extra):
    """Differentiable relaxed final energy (see module docstring)."""
    if not isinstance(k, torch.Tensor):
        k = torch.tensor(float(k), dtype=torch.float32, device=zeta.device)
    return RelaxedEnergy.apply(zeta, dt, k, J, h, q_init, p_init, prec, ckpt_every, extra)
