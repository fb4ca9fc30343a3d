"""torch.autograd binding of si_grad.

``relaxed_energy(J, zeta, dt, k, q_init, ...)`` returns the relaxed Ising
energy at the final step, L = sum_r (-1/2 q_r^T J q_r - h^T q_r), as a scalar
tensor that is differentiable with respect to the schedules ``zeta``, ``dt``
and the spring constant ``k``.  Forward and backward both come from one call
of the library's adjoint sweep (si_grad); nothing is computed in PyTorch.

The binding works on device memory.  CUDA tensors are handed to the library
by pointer, on the caller's current stream, and the gradients are written
straight into CUDA tensors; nothing is staged through host memory.  The
library context that holds the copy of J is created once and cached.  The
cache keeps a reference to J (and h), keyed on their identity together with
the replica and step counts, the precision, the checkpoint interval, the
extra parameters and the stream; a tensor written in place since (its
version counter moved) gets a fresh context.  A new value of k reaches the
cached context through si_set_params, so tuning k does not copy J again.
``clear_cache()`` releases the contexts (needed after writing into a NumPy J
in place, which has no version counter).
"""
from __future__ import annotations

import threading

import numpy as np
import torch

from . import _binding as b

_cache: dict = {}
_lock = threading.Lock()
stats = {"created": 0, "reused": 0}


def clear_cache():
    """Destroy every cached library context."""
    with _lock:
        for entry in _cache.values():
            entry[3].close()
        _cache.clear()


def _version(x):
    return x._version if isinstance(x, torch.Tensor) else None


def _as_arg(x, dev):
    """A contiguous float32 array for the library: CUDA tensors stay on the
    device (moved to `dev` if they live elsewhere); host data is passed as
    NumPy (the library copies it in)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        x = x.detach()
        if dev is not None and x.device != dev:
            x = x.to(dev)
        return x.to(torch.float32).contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


def _context(J, h, R, steps, prec, ckpt_every, extra, k, stream):
    key = (id(J), id(h), R, steps, prec, int(ckpt_every), tuple(sorted((extra or {}).items())),
           int(stream.cuda_stream) if stream is not None else 0)
    versions = (_version(J), _version(h))
    with _lock:
        entry = _cache.get(key)
        if entry is not None and entry[2] != versions:
            entry[3].close()          # J or h was written in place since
            entry = None
        if entry is None:
            dev = stream.device if stream is not None else None
            Jd = _as_arg(J, dev)
            c = b.Context(Jd, _as_arg(h, dev), n=int(Jd.shape[0]), replicas=R, steps=steps, prec=prec,
                          k=float(k), ckpt_every=int(ckpt_every),
                          stream=None if stream is None else stream.cuda_stream, **(extra or {}))
            # the references keep id(J), id(h) from being reused while cached
            _cache[key] = (J, h, versions, c)
            stats["created"] += 1
            return c
        c = entry[3]
        stats["reused"] += 1
        if np.float32(c.params.k) != np.float32(float(k)):
            c.set_params(k=float(k))
        return c


class RelaxedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, zeta, dt, k, J, h, q_init, p_init, prec, ckpt_every, extra):
        steps = int(zeta.numel())
        on_gpu = zeta.is_cuda
        dev = zeta.device
        stream = torch.cuda.current_stream(dev) if on_gpu else None
        n = int(J.shape[0])
        R = int((q_init.numel() if isinstance(q_init, torch.Tensor) else np.size(q_init)) // n)
        c = _context(J, h, R, steps, prec, ckpt_every, extra, float(k), stream)
        # outputs: device tensors when the schedule lives on the GPU
        out_dev = dev if on_gpu else torch.device("cpu")
        gz = torch.zeros(steps, dtype=torch.float32, device=out_dev)
        gd = torch.zeros(steps, dtype=torch.float32, device=out_dev)
        gk = torch.empty(1, dtype=torch.float32, device=out_dev)
        obj = torch.empty(1, dtype=torch.float32, device=out_dev)
        args_dev = dev if on_gpu else None
        c.grad_into(_as_arg(zeta, args_dev), _as_arg(dt, args_dev), _as_arg(q_init, args_dev),
                    _as_arg(p_init, args_dev), gz if steps else None, gd if steps else None, gk, obj)
        ctx.save_for_backward(gz, gd, gk[0])
        return obj[0]

    @staticmethod
    def backward(ctx, gout):
        gz, gd, gk = ctx.saved_tensors
        return (gout * gz, gout * gd, gout * gk, None, None, None, None, None, None, None)


def relaxed_energy(J, zeta, dt, k, q_init, p_init=None, h=None, prec="fp32", ckpt_every=50, **extra):
    """Differentiable relaxed final energy (see module docstring)."""
    if not isinstance(k, torch.Tensor):
        k = torch.tensor(float(k), dtype=torch.float32, device=zeta.device)
    return RelaxedEnergy.apply(zeta, dt, k, J, h, q_init, p_init, prec, ckpt_every, extra)
