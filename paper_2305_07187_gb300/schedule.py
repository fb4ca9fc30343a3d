"""Coupling-coefficient schedule tuned by the adjoint gradient.

The paper ramps zeta linearly, piecewise constant, from 0.8 zeta0 to
10 zeta0 (the "dynamic equilibrium" of Fig. 5) and notes that the slower the
ramp, the better the result.  Here the schedule is a free function: K knot
values on a uniform grid over the run, linearly interpolated to the T steps,
zeta = W c with W the (T, K) interpolation matrix.  si_grad returns dL/dzeta_n
of the relaxed final energy L; the knot gradient is W^T dL/dzeta.  Adam steps
on the knots, projected onto zeta >= 0, lower L.

Nothing of the method's arithmetic runs here: the forward run, the adjoint
sweep and the objective all come from the library (or, in tests, from any
callable with the same contract).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def knot_matrix(T: int, K: int) -> np.ndarray:
    """(T, K) linear interpolation matrix from K knots at x_k = k (T-1)/(K-1)
    (step units) to the steps n = 0..T-1; each row sums to 1."""
    if K < 2 or T < 1:
        raise ValueError("need K >= 2 knots and T >= 1 steps")
    W = np.zeros((T, K), dtype=np.float64)
    x = np.arange(T, dtype=np.float64) * (K - 1) / max(T - 1, 1)
    lo = np.minimum(np.floor(x).astype(np.int64), K - 2)
    frac = x - lo
    W[np.arange(T), lo] = 1.0 - frac
    W[np.arange(T), lo + 1] = frac
    return W


def expand(knots, T: int) -> np.ndarray:
    """Per-step schedule (float32) of the knot values."""
    knots = np.asarray(knots, dtype=np.float64)
    return (knot_matrix(T, knots.size) @ knots).astype(np.float32)


def ramp_knots(K: int, start: float, end: float) -> np.ndarray:
    """Knots of the paper's linear ramp (plateau length 1)."""
    return np.linspace(start, end, K)


def transfer(knots, n_from: int, n_to: int) -> np.ndarray:
    """Carry a schedule tuned at n_from spins to n_to spins for random +-1
    complete graphs.  The coupling force of a spin grows like sqrt(n) (the
    spectral radius of J is about 2 sqrt(n)), so zeta is scaled by
    sqrt(n_from / n_to) to keep zeta * |J q| against the spring k q."""
    return np.asarray(knots, dtype=np.float64) * math.sqrt(n_from / n_to)


@dataclass
class TuneResult:
    knots: np.ndarray                  # best knots found
    objective: float                   # L at the best knots
    initial: float                     # L at the starting knots
    history: list = field(default_factory=list)   # L at every iterate


def tune_zeta(grad_fn, knots0, T: int, iters: int = 20, lr: float = 0.02,
              zeta_min: float = 0.0, zeta_max: float | None = None,
              betas=(0.9, 0.999), eps: float = 1e-8) -> TuneResult:
    """Projected Adam on the knot values.

    grad_fn(zeta[T] float32) -> (L, dL/dzeta[T]).  Returns the best knots
    seen (lowest L), so the result is never worse than the start."""
    c = np.asarray(knots0, dtype=np.float64).copy()
    W = knot_matrix(T, c.size)
    m1 = np.zeros_like(c)
    m2 = np.zeros_like(c)
    best_c, best_L, first = c.copy(), math.inf, None
    hist = []
    for it in range(iters + 1):
        L, gz = grad_fn((W @ c).astype(np.float32))
        L = float(L)
        hist.append(L)
        if first is None:
            first = L
        if L < best_L:
            best_L, best_c = L, c.copy()
        if it == iters:
            break
        g = W.T @ np.asarray(gz, dtype=np.float64)
        m1 = betas[0] * m1 + (1 - betas[0]) * g
        m2 = betas[1] * m2 + (1 - betas[1]) * g * g
        mh = m1 / (1 - betas[0] ** (it + 1))
        vh = m2 / (1 - betas[1] ** (it + 1))
        c = c - lr * mh / (np.sqrt(vh) + eps)
        c = np.maximum(c, zeta_min)
        if zeta_max is not None:
            c = np.minimum(c, zeta_max)
    return TuneResult(best_c, best_L, first, hist)


class LibraryGrad:
    """grad_fn backed by si_grad on one FP32 (or FP64) context of T steps,
    created once and reused for every iterate.  Use as a context manager."""

    def __init__(self, J, q_init, dt, h=None, prec="fp32", **params):
        from . import _binding as b
        J = np.asarray(J, dtype=np.float32)
        self.n = J.shape[0]
        self.q_init = np.ascontiguousarray(q_init, dtype=np.float32).reshape(-1, self.n)
        self.dt = np.ascontiguousarray(dt, dtype=np.float32)
        self.ctx = b.Context(J, h, replicas=self.q_init.shape[0], steps=self.dt.size, prec=prec, **params)

    def __call__(self, zeta):
        L, gz, _, _ = self.ctx.grad(zeta, self.dt, self.q_init)
        return L, gz

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
