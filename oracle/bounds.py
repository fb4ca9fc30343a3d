"""Error bounds of the GPU arithmetic against the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the parity tests and
``__graft_entry__.smoke()`` use these bounds to check the tensor-core path.
They hold none of the method's arithmetic beyond what a bound needs.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24   # FP32 unit roundoff


def bf16_step_bound(J, q, p, zeta, dt, kw, bf16_term=True, h=None):
    """Elementwise bound on |GPU - oracle| for one tensor-core step from the
    same FP32 state: bf16 round-to-nearest of q in the force (relative error
    at most the bf16 unit roundoff 2^-8: 8 significant bits), FP32
    accumulation of n products (n 2^-24), a few FP32 roundings of the update;
    the walls are 1-Lipschitz.  Returns (bound on q, bound on p)."""
    J = np.asarray(J, np.float64)
    n = J.shape[0]
    S = np.abs(q) @ np.abs(J).T
    eF = ((2.0 ** -8 if bf16_term else 0.0) + n * U32) * S
    k, m, q0 = kw["k"], kw["m"], kw["q0"]
    F = q @ J.T + (0.0 if h is None else np.asarray(h, np.float64))
    pn = p + dt * (-k * (q - q0) + zeta * F)
    ep = abs(zeta * dt) * eF + 8 * U32 * (np.abs(p) + np.abs(pn) + dt * (abs(k) * np.abs(q - q0) + abs(zeta) * np.abs(F)))
    eq = (dt / m) * ep + 8 * U32 * (np.abs(q) + (dt / m) * np.abs(pn))
    return eq, ep
