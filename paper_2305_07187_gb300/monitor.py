"""Hamiltonian-drift monitor.

At a constant coupling coefficient zeta the spring system of Eqs. 2-4 has the
Hamiltonian H = sum p^2/(2m) + k/2 sum (q - q0)^2 + zeta (-1/2 q^T J q - h^T q).
The symplectic step of Eq. 8 keeps H within O(dt) of its start, with no
secular drift, as long as no spin touches a wall (the walls of Eq. 6 are
inelastic and remove energy).  ``hamiltonian_drift`` runs a context in
segments of ``ctx.steps`` steps at constant zeta and evaluates H of every
replica after each segment in FP64 on the device (si_hamiltonian).  Growth of
|H - H_0| beyond the O(dt) band flags a time step too large for the
couplings, or a fault in the integrator.
"""
from __future__ import annotations

import numpy as np


def hamiltonian_drift(ctx, zeta, dt, q_init, p_init=None, segments=10):
    """Returns (H, drift): H[segments + 1][R] (FP64, H[0] of the initial
    state) and drift[R] = max_t |H_t - H_0| / max(|H_0|, tiny)."""
    T = ctx.steps
    z = np.full(T, zeta, np.float32)
    d = np.full(T, dt, np.float32)
    q = np.ascontiguousarray(q_init, dtype=np.float32).reshape(-1, ctx.n)
    p = np.zeros_like(q) if p_init is None else np.ascontiguousarray(p_init, dtype=np.float32).reshape(q.shape)
    H = [ctx.hamiltonian(q, p, zeta)]
    for _ in range(segments):
        q, p, _ = ctx.run(z, d, q, p)
        H.append(ctx.hamiltonian(q, p, zeta))
    H = np.stack(H)
    drift = np.abs(H - H[0]).max(axis=0) / np.maximum(np.abs(H[0]), np.finfo(np.float64).tiny)
    return H, drift
