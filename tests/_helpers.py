"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle
from oracle import bounds
from paper_2305_07187_gb300 import _binding as b
from paper_2305_07187_gb300 import inputs

SQ2F = b.SQRT2_F32  # the float32 wall the library uses by default
TOL_FP64_100 = 1e-10  # FP64 debug path, 100 free-running steps (normwise relative)


def params_f64(ctx):
    """The context's integrator parameters as the oracle should receive them
    (the float32 values the library holds, widened exactly)."""
    p = ctx.params
    return dict(k=float(np.float32(p.k)), m=float(np.float32(p.m)), q0=float(np.float32(p.q0)),
                q_max=float(np.float32(p.q_max)), p_max=float(np.float32(p.p_max)),
                order=int(p.update_order), wall_zero_p=bool(p.wall_zero_p))


def normwise_rel(qg, pg, qo, po):
    num = max(np.abs(qg - qo).max(), np.abs(pg - po).max())
    den = max(np.abs(qo).max(), np.abs(po).max(), 1e-30)
    return num / den


def teacher_forced(ctx1, J, h, zeta, dt, q, p, steps_to_check):
    """Drive a steps=1 context along its own trajectory; at each step compare
    the GPU step with the oracle's FP64 step from the identical FP32 state.
    Returns the worst normwise relative error and the final state."""
    worst = 0.0
    kw = params_f64(ctx1)
    J64 = np.asarray(J, np.float64)
    h64 = None if h is None else np.asarray(h, np.float64)
    for t in steps_to_check:
        qg, pg, _ = ctx1.run(zeta[t:t + 1], dt[t:t + 1], q, p)
        qo, po = oracle.run(J64, h64, zeta[t:t + 1].astype(np.float64),
                            dt[t:t + 1].astype(np.float64), q.astype(np.float64),
                            p.astype(np.float64), **kw)
        worst = max(worst, normwise_rel(qg, pg, qo, po))
        q, p = qg, pg
    return worst, q, p


U32 = 2.0 ** -24

bf16_step_bound = bounds.bf16_step_bound


def random_spins(R, n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return np.where(g.random((R, n)) < 0.5, -1, 1).astype(np.int8)


__all__ = ["oracle", "inputs", "b", "SQ2F", "params_f64", "normwise_rel", "teacher_forced",
           "random_spins", "bf16_step_bound"]
