"""Synthetic studies on the batched path.

The paper's figures ask how the coupling-coefficient strategy shapes the
result (Fig. 5: fixed small, fixed large, and ramped zeta with different step
lengths), how the energy falls over a run (Fig. 4) and how the per-replica
results are distributed (Fig. 6).  The benchmark instance and the
comparison systems are not available, so these studies run on seeded
stand-in graphs and report distributions only:
- zeta strategies: fixed 0.8 zeta0, fixed 10 zeta0, linear ramps with
  plateaus of L = 1, 200 and 1000 steps, and a schedule tuned by the
  adjoint gradient;
- the update-order and wall variants (literal Eq. 5, momentum-zeroing wall,
  wall at |q| = 1);
- empirical CDFs of the final cuts and energy trajectories read out every
  K steps.

Host logic only: every run and every readout goes through the library.
"""
from __future__ import annotations

import numpy as np

from . import inputs
from . import schedule as _schedule

STRATEGIES = ("fixed-0.8z0", "fixed-10z0", "ramp-L1", "ramp-L200", "ramp-L1000")


def zeta_strategies(T: int, tuned_knots=None) -> dict:
    """The coupling-coefficient schedules of the zeta study, each [T] float32."""
    out = {
        "fixed-0.8z0": np.full(T, inputs.ZETA_START, np.float32),
        "fixed-10z0": np.full(T, inputs.ZETA_END, np.float32),
        "ramp-L1": inputs.zeta_ramp(T, plateau=1),
        "ramp-L200": inputs.zeta_ramp(T, plateau=200),
        "ramp-L1000": inputs.zeta_ramp(T, plateau=1000),
    }
    if tuned_knots is not None:
        out["tuned"] = _schedule.expand(tuned_knots, T)
    return out


def empirical_cdf(values):
    """(x, F): sorted values and F(x_k) = (k + 1) / len."""
    x = np.sort(np.asarray(values).ravel())
    return x, np.arange(1, x.size + 1, dtype=np.float64) / max(x.size, 1)


def summarize(values) -> dict:
    v = np.asarray(values, dtype=np.float64).ravel()
    return {"best": float(v.max()), "median": float(np.median(v)), "mean": float(v.mean()),
            "p10": float(np.percentile(v, 10)), "p90": float(np.percentile(v, 90)), "count": int(v.size)}


def final_cuts(J, q0, zeta, dt, prec="j_fp8_q_bf16", stream=None, **params):
    """Run every replica through the whole schedule; return (cuts int64, spins int8)."""
    from . import _binding as b
    q0 = np.ascontiguousarray(q0, dtype=np.float32)
    R = q0.shape[0]
    with b.Context(J, replicas=R, steps=len(zeta), prec=prec, stream=stream, **params) as ctx:
        _, _, s = ctx.run(zeta, dt, q0)
        _, cut, _ = ctx.energy(s)
    return cut.astype(np.int64), s


def energy_trajectory(J, q0, zeta, dt, every: int, prec="j_fp8_q_bf16", stream=None, **params):
    """Exact Ising energy of every replica's sign readout after every `every`
    steps: segments of `every` steps that continue from the context's own
    state (si_run with q_init NULL), each followed by the readout of the
    run's spins in place.  Returns (steps [S], energies int64 [S][R], final
    spins)."""
    from . import _binding as b
    T = len(zeta)
    if every <= 0 or T % every:
        raise ValueError("the run length must be a multiple of the readout interval")
    q = np.ascontiguousarray(q0, dtype=np.float32)
    R, n = q.shape
    nseg = T // every
    s = np.empty((R, n), np.int8)
    steps, energies = [], []
    with b.Context(J, replicas=R, steps=every, prec=prec, stream=stream, **params) as ctx:
        for seg in range(nseg):
            sl = slice(seg * every, (seg + 1) * every)
            ctx.run_into(zeta[sl], dt[sl], q if seg == 0 else None, None, None, None,
                         s if seg == nseg - 1 else None)
            e, _, _ = ctx.energy(None)
            steps.append((seg + 1) * every)
            energies.append(e.astype(np.int64))
    return np.asarray(steps), np.stack(energies), s
