"""The update-order and wall variants on the tensor-core and grouped paths:
literal Eq. 5 (both updates from the old state), the inelastic wall that
zeroes the momentum of a clipped spin, and the wall at |q| = 1 instead of
sqrt(2).  Per step from an identical FP32 state, every element within the
bf16 bound (derived in test_gpu_tc); with wall_zero_p, elements whose clip
decision sits within rounding of the wall may differ and must be rare."""
import numpy as np
import pytest

from _helpers import b, bf16_step_bound, inputs, oracle, params_f64

pytestmark = pytest.mark.gpu

VARIANTS = [
    dict(update_order=1),
    dict(wall_zero_p=1),
    dict(q_max=1.0),
    dict(update_order=1, wall_zero_p=1, q_max=1.0),
]


def _check_step(qg, pg, qo, po, eq, ep, kw):
    bad_q = np.abs(qg - qo) > eq
    bad_p = np.abs(pg - po) > ep
    if kw["wall_zero_p"]:
        qmax = kw["q_max"]
        flip = (np.abs(qg) >= np.float32(qmax)) != (np.abs(qo) >= qmax)
        assert flip.mean() <= 1e-3, flip.mean()
        bad_p &= ~flip
        bad_q &= ~flip
    assert not bad_q.any() and not bad_p.any()


def _scaled_positions(n, R, seed):
    # larger starting amplitude so that walls are reached within a few steps
    return (inputs.positions(n, R, seed0=seed) * 8).astype(np.float32)


@pytest.mark.parametrize("variant", VARIANTS)
def test_tensor_path_variants_per_step(variant):
    n, R, T = 300, 40, 10
    J = inputs.pm1_coupling(n, seed=77)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q = _scaled_positions(n, R, 7700)
    p = np.zeros_like(q)
    touched = 0
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16", **variant) as ctx:
        kw = params_f64(ctx)
        for t in range(T):
            qg, pg, _ = ctx.run(zeta[t:t + 1], dt[t:t + 1], q, p)
            qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], q, p, **kw)
            eq, ep = bf16_step_bound(J, q.astype(np.float64), p.astype(np.float64), float(zeta[t]), float(dt[t]), kw)
            _check_step(qg, pg, qo, po, eq, ep, kw)
            touched += int((np.abs(qo) >= kw["q_max"]).sum())
            q, p = qg, pg
    assert touched > 0  # the wall was reached


@pytest.mark.parametrize("variant", VARIANTS)
def test_grouped_path_variants_per_step(variant):
    members = [(200, 32), (77, 16)]
    Js = [inputs.pm1_coupling(n, seed=80 + k) for k, (n, _) in enumerate(members)]
    qs = [_scaled_positions(n, R, 8000 + k) for k, (n, R) in enumerate(members)]
    ps = [np.zeros_like(q) for q in qs]
    T = 6
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    with b.Group(Js, None, replicas=[R for _, R in members], steps=1, precs=["j_fp8_q_bf16"] * 2,
                 **variant) as g:
        p0 = b.default_params(**variant)
        kw = dict(k=float(np.float32(p0.k)), m=float(np.float32(p0.m)), q0=float(np.float32(p0.q0)),
                  q_max=float(np.float32(p0.q_max)), p_max=float(np.float32(p0.p_max)),
                  order=int(p0.update_order), wall_zero_p=bool(p0.wall_zero_p))
        for t in range(T):
            qg, pg, _ = g.run(zeta[t:t + 1], dt[t:t + 1], qs, ps)
            for k in range(len(members)):
                qo, po = oracle.run(Js[k], None, zeta[t:t + 1], dt[t:t + 1], qs[k], ps[k], **kw)
                eq, ep = bf16_step_bound(Js[k], qs[k].astype(np.float64), ps[k].astype(np.float64),
                                         float(zeta[t]), float(dt[t]), kw)
                _check_step(qg[k], pg[k], qo, po, eq, ep, kw)
            qs, ps = qg, pg
