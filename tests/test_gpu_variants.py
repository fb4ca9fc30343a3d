"""The update-order and wall variants on every path: literal Eq. 5 (both
updates from the old state), the inelastic wall that zeroes the momentum of a
clipped spin, and the wall at |q| = 1 instead of sqrt(2).  Per step from an
identical FP32 state: on the tensor-core and grouped paths every element
within the bf16 bound (derived in test_gpu_tc), on the FP32 CUDA-core paths
(k_plain for R <= 4, k_tiled_f32 above) within the 1e-6 normwise bar.  With
wall_zero_p a spin whose clip decision differs between GPU and oracle has a
different momentum (0 against a finite value); such a spin is excused only
when the unclipped side sits within the step's error bound of the wall, and
such spins must be rare."""
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


def _clip_flips(qg, pg, qo, po, eq, kw):
    """Spins whose wall decision differs between GPU and oracle: on one side
    the position was clipped and the momentum zeroed, on the other it was not
    (it stayed inside, or landed exactly on the wall without being clipped,
    which leaves p as it was).  Asserts that each lies within the position
    bound eq of the wall (the walls are 1-Lipschitz, so the unclipped side's
    |q| is at least q_max - eq) and that they are rare."""
    qmax = kw["q_max"]
    zeroed_g = (np.abs(qg) >= np.float32(qmax)) & (pg == 0)
    zeroed_o = (np.abs(qo) >= qmax) & (po == 0)
    flip = zeroed_g != zeroed_o
    near = (qmax - np.minimum(np.abs(qg).astype(np.float64), np.abs(qo))) <= eq
    assert not (flip & ~near).any(), "clip decision differs away from the wall"
    assert flip.mean() <= 1e-3, flip.mean()
    return flip


def _check_step(qg, pg, qo, po, eq, ep, kw):
    bad_q = np.abs(qg - qo) > eq
    bad_p = np.abs(pg - po) > ep
    if kw["wall_zero_p"]:
        flip = _clip_flips(qg, pg, qo, po, eq, kw)
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


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("R", [3, 40])
def test_fp32_paths_variants_per_step(variant, R):
    """The FP32 CUDA-core kernels (k_plain at R = 3, k_tiled_f32 at R = 40)
    under every variant: per-step normwise relative error <= 1e-6 over the
    spins whose wall decision agrees; a differing decision must sit within
    1e-5 relative of the wall (about 100 FP32 roundings of q)."""
    n, T = 300, 12
    J = inputs.pm1_coupling(n, seed=78)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q = _scaled_positions(n, R, 7800)
    p = np.zeros_like(q)
    touched = 0
    with b.Context(J, replicas=R, steps=1, prec="fp32", **variant) as ctx:
        assert ("plain_persistent" if R <= 4 else "simt_tiled") in ctx.describe()
        kw = params_f64(ctx)
        for t in range(T):
            qg, pg, _ = ctx.run(zeta[t:t + 1], dt[t:t + 1], q, p)
            qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], q, p, **kw)
            keep = np.ones(qg.shape, bool)
            if kw["wall_zero_p"]:
                keep = ~_clip_flips(qg, pg, qo, po, 1e-5 * kw["q_max"], kw)
            num = max(np.abs(qg - qo)[keep].max(), np.abs(pg - po)[keep].max())
            den = max(np.abs(qo).max(), np.abs(po).max())
            assert num / den <= 1e-6, (t, num / den)
            touched += int((np.abs(qo) >= kw["q_max"]).sum())
            q, p = qg, pg
    assert touched > 0  # the wall was reached
