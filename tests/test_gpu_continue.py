"""si_run with q_init NULL continues from the context's state: a segmented
run equals the same run restarted from the previous segment's outputs (bit
for bit on the FP32 and tensor paths, whose state is FP32), and in FP64 it
keeps the double state (checked against the oracle's unsegmented run)."""
import numpy as np
import pytest

from _helpers import TOL_FP64_100, b, inputs, normwise_rel, oracle, params_f64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,n,R", [("fp32", 300, 1), ("fp32", 130, 3), ("fp32", 77, 9),
                                      ("j_fp8_q_bf16", 300, 70), ("j_fp8_q_bf16", 2000, 256)])
def test_continue_equals_restart_from_outputs(prec, n, R):
    T = 13   # odd: the final state sits in the second exchange buffer
    J = inputs.pm1_coupling(n, seed=31)
    z, d = inputs.zeta_ramp(3 * T), inputs.dt_const(3 * T)
    q0 = inputs.positions(n, R, seed0=310)
    with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
        q1, p1, _ = ctx.run(z[:T], d[:T], q0)
        q2, p2, s2 = ctx.run(z[T:2 * T], d[T:2 * T], None)
        q3, p3, s3 = ctx.run(z[2 * T:], d[2 * T:], None)
        e3, c3, _ = ctx.energy(None)
    with b.Context(J, replicas=R, steps=T, prec=prec) as cx:
        q2x, p2x, s2x = cx.run(z[T:2 * T], d[T:2 * T], q1, p1)
        q3x, p3x, s3x = cx.run(z[2 * T:], d[2 * T:], q2x, p2x)
    for a_, b_ in ((q2, q2x), (p2, p2x), (s2, s2x), (q3, q3x), (p3, p3x), (s3, s3x)):
        np.testing.assert_array_equal(a_, b_)
    np.testing.assert_array_equal(e3, oracle.energy(J, None, s3).astype(np.int64))
    np.testing.assert_array_equal(c3, oracle.cut(J, s3).astype(np.int64))


@pytest.mark.parametrize("n,R", [(64, 1), (65, 9)])
def test_continue_fp64_keeps_the_double_state(n, R):
    """Two 50-step segments in FP64 against the oracle's 100-step run, at the
    FP64 debug bar (the state never passes through float)."""
    T = 50
    J = inputs.pm1_coupling(n, seed=32)
    z, d = inputs.zeta_ramp(2 * T), inputs.dt_const(2 * T)
    q0 = inputs.positions(n, R, seed0=320)
    with b.Context(J, replicas=R, steps=T, prec="fp64") as ctx:
        ctx.run(z[:T], d[:T], q0)
        _, _, sg = ctx.run(z[T:], d[T:], None)
        qg, pg = ctx.get_state()
        kw = params_f64(ctx)
    qo, po = oracle.run(J, None, z, d, q0, **kw)
    assert normwise_rel(qg, pg, qo, po) <= TOL_FP64_100
    np.testing.assert_array_equal(sg, oracle.sign(qo))


def test_continue_after_grad_starts_from_its_forward_state():
    n, R, T = 96, 4, 20
    J = inputs.pm1_coupling(n, seed=33)
    z, d = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=330)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as ctx:
        ctx.grad(z, d, q0)
        qT, pT = ctx.get_state()
        q1, p1, _ = ctx.run(z, d, None)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as cx:
        q1x, p1x, _ = cx.run(z, d, qT.astype(np.float32), pT.astype(np.float32))
    np.testing.assert_array_equal(q1, q1x)
    np.testing.assert_array_equal(p1, p1x)


def test_continue_needs_a_state_and_no_momenta():
    n, T = 40, 5
    J = inputs.pm1_coupling(n, seed=34)
    z, d = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, 1, seed0=340)
    with b.Context(J, replicas=1, steps=T) as ctx:
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.run(z, d, None)
        assert ei.value.status == b.SI_ERR_INVALID_ARG
        ctx.run(z, d, q0)
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.run(z, d, None, np.zeros((1, n), np.float32))
        assert ei.value.status == b.SI_ERR_INVALID_ARG
        q, _, _ = ctx.run(z, d, None)
    assert np.isfinite(q).all()
