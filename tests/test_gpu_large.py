"""si_create / si_run at sizes whose persistent tensor-core grid would not be
co-resident (many M tiles x replica blocks).  The library then serves the
context with the grouped per-step kernel as a one-member group; every call
of the context keeps its meaning: runs continue in place, the readout takes
the run's own spins, and the state copies read the member's state.

Parity: teacher-forced per step against the FP64 oracle on a slice of the
replicas (the bf16 bound of test_gpu_tc), runs equal to the grouped API's
one-member group bit for bit, and at n = 32768 two steps against the oracle.
"""
import numpy as np
import pytest

from _helpers import b, bf16_step_bound, inputs, oracle, params_f64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["j_fp8_q_bf16", "j_bf16_q_bf16"])
def test_n8192_r512_per_step_on_a_replica_slice(prec):
    n, R, T, S = 8192, 512, 3, 6
    J = inputs.pm1_coupling(n, seed=81) if prec == "j_fp8_q_bf16" else inputs.gauss_coupling_bf16(n, seed=81)
    zeta = inputs.zeta_ramp(2000)[1200:1200 + T]
    dt = inputs.dt_const(T)
    q = (inputs.positions(n, R, seed0=8100) * 4).astype(np.float32)
    p = np.zeros_like(q)
    with b.Context(J, replicas=R, steps=1, prec=prec) as ctx:
        assert "grouped-step" in ctx.describe()
        kw = params_f64(ctx)
        for t in range(T):
            qg, pg, sg = ctx.run(zeta[t:t + 1], dt[t:t + 1], q, p)
            qs, ps = q[:S], p[:S]
            qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], qs, ps, **kw)
            eq, ep = bf16_step_bound(J, qs.astype(np.float64), ps.astype(np.float64), float(zeta[t]),
                                     float(dt[t]), kw)
            assert (np.abs(qg[:S] - qo) <= eq).all() and (np.abs(pg[:S] - po) <= ep).all(), t
            np.testing.assert_array_equal(sg, oracle.sign(qg))
            q, p = qg, pg


def test_n8192_continued_segments_equal_one_run_and_the_group_api():
    """Two segments continued in place (q_init NULL) == one run of both
    schedules == the same instance as a one-member si_create_group; the exact
    readout of the run's own spins equals the oracle's energy."""
    import torch
    n, R, T = 8192, 512, 12
    dev = torch.device("cuda")
    J = inputs.pm1_coupling(n, seed=82)
    zeta = inputs.zeta_ramp(2000)[600:600 + 2 * T]
    dt = inputs.dt_const(2 * T)
    q0 = inputs.positions(n, R, seed0=8200)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        ctx.run_into(torch.from_numpy(zeta[:T]).to(dev), torch.from_numpy(dt[:T]).to(dev),
                     torch.from_numpy(q0).to(dev))
        q2, p2, s2 = ctx.run(zeta[T:], dt[T:], None)
        e2, c2, _ = ctx.energy(None)
    with b.Context(J, replicas=R, steps=2 * T, prec="j_fp8_q_bf16") as cx:
        q1, p1, s1 = cx.run(zeta, dt, q0)
    with b.Group([J], None, replicas=[R], steps=2 * T, precs=["j_fp8_q_bf16"]) as g:
        qg, pg, sg = g.run(zeta, dt, [q0])
    for a_, b_ in ((q2, q1), (p2, p1), (s2, s1), (q1, qg[0]), (p1, pg[0]), (s1, sg[0])):
        np.testing.assert_array_equal(a_, b_)
    sub = slice(0, 4)
    np.testing.assert_array_equal(e2[sub], oracle.energy(J, None, s2[sub]).astype(np.int64))
    np.testing.assert_array_equal(c2[sub], oracle.cut(J, s2[sub]).astype(np.int64))


def test_n32768_two_steps_against_the_oracle():
    """The scale workload's size: n = 32768 (J drawn on the device, kept as
    e4m3: 1 GiB), 16 replicas, two one-step calls, the second continuing in
    place; on two replicas each step against the FP64 oracle's step from the
    same state, within the bf16 bound; the exact cut of the GPU's spins
    against the oracle's."""
    import torch
    n, R, S = 32768, 16, 2
    dev = torch.device("cuda")
    Jd = inputs.pm1_coupling_torch(n, seed=11, device=dev)
    q0 = (inputs.positions(n, R, seed0=3200) * 4).astype(np.float32)
    zeta = inputs.zeta_ramp(5000)[2000:2002] * np.float32(np.sqrt(2000.0 / n))
    dt = inputs.dt_const(2)
    with b.Context(Jd, n=n, replicas=R, steps=1, prec="j_fp8_q_bf16") as ctx:
        desc = ctx.describe()
        q1, p1, _ = ctx.run(zeta[0:1], dt[0:1], q0)
        q2, p2, s2 = ctx.run(zeta[1:2], dt[1:2], None)
        _, c2, _ = ctx.energy(None)
        kw = params_f64(ctx)
    assert "grouped-step" in desc and "J=e4m3(1B)" in desc
    J = Jd.cpu().numpy()
    del Jd
    torch.cuda.empty_cache()
    for t, (qa, pa, qg, pg) in enumerate(((q0, np.zeros_like(q0), q1, p1), (q1, p1, q2, p2))):
        qs, ps = qa[:S], pa[:S]
        qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], qs, ps, **kw)
        eq, ep = bf16_step_bound(J, qs.astype(np.float64), ps.astype(np.float64), float(zeta[t]), float(dt[t]), kw)
        assert (np.abs(qg[:S] - qo) <= eq).all() and (np.abs(pg[:S] - po) <= ep).all(), t
    np.testing.assert_array_equal(s2, oracle.sign(q2))
    np.testing.assert_array_equal(c2[:S], oracle.cut(J, s2[:S]).astype(np.int64))
