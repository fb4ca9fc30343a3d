"""The opt-in CTA-pair form of the persistent tensor-core kernel (two CTAs of
a cluster share each tcgen05 MMA of M = 256, SI_TC_PAIR=1) against the FP64
oracle per step (Eq. 8 with the walls of Eq. 6, within the bf16-operand
bound) and bit for bit against chained single-step launches, including the
full N=2000, R=1024, T=2000 launch.  Its K loop accumulates in another order
than the single-CTA kernel, so the two agree to rounding, not bit for bit."""
import numpy as np
import pytest

from _helpers import b, bf16_step_bound, inputs, oracle, params_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def pairs_on(monkeypatch):
    monkeypatch.setenv("SI_TC_PAIR", "1")


@pytest.mark.parametrize("n,R", [(300, 256), (2000, 130), (2001, 512)])
def test_pair_per_step_within_bf16_bound(n, R):
    J = inputs.pm1_coupling(n, seed=n + 11)
    T = 8
    zeta = inputs.zeta_ramp(T, start=0.04, end=0.5)
    dt = inputs.dt_const(T)
    q = inputs.positions(n, R, seed0=31)
    p = np.zeros_like(q)
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16") as ctx:
        assert "cta_pairs" in ctx.describe()
        kw = params_f64(ctx)
        for t in range(T):
            qg, pg, _ = ctx.run(zeta[t:t + 1], dt[t:t + 1], q, p)
            qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], q, p, **kw)
            eq, ep = bf16_step_bound(J, q.astype(np.float64), p.astype(np.float64), float(zeta[t]), float(dt[t]), kw)
            assert (np.abs(qg - qo) <= eq).all() and (np.abs(pg - po) <= ep).all(), "step %d" % t
            q, p = qg, pg


def _same(a, b_):
    for x, y in zip(a, b_):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("n,R,T", [(2001, 130, 33), (300, 256, 21)])
def test_pair_run_equals_chained_single_steps(n, R, T):
    J = inputs.pm1_coupling(n, seed=1)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q0 = (inputs.positions(n, R, seed0=4100) * 8).astype(np.float32)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "cta_pairs" in ctx.describe()
        full = ctx.run(zeta, dt, q0)
    q, p, s = q0, np.zeros_like(q0), None
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16") as c1:
        for t in range(T):
            q, p, s = c1.run(zeta[t:t + 1], dt[t:t + 1], q, p)
    _same(full, (q, p, s))
    assert (np.abs(full[0]) == b.SQRT2_F32).any()


def test_pair_full_workload_equals_chained_single_steps():
    import torch
    n, R, T = 2000, 1024, 2000
    dev = torch.device("cuda")
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "cta_pairs" in ctx.describe()
        full = ctx.run(zeta, dt, q0)
        e, c, _ = ctx.energy(full[2])
    np.testing.assert_array_equal(e, oracle.energy(J, None, full[2]).astype(np.int64))
    z_d, d_d = torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev)
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16") as c1:
        c1.run_into(z_d[0:1], d_d[0:1], torch.from_numpy(q0).to(dev))
        for t in range(1, T - 1):
            c1.run_into(z_d[t:t + 1], d_d[t:t + 1], None)
        chained = c1.run(zeta[T - 1:T], dt[T - 1:T], None)
    _same(full, chained)


@pytest.mark.parametrize("rank", [None, 0, 1])
def test_pair_stalled_wait_times_out_and_device_recovers(rank, monkeypatch):
    """A pair whose step wait runs out (SI_DEBUG_STALL_STEP) leaves the run
    with SI_ERR_TIMEOUT after every copy of both CTAs has landed on the even
    CTA's barriers; the context and the device stay usable.  With both CTAs
    stalled they have issued the same stages; with only the even CTA
    (rank 0) stalled the odd one has filled stages alone, which the even CTA
    arms at the end; with only the odd CTA (rank 1) stalled the even CTA has
    armed stages whose odd half never came, whose bytes it counts as done."""
    n, R, T = 300, 256, 12
    J = inputs.pm1_coupling(n, seed=4)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=40)
    monkeypatch.setenv("SI_DEBUG_STALL_STEP", "3")
    if rank is not None:
        monkeypatch.setenv("SI_DEBUG_STALL_RANK", str(rank))
    monkeypatch.setenv("SI_SPIN_LIMIT_NS", "200000000")
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "cta_pairs" in ctx.describe()
        for _ in range(2):
            with pytest.raises(b.SpringIsingError) as ei:
                ctx.run(zeta, dt, q0)
            assert ei.value.status == b.SI_ERR_TIMEOUT
    monkeypatch.delenv("SI_DEBUG_STALL_STEP")
    monkeypatch.delenv("SI_DEBUG_STALL_RANK", raising=False)
    monkeypatch.delenv("SI_SPIN_LIMIT_NS")
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "cta_pairs" in ctx.describe()
        q, p, s = ctx.run(zeta, dt, q0)
        e, _, _ = ctx.energy(s)
    assert np.abs(q).max() <= b.SQRT2_F32 and np.abs(p).max() <= 2.0
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
