"""Failure detection on the GPU without a GPU fault: at step
SI_DEBUG_STALL_STEP a step wait is left without its producer (the FP32 plain
path: the first CTA does not publish its tagged q words; the tensor path: the
wait is pointed at a count no CTA will publish), so the bounded wait must run
out; the call returns SI_ERR_TIMEOUT, the kernel ends on its own, and the
device stays usable for the next context."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,R", [("fp32", 1), ("j_fp8_q_bf16", 256)])
def test_stalled_wait_times_out_and_device_recovers(prec, R, monkeypatch):
    n, T = 300, 12
    J = inputs.pm1_coupling(n, seed=4)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=40)
    monkeypatch.setenv("SI_DEBUG_STALL_STEP", "3")
    monkeypatch.setenv("SI_SPIN_LIMIT_NS", "200000000")
    with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
        for _ in range(2):
            with pytest.raises(b.SpringIsingError) as ei:
                ctx.run(zeta, dt, q0)
            assert ei.value.status == b.SI_ERR_TIMEOUT
    monkeypatch.delenv("SI_DEBUG_STALL_STEP")
    monkeypatch.delenv("SI_SPIN_LIMIT_NS")
    with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
        q, p, s = ctx.run(zeta, dt, q0)
        e, _, _ = ctx.energy(s)
    assert np.abs(q).max() <= b.SQRT2_F32 and np.abs(p).max() <= 2.0
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))


@pytest.mark.parametrize("prec,R", [("fp32", 1), ("j_fp8_q_bf16", 256)])
def test_error_of_an_early_returning_run_surfaces_at_the_next_synchronising_call(prec, R, monkeypatch):
    """si_run with device inputs and no host output returns once its work is
    enqueued; the timed-out wait is then reported by si_synchronize, and the
    failed run leaves no spins to read out."""
    import torch
    n, T = 300, 12
    J = inputs.pm1_coupling(n, seed=5)
    z = torch.from_numpy(inputs.zeta_ramp(T)).cuda()
    d = torch.from_numpy(inputs.dt_const(T)).cuda()
    q = torch.from_numpy(inputs.positions(n, R, seed0=50)).cuda()
    monkeypatch.setenv("SI_DEBUG_STALL_STEP", "3")
    monkeypatch.setenv("SI_SPIN_LIMIT_NS", "200000000")
    with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
        ctx.run_into(z, d, q)
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.synchronize()
        assert ei.value.status == b.SI_ERR_TIMEOUT
        ctx.run_into(z, d, q)
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.get_state()                 # reports the pending error, not a half-written state
        assert ei.value.status == b.SI_ERR_TIMEOUT
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.energy(None)
        assert ei.value.status == b.SI_ERR_INVALID_ARG
        ctx.synchronize()   # nothing pending any more


@pytest.mark.parametrize("prec,R", [("fp32", 1), ("j_fp8_q_bf16", 256)])
def test_kernel_time_of_a_timed_out_run_reports_the_error(prec, R, monkeypatch):
    """si_last_kernel_time after an early-returning run whose wait ran out
    returns SI_ERR_TIMEOUT instead of the duration of the aborted kernel."""
    import torch
    n, T = 300, 12
    J = inputs.pm1_coupling(n, seed=6)
    z = torch.from_numpy(inputs.zeta_ramp(T)).cuda()
    d = torch.from_numpy(inputs.dt_const(T)).cuda()
    q = torch.from_numpy(inputs.positions(n, R, seed0=60)).cuda()
    monkeypatch.setenv("SI_DEBUG_STALL_STEP", "3")
    monkeypatch.setenv("SI_SPIN_LIMIT_NS", "200000000")
    with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
        ctx.enable_timing(True)
        ctx.run_into(z, d, q)
        with pytest.raises(b.SpringIsingError) as ei:
            ctx.last_kernel_ms()
        assert ei.value.status == b.SI_ERR_TIMEOUT
        ctx.synchronize()   # the error was reported once
