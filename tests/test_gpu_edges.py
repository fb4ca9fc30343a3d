"""Degenerate and boundary cases of the newer entry points: a gradient over
zero steps, a one-spin group member, a group of a single replica, and a
Hamiltonian of an all-zero state."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle, random_spins

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_grad_over_zero_steps(prec):
    n, R = 50, 3
    J = inputs.pm1_coupling(n, seed=31)
    q0 = inputs.positions(n, R, seed0=3100)
    with b.Context(J, replicas=R, steps=0, prec=prec) as c:
        obj, gz, gd, gk = c.grad(np.zeros(0, np.float32), np.zeros(0, np.float32), q0)
    assert gz.size == 0 and gd.size == 0 and gk == 0.0
    ref = oracle.relaxed_energy(J, None, q0.astype(np.float64)).sum()
    assert abs(obj - ref) <= 1e-5 * abs(ref)


def test_group_with_one_spin_and_one_replica_members():
    Js = [np.zeros((1, 1), np.float32), inputs.pm1_coupling(40, seed=32), inputs.pm1_coupling(3, seed=33)]
    Rs = [5, 1, 16]
    qs = [inputs.positions(J.shape[0], R, seed0=3200 + k) for k, (J, R) in enumerate(zip(Js, Rs))]
    T = 3
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    p0 = b.default_params()
    kw = dict(k=float(p0.k), m=float(p0.m), q0=float(p0.q0), q_max=float(np.float32(p0.q_max)), p_max=float(p0.p_max))
    with b.Group(Js, None, replicas=Rs, steps=T, precs="j_fp8_q_bf16") as g:
        qg, pg, sg = g.run(zeta, dt, qs)
        for k in range(len(Js)):
            qo, po = oracle.run(Js[k], None, zeta, dt, qs[k], **kw)
            np.testing.assert_allclose(qg[k], qo, rtol=0, atol=1e-3)
            np.testing.assert_array_equal(sg[k], oracle.sign(qg[k]))
            e, c, _ = g.energy(k, sg[k])
            np.testing.assert_array_equal(e, oracle.energy(Js[k], None, sg[k]).astype(np.int64))
    # the one-spin member is a free spring: q follows the oracle closely
    np.testing.assert_allclose(qg[0], oracle.run(Js[0], None, zeta, dt, qs[0], **kw)[0], rtol=0, atol=1e-6)


def test_hamiltonian_of_zero_state_is_zero():
    n, R = 33, 4
    J = inputs.gauss_coupling_bf16(n, seed=34)
    with b.Context(J, replicas=R, steps=1, prec="fp32", q0=0.0) as c:
        H = c.hamiltonian(np.zeros((R, n), np.float32), np.zeros((R, n), np.float32), 0.7)
    assert (H == 0.0).all()


@pytest.mark.parametrize("prec,n,R", [("fp32", 130, 3), ("fp32", 77, 9), ("j_fp8_q_bf16", 300, 70)])
def test_energy_of_the_last_run_without_passing_spins(prec, n, R):
    """si_energy with spins NULL reads the sign readout of the last si_run
    (also for a run of zero steps); it is refused before any run and after a
    gradient sweep, which replaces the state."""
    J = inputs.pm1_coupling(n, seed=35)
    q0 = inputs.positions(n, R, seed0=3500)
    for T in (5, 0):
        with b.Context(J, replicas=R, steps=T, prec=prec) as c:
            with pytest.raises(b.SpringIsingError):
                c.energy(None)
            _, _, s = c.run(inputs.zeta_ramp(T), inputs.dt_const(T), q0)
            e0, c0, f0 = c.energy(s)
            e1, c1, f1 = c.energy(None)
            np.testing.assert_array_equal(e1, e0)
            np.testing.assert_array_equal(c1, c0)
            np.testing.assert_array_equal(e1, oracle.energy(J, None, s).astype(np.int64))
            if prec == "fp32" and T > 0:
                c.grad(inputs.zeta_ramp(T), inputs.dt_const(T), q0)
                with pytest.raises(b.SpringIsingError):
                    c.energy(None)


def test_energy_of_the_last_run_around_other_readouts():
    """On the tensor path the last run's step kernel also leaves its sign
    readout as the exact readout's bf16 operand.  Readouts of other spins in
    between (more replicas than the context's too) and continued runs must
    not disturb si_energy with spins NULL."""
    n, R, T = 300, 70, 6
    J = inputs.pm1_coupling(n, seed=36)
    q0 = inputs.positions(n, R, seed0=3600)
    z, d = inputs.zeta_ramp(T), inputs.dt_const(T)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as c:
        _, _, s1 = c.run(z, d, q0)
        e1, c1, _ = c.energy(None)                     # straight after the run
        other = random_spins(2 * R + 7, n, seed=37)
        eo, co, _ = c.energy(other)
        e2, c2, _ = c.energy(None)                     # after a readout of other spins
        _, _, s3 = c.run(z, d, None)
        e3, c3, _ = c.energy(None)
    ref1 = oracle.energy(J, None, s1).astype(np.int64)
    np.testing.assert_array_equal(e1, ref1)
    np.testing.assert_array_equal(e2, ref1)
    np.testing.assert_array_equal(c1, oracle.cut(J, s1).astype(np.int64))
    np.testing.assert_array_equal(c2, c1)
    np.testing.assert_array_equal(eo, oracle.energy(J, None, other).astype(np.int64))
    np.testing.assert_array_equal(co, oracle.cut(J, other).astype(np.int64))
    np.testing.assert_array_equal(e3, oracle.energy(J, None, s3).astype(np.int64))
    np.testing.assert_array_equal(c3, oracle.cut(J, s3).astype(np.int64))


@pytest.mark.parametrize("prec,n,R", [("fp32", 130, 3), ("fp32", 77, 9), ("j_fp8_q_bf16", 300, 70)])
def test_early_returning_calls_give_the_synchronous_results(prec, n, R):
    """si_run and si_energy with device data only return before their work
    has finished; after si_synchronize their outputs equal those of the same
    calls with host outputs."""
    import torch
    T = 7
    J = inputs.pm1_coupling(n, seed=38)
    z, d = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=3800)
    with b.Context(J, replicas=R, steps=T, prec=prec) as c:
        zd, dd, qd = (torch.from_numpy(x).cuda() for x in (z, d, q0))
        qo = torch.empty((R, n), dtype=torch.float32, device="cuda")
        so = torch.empty((R, n), dtype=torch.int8, device="cuda")
        eo = torch.empty(R, dtype=torch.int32, device="cuda")
        co = torch.empty(R, dtype=torch.int32, device="cuda")
        c.run_into(zd, dd, qd, None, qo, None, so)
        c.energy_into(None, R, eo, co, None)
        c.synchronize()
        q_h, _, s_h = c.run(z, d, q0)
        e_h, c_h, _ = c.energy(s_h)
    np.testing.assert_array_equal(qo.cpu().numpy(), q_h)
    np.testing.assert_array_equal(so.cpu().numpy(), s_h)
    np.testing.assert_array_equal(eo.cpu().numpy(), e_h)
    np.testing.assert_array_equal(co.cpu().numpy(), c_h)


@pytest.mark.parametrize("prec,R", [("fp32", 1), ("j_fp8_q_bf16", 256)])
def test_pinned_host_schedule_may_be_reused_once_the_call_returns(prec, R):
    """si_run with a host input returns only after its work has finished, so
    a pinned schedule may be overwritten as soon as the call returns: queue a
    long run first (device arguments only, returns early), then a run whose
    zeta and dt are pinned host memory and whose outputs are device memory,
    overwrite zeta and dt at once, and compare with a synchronous run."""
    import torch
    dev = torch.device("cuda")
    n, T = 2000, 2000
    J = inputs.pm1_coupling(n, seed=36)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=3600)
    with b.Context(J, replicas=R, steps=T, prec=prec) as c:
        q_ref, p_ref, s_ref = c.run(zeta, dt, q0)
        z_d, d_d, q_d = (torch.from_numpy(x).to(dev) for x in (zeta, dt, q0))
        z_h, d_h = torch.from_numpy(zeta.copy()).pin_memory(), torch.from_numpy(dt.copy()).pin_memory()
        qo = torch.empty((R, n), dtype=torch.float32, device=dev)
        po, so = torch.empty_like(qo), torch.empty((R, n), dtype=torch.int8, device=dev)
        c.run_into(z_d, d_d, q_d)                       # long, returns once enqueued
        c.run_into(z_h, d_h, q_d, None, qo, po, so)     # host inputs: returns when done
        z_h.fill_(123.0)
        d_h.fill_(-7.0)
        c.synchronize()
        torch.cuda.synchronize()
    np.testing.assert_array_equal(qo.cpu().numpy(), q_ref)
    np.testing.assert_array_equal(po.cpu().numpy(), p_ref)
    np.testing.assert_array_equal(so.cpu().numpy(), s_ref)
