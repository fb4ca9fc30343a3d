"""GPU parity of the FP32 / FP64 CUDA-core paths and of the exact energy
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from _helpers import TOL_FP64_100, b, inputs, normwise_rel, oracle, params_f64, random_spins, teacher_forced

pytestmark = pytest.mark.gpu

TOL_FP32_STEP = 1e-6     # per-step normwise relative, FP32 plain path


@pytest.mark.parametrize("n,R", [(1, 1), (17, 1), (127, 2), (129, 3), (300, 4),
                                 (2000, 1), (2001, 1), (5, 5), (70, 17), (130, 64), (257, 100),
                                 (2001, 15), (2001, 16), (300, 130), (129, 257)])
def test_fp32_per_step_teacher_forced(n, R):
    J = inputs.pm1_coupling(n, seed=n)
    T = 40
    zeta = inputs.zeta_ramp(T, start=0.04, end=0.5)
    dt = inputs.dt_const(T)
    q = inputs.positions(n, R, seed0=7 * n)
    p = np.zeros_like(q)
    with b.Context(J, n=n, replicas=R, steps=1, prec="fp32") as ctx:
        worst, q, p = teacher_forced(ctx, J, None, zeta, dt, q, p, range(T))
    assert worst <= TOL_FP32_STEP, worst


def test_fp32_gaussian_with_field_and_options():
    n, R, T = 150, 6, 25
    J = inputs.gauss_coupling_bf16(n, seed=5)
    h = inputs.field(n, seed=6)
    zeta = np.linspace(0.2, 0.6, T).astype(np.float32)
    dt = np.full(T, 0.15, np.float32)
    q = inputs.positions(n, R, seed0=50) * 5
    p = np.zeros_like(q)
    for order in (0, 1):
        with b.Context(J, h, replicas=R, steps=1, prec="fp32", update_order=order,
                       k=0.7, m=1.5, q0=0.05) as ctx:
            worst, _, _ = teacher_forced(ctx, J, h, zeta, dt, q, p, range(T))
        assert worst <= TOL_FP32_STEP, (order, worst)


@pytest.mark.parametrize("n,R", [(64, 1), (64, 9), (129, 3)])
def test_fp64_debug_100_steps(n, R):
    """FP64 debug mode, 100 free-running steps, normwise relative <= 1e-10."""
    T = 100
    J = inputs.pm1_coupling(n, seed=11)
    zeta = inputs.zeta_ramp(T)
    dt = inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=1100)
    with b.Context(J, replicas=R, steps=T, prec="fp64") as ctx:
        _, _, sg = ctx.run(zeta, dt, q0)
        qg, pg = ctx.get_state()
        kw = params_f64(ctx)
    qo, po = oracle.run(J, None, zeta, dt, q0, **kw)
    assert normwise_rel(qg, pg, qo, po) <= TOL_FP64_100
    np.testing.assert_array_equal(sg, oracle.sign(qo))


@pytest.mark.parametrize("n,R", [(1, 1), (2, 3), (17, 9), (100, 16), (2000, 33)])
def test_exact_energy_and_cut(n, R):
    J = inputs.pm1_coupling(n, seed=n + 1)
    s = random_spins(R, n, seed=n)
    with b.Context(J, replicas=1, steps=0) as ctx:
        e, c, f = ctx.energy(s)
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))
    np.testing.assert_allclose(f, oracle.energy(J, None, s), rtol=0, atol=1e-3 * max(1, n))


def test_exact_energy_integer_field():
    n, R = 90, 10
    J = inputs.pm1_coupling(n, seed=3) * 3
    h = np.round(inputs.field(n, seed=4) * 10).astype(np.float32)
    s = random_spins(R, n, seed=8)
    with b.Context(J, h) as ctx:
        e, c, _ = ctx.energy(s)
    np.testing.assert_array_equal(e, oracle.energy(J, h, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))


def test_float_energy_gaussian():
    n, R = 300, 7
    J = inputs.gauss_coupling_bf16(n, seed=9)
    h = inputs.field(n, seed=10)
    s = random_spins(R, n, seed=11)
    with b.Context(J, h) as ctx:
        with pytest.raises(b.SpringIsingError):
            ctx.energy(s, exact=True)
        _, _, f = ctx.energy(s, exact=False)
    ref = oracle.energy(J, h, s)
    bound = 1e-5 * (np.abs(J).sum() + np.abs(h).sum())
    np.testing.assert_allclose(f, ref, rtol=0, atol=bound)


def test_full_size_plain_fp32_run():
    """The N=2000, R=1, T=1000 plain run: walls hold, the final energy is the
    oracle's exact energy of the GPU's own spins, and sampled steps of the
    GPU trajectory pass the per-step parity check."""
    n, R, T = 2000, 1, 1000
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as ctx:
        assert "plain_persistent" in ctx.describe()
        q, p, s = ctx.run(zeta, dt, q0)
        e, c, _ = ctx.energy(s)
    assert np.abs(q).max() <= b.SQRT2_F32 and np.abs(p).max() <= 2.0
    np.testing.assert_array_equal(s, oracle.sign(q))
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))
    assert c[0] > 0
    # per-step parity on steps sampled along a GPU trajectory (late steps)
    with b.Context(J, replicas=R, steps=1) as ctx1:
        worst, _, _ = teacher_forced(ctx1, J, None, zeta, dt, q, p, range(T - 5, T))
    assert worst <= TOL_FP32_STEP


def test_negation_and_gauge_symmetry_bit_exact():
    n, R, T = 200, 3, 150
    J = inputs.pm1_coupling(n, seed=21)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=2100)
    D = np.where(np.random.Generator(np.random.PCG64(1)).random(n) < 0.5, -1, 1).astype(np.float32)
    for prec in ("fp32", "fp64"):
        with b.Context(J, replicas=R, steps=T, prec=prec) as ctx:
            qa, pa, sa = ctx.run(zeta, dt, q0)
            qb, pb, sb = ctx.run(zeta, dt, -q0)
        assert np.array_equal(qa, -qb) and np.array_equal(pa, -pb) and np.array_equal(sa, -sb)
        with b.Context(D[:, None] * J * D[None, :], replicas=R, steps=T, prec=prec) as ctx:
            qc, pc, _ = ctx.run(zeta, dt, q0 * D)
        assert np.array_equal(qa * D, qc) and np.array_equal(pa * D, pc)


def test_determinism_and_host_device_pointers():
    import torch
    n, R, T = 500, 8, 60
    J = inputs.pm1_coupling(n, seed=31)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=3100)
    with b.Context(J, replicas=R, steps=T) as ctx:
        q1, p1, s1 = ctx.run(zeta, dt, q0)
        q2, p2, s2 = ctx.run(zeta, dt, q0)
        dev = torch.device("cuda")
        qd = torch.empty((R, n), dtype=torch.float32, device=dev)
        pd = torch.empty_like(qd)
        sd = torch.empty((R, n), dtype=torch.int8, device=dev)
        ctx.run_into(torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev),
                     torch.from_numpy(q0).to(dev), None, qd, pd, sd)
        torch.cuda.synchronize()
    assert np.array_equal(q1, q2) and np.array_equal(p1, p2) and np.array_equal(s1, s2)
    assert np.array_equal(q1, qd.cpu().numpy()) and np.array_equal(s1, sd.cpu().numpy())


def test_zero_steps_gives_initial_spins():
    n, R = 33, 2
    J = inputs.pm1_coupling(n, seed=2)
    q0 = inputs.positions(n, R, seed0=1)
    q0[0, 0] = 0.0
    with b.Context(J, replicas=R, steps=0) as ctx:
        q, p, s = ctx.run(np.zeros(0, np.float32), np.zeros(0, np.float32), q0)
    np.testing.assert_array_equal(q, q0)
    np.testing.assert_array_equal(s, oracle.sign(q0))


def test_invalid_inputs_rejected():
    n = 10
    J = inputs.pm1_coupling(n, seed=1)
    Ja = J.copy(); Ja[0, 1] = 3.0
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(Ja)
    assert ei.value.status == b.SI_ERR_NOT_SYMMETRIC
    Jd = J.copy(); Jd[2, 2] = 1.0
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(Jd)
    assert ei.value.status == b.SI_ERR_NOT_SYMMETRIC
    Jn = J.copy(); Jn[0, 1] = Jn[1, 0] = np.nan
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(Jn)
    assert ei.value.status == b.SI_ERR_INVALID_ARG
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(J, m=0.0)
    assert ei.value.status == b.SI_ERR_INVALID_ARG
    Jg = inputs.gauss_coupling_bf16(n, seed=1)
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(Jg, prec="j_fp8_q_bf16")
    assert ei.value.status == b.SI_ERR_INVALID_ARG
