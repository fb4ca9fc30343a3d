"""The multi-step launches that the benchmarks time, pinned bit for bit to
chains of single-step launches.

The paper's iteration is one network pass applied again and again (Fig. 3;
Eq. 8 per time step), so T steps in one persistent launch must equal T calls
of one step each, every call starting from the previous call's outputs.  The
single-step calls are the ones the per-step parity tests compare with the
oracle (test_gpu_simt, test_gpu_tc, test_gpu_group), so these tests carry
that parity over to the launches whose time is reported: the persistent
tensor-core kernel (its dataflow exchange of the bf16 operand between CTAs
and the state kept in TMEM), the persistent FP32 matvec (its step-tagged
exchange words), the register-tiled FP32 kernel (its spin-major state) and
the captured graph of grouped steps.  A consumer that read the wrong operand
plane or a block published one step late would break bit equality.
"""
import numpy as np
import pytest

from _helpers import b, inputs

pytestmark = pytest.mark.gpu


def _wall_positions(n, R, seed):
    # amplitude large enough that some spins reach the walls within the run
    return (inputs.positions(n, R, seed0=seed) * 8).astype(np.float32)


def _chain_from_outputs(ctx1, zeta, dt, q, p):
    s = None
    for t in range(len(zeta)):
        q, p, s = ctx1.run(zeta[t:t + 1], dt[t:t + 1], q, p)
    return q, p, s


def _assert_same(a, b_, what):
    qa, pa, sa = a
    qb, pb, sb = b_
    np.testing.assert_array_equal(qa, qb, err_msg=what + ": q")
    np.testing.assert_array_equal(pa, pb, err_msg=what + ": p")
    np.testing.assert_array_equal(sa, sb, err_msg=what + ": spins")


@pytest.mark.parametrize("n,R,T,tile_n,e4", [(2000, 1024, 64, 0, 0), (2001, 130, 33, 64, 0), (2001, 130, 33, 128, 0),
                                             (300, 17, 21, 64, 0), (2001, 130, 33, 64, 1), (2001, 130, 33, 128, 1)])
def test_tc_run_equals_chained_single_steps(n, R, T, tile_n, e4, monkeypatch):
    """k_tc_run over T steps in one launch == T launches of one step each,
    restarted from the host outputs (both replica tiles, ragged n and R; also
    with the e4m3 J operand widened into tensor memory, e4=1)."""
    monkeypatch.setenv("SI_TC_J_E4M3", str(e4))
    J = inputs.pm1_coupling(n, seed=1)
    zeta = inputs.zeta_ramp(2000)[1000:1000 + T]   # the middle of the workload's ramp
    dt = inputs.dt_const(T)
    q0 = _wall_positions(n, R, 4100)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16", tile_n=tile_n) as ctx:
        desc = ctx.describe()
        full = ctx.run(zeta, dt, q0)
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16", tile_n=tile_n) as c1:
        assert c1.describe().split(" grid=")[0] == desc.split(" grid=")[0]
        chained = _chain_from_outputs(c1, zeta, dt, q0, np.zeros_like(q0))
    if tile_n:
        assert "tile=128x%d" % tile_n in desc
    _assert_same(full, chained, desc)
    assert (np.abs(full[0]) == b.SQRT2_F32).any()   # walls were reached


def test_tc_run_full_workload_equals_chained_single_steps():
    """The benchmarked launch itself: N=2000, R=1024, all T=2000 steps of the
    linear ramp in one k_tc_run launch == 2000 one-step launches chained on
    the device (continuing in place, which test_gpu_continue shows equal to
    restarting from the outputs)."""
    import torch
    n, R, T = 2000, 1024, 2000
    dev = torch.device("cuda")
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "tile=128x128" in ctx.describe()
        full = ctx.run(zeta, dt, q0)
    z_d, d_d = torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev)
    q_d = torch.from_numpy(q0).to(dev)
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16") as c1:
        c1.run_into(z_d[0:1], d_d[0:1], q_d)
        for t in range(1, T - 1):
            c1.run_into(z_d[t:t + 1], d_d[t:t + 1], None)
        chained = c1.run(zeta[T - 1:T], dt[T - 1:T], None)
    _assert_same(full, chained, "N=2000 R=1024 T=2000")


@pytest.mark.parametrize("n,R,T", [(2000, 1, 50), (2001, 3, 31), (129, 2, 17)])
def test_plain_fp32_equals_chained_single_steps(n, R, T):
    """k_plain<float> (R <= 4): step-tagged exchange words across CTAs."""
    J = inputs.pm1_coupling(n, seed=n)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q0 = _wall_positions(n, R, 4200)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as ctx:
        assert "plain_persistent" in ctx.describe()
        full = ctx.run(zeta, dt, q0)
    with b.Context(J, replicas=R, steps=1, prec="fp32") as c1:
        chained = _chain_from_outputs(c1, zeta, dt, q0, np.zeros_like(q0))
    _assert_same(full, chained, "plain n=%d R=%d" % (n, R))


def test_plain_fp32_full_workload_equals_chained_single_steps():
    """The FP32 plain workload launch (N=2000, R=1, T=1000) against 1000
    one-step launches continued in place."""
    import torch
    n, R, T = 2000, 1, 1000
    dev = torch.device("cuda")
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as ctx:
        full = ctx.run(zeta, dt, q0)
    z_d, d_d = torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev)
    with b.Context(J, replicas=R, steps=1, prec="fp32") as c1:
        c1.run_into(z_d[0:1], d_d[0:1], torch.from_numpy(q0).to(dev))
        for t in range(1, T - 1):
            c1.run_into(z_d[t:t + 1], d_d[t:t + 1], None)
        chained = c1.run(zeta[T - 1:T], dt[T - 1:T], None)
    _assert_same(full, chained, "plain N=2000 T=1000")


@pytest.mark.parametrize("n,R,T", [(300, 257, 23), (129, 130, 12)])
def test_tiled_fp32_equals_chained_single_steps(n, R, T):
    """k_tiled_f32 (R > 4): the spin-major state it keeps during a run."""
    J = inputs.pm1_coupling(n, seed=n + 5)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q0 = _wall_positions(n, R, 4300)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as ctx:
        assert "simt_tiled" in ctx.describe()
        full = ctx.run(zeta, dt, q0)
    with b.Context(J, replicas=R, steps=1, prec="fp32") as c1:
        chained = _chain_from_outputs(c1, zeta, dt, q0, np.zeros_like(q0))
    _assert_same(full, chained, "tiled n=%d R=%d" % (n, R))


@pytest.mark.parametrize("n,R", [(129, 3), (65, 9)])
def test_fp64_equals_chained_single_steps(n, R):
    """FP64 debug path (grid barrier / per-step tiles): chained in place so the
    double state never passes through float; compared through si_get_state."""
    T = 25
    J = inputs.pm1_coupling(n, seed=n + 6)
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    q0 = _wall_positions(n, R, 4400)
    with b.Context(J, replicas=R, steps=T, prec="fp64") as ctx:
        _, _, s_full = ctx.run(zeta, dt, q0)
        q_full, p_full = ctx.get_state()
    with b.Context(J, replicas=R, steps=1, prec="fp64") as c1:
        c1.run(zeta[0:1], dt[0:1], q0)
        s = None
        for t in range(1, T):
            _, _, s = c1.run(zeta[t:t + 1], dt[t:t + 1], None)
        q_ch, p_ch = c1.get_state()
    _assert_same((q_full, p_full, s_full), (q_ch, p_ch, s), "fp64 n=%d R=%d" % (n, R))


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4])
def test_grouped_graph_equals_chained_single_steps(policy, monkeypatch):
    """The captured graph of T grouped steps == T one-step group runs restarted
    from the outputs, over a mixed member list (+-1 and Gaussian, ragged n and
    R, both tile widths, split tiles), under every tile policy."""
    monkeypatch.setenv("SI_GROUP_POLICY", str(policy))
    members = [(17, 16, "pm1"), (128, 48, "gauss"), (300, 64, "pm1"), (513, 130, "gauss"),
               (1000, 200, "pm1"), (64, 1, "pm1"), (130, 300, "pm1")]
    Js, hs, qs = [], [], []
    for k, (n, R, kind) in enumerate(members):
        Js.append(inputs.pm1_coupling(n, seed=500 + k) if kind == "pm1"
                  else inputs.gauss_coupling_bf16(n, seed=500 + k))
        hs.append(inputs.field(n, seed=600 + k, scale=0.3) if kind == "gauss" else None)
        qs.append(_wall_positions(n, R, 4500 + 10 * k))
    precs = ["j_fp8_q_bf16" if kind == "pm1" else "j_bf16_q_bf16" for (_, _, kind) in members]
    Rs = [R for (_, R, _) in members]
    T = 17
    zeta = inputs.zeta_ramp(T, start=0.2, end=0.5)
    dt = inputs.dt_const(T)
    with b.Group(Js, hs, replicas=Rs, steps=T, precs=precs) as g:
        qf, pf, sf = g.run(zeta, dt, qs)
    q, p = qs, [np.zeros_like(x) for x in qs]
    with b.Group(Js, hs, replicas=Rs, steps=1, precs=precs) as g1:
        for t in range(T):
            q, p, s = g1.run(zeta[t:t + 1], dt[t:t + 1], q, p)
    for k in range(len(members)):
        _assert_same((qf[k], pf[k], sf[k]), (q[k], p[k], s[k]), "member %d policy %d" % (k, policy))
