"""GPU parity of the tcgen05 tensor-core path (J as bf16, q rounded to bf16
as the MMA operand, FP32 accumulation and state) against the FP64 oracle.

Tolerance, derived from the arithmetic: the operand rounding changes each
force by at most 2^-8 * S_i with S_i = sum_j |J_ij| |q_j| (round to nearest
bf16: 8 significant bits, unit roundoff 2^-8), FP32 accumulation of n products adds at most n * 2^-24 * S_i, the
update itself rounds a handful of FP32 operations, and the walls are
1-Lipschitz.  Every element must fall inside that bound; with bf16-exact
positions only the accumulation term remains.
"""
import numpy as np
import pytest

from _helpers import b, bf16_step_bound, inputs, oracle, params_f64, random_spins

pytestmark = pytest.mark.gpu


def _bound(J, q, p, zeta, dt, kw, bf16_term=True, h=None):
    return bf16_step_bound(J, q, p, zeta, dt, kw, bf16_term=bf16_term, h=h)


def _teacher_forced_tc(J, R, T, prec="j_fp8_q_bf16", bf16_exact=False, h=None, seed=5, tile_n=0):
    n = J.shape[0]
    zeta = inputs.zeta_ramp(T, start=0.04, end=0.5)
    dt = inputs.dt_const(T)
    q = inputs.positions(n, R, seed0=seed)
    p = np.zeros_like(q)
    worst = 0.0
    with b.Context(J, h, replicas=R, steps=1, prec=prec, tile_n=tile_n) as ctx:
        kw = params_f64(ctx)
        for t in range(T):
            if bf16_exact:
                q = inputs.round_to_bf16(q)
            qg, pg, _ = ctx.run(zeta[t:t + 1], dt[t:t + 1], q, p)
            qo, po = oracle.run(J, h, zeta[t:t + 1], dt[t:t + 1], q, p, **kw)
            eq, ep = _bound(J, q.astype(np.float64), p.astype(np.float64), float(zeta[t]), float(dt[t]), kw,
                            bf16_term=not bf16_exact, h=h)
            rq = np.abs(qg - qo) / np.maximum(eq, 1e-300)
            rp = np.abs(pg - po) / np.maximum(ep, 1e-300)
            worst = max(worst, rq.max(), rp.max())
            q, p = qg, pg
    return worst


@pytest.mark.parametrize("n,R", [(1, 1), (17, 3), (128, 16), (129, 17), (300, 64), (640, 100),
                                 (2000, 130), (2001, 15), (2001, 17)])
def test_tc_per_step_within_bf16_bound(n, R):
    J = inputs.pm1_coupling(n, seed=n)
    assert _teacher_forced_tc(J, R, T=12) <= 1.0


@pytest.mark.parametrize("n,R", [(200, 64), (2000, 256)])
def test_tc_bf16_exact_positions_accumulation_only(n, R):
    J = inputs.pm1_coupling(n, seed=2 * n)
    assert _teacher_forced_tc(J, R, T=8, bf16_exact=True) <= 1.0


def test_tc_gaussian_bf16_with_field():
    n, R = 333, 48
    J = inputs.gauss_coupling_bf16(n, seed=3)
    h = inputs.field(n, seed=4)
    assert _teacher_forced_tc(J, R, T=10, prec="j_bf16_q_bf16", h=h) <= 1.0


@pytest.mark.parametrize("tile_n", [64, 128])
def test_tc_both_tiles(tile_n):
    J = inputs.pm1_coupling(700, seed=9)
    assert _teacher_forced_tc(J, 200, T=6, tile_n=tile_n) <= 1.0


def test_tc_free_run_full_config():
    """N=2000, R=1024, T=2000 (the batched workload): walls hold, spins are
    sign(q), the exact energy/cut of the GPU spins equals the oracle's, and two
    late steps pass the per-step bound when restarted from the GPU state."""
    n, R, T = 2000, 1024, 2000
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        assert "tcgen05" in ctx.describe()
        q, p, s = ctx.run(zeta, dt, q0)
        e, c, _ = ctx.energy(s)
        kw = params_f64(ctx)
    assert np.abs(q).max() <= b.SQRT2_F32 and np.abs(p).max() <= 2.0
    np.testing.assert_array_equal(s, oracle.sign(q))
    sub = slice(0, 64)
    np.testing.assert_array_equal(e[sub], oracle.energy(J, None, s[sub]).astype(np.int64))
    np.testing.assert_array_equal(c[sub], oracle.cut(J, s[sub]).astype(np.int64))
    # energies are exact integers of the right parity and the cut identity holds
    s_upper = np.triu(J, 1).sum()
    np.testing.assert_array_equal(c.astype(np.int64), (-(s_upper + e.astype(np.int64)) // 2))
    assert np.median(c) > 0
    # restart two steps from the GPU's own state on a few replicas
    with b.Context(J, replicas=8, steps=1, prec="j_fp8_q_bf16") as ctx1:
        qq, pp = q[:8].copy(), p[:8].copy()
        for t in (T - 2, T - 1):
            qg, pg, _ = ctx1.run(zeta[t:t + 1], dt[t:t + 1], qq, pp)
            qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], qq, pp, **kw)
            eq, ep = _bound(J, qq.astype(np.float64), pp.astype(np.float64), float(zeta[t]), float(dt[t]), kw)
            assert (np.abs(qg - qo) <= eq).all() and (np.abs(pg - po) <= ep).all()
            qq, pp = qg, pg


def test_tc_negation_symmetry_and_determinism():
    n, R, T = 400, 96, 120
    J = inputs.pm1_coupling(n, seed=21)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=2100)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as ctx:
        qa, pa, sa = ctx.run(zeta, dt, q0)
        qb, pb, sb = ctx.run(zeta, dt, -q0)
        qc, pc, sc = ctx.run(zeta, dt, q0)
    assert np.array_equal(qa, -qb) and np.array_equal(pa, -pb) and np.array_equal(sa, -sb)
    assert np.array_equal(qa, qc) and np.array_equal(pa, pc)


def test_tc_energy_of_random_spins():
    n, R = 2000, 40
    J = inputs.pm1_coupling(n, seed=6)
    s = random_spins(R, n, seed=6)
    with b.Context(J, replicas=R, steps=1, prec="j_fp8_q_bf16") as ctx:
        e, c, f = ctx.energy(s)
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))


@pytest.mark.parametrize("n,R", [(17, 1), (300, 100), (2000, 1024), (3001, 130)])
def test_tensor_core_energy_readout_exact(n, R, monkeypatch):
    """Tensor-path contexts compute the exact energy on the tensor cores
    (sigma and integer J exact in bf16, integer sums below 2^24); it must
    equal the oracle and the dp4a readout bit for bit."""
    J = inputs.pm1_coupling(n, seed=n) * 3
    h = np.round(inputs.field(n, seed=n + 1) * 10).astype(np.float32)
    s = random_spins(R, n, seed=n + 2)
    with b.Context(J, h, replicas=1, steps=1, prec="j_bf16_q_bf16") as ctx:
        e, c, _ = ctx.energy(s)
        monkeypatch.setenv("SI_ENERGY_DP4A", "1")
        e2, c2, _ = ctx.energy(s)
        monkeypatch.delenv("SI_ENERGY_DP4A")
    np.testing.assert_array_equal(e, oracle.energy(J, h, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))
    np.testing.assert_array_equal(e, e2)
    np.testing.assert_array_equal(c, c2)
