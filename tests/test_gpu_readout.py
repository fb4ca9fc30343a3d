"""The exact energy readout fused into the persistent tensor-core kernel
(si_params.fused_readout = 1): after the last step the kernel runs one more
pass over J with sign(q(T)) as the operand and sums sigma^T J sigma per
replica, so that si_energy with spins NULL only finishes E of Eq. 1 and the
cut of Eq. 2.  The results must equal, bit for bit, the oracle's energy and
cut of the run's own spins and the separate tensor-core readout of the same
spins; continued segments must equal one run (the continuing run now starts
from the bf16 operand plane the previous run left)."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle

pytestmark = pytest.mark.gpu


def _int_field(n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-3, 4, size=n).astype(np.float32)


@pytest.mark.parametrize("n,R,T,with_h", [(2000, 1024, 40, False), (2001, 130, 17, True), (300, 17, 9, True),
                                          (129, 65, 5, False)])
def test_fused_readout_equals_oracle_and_separate_readout(n, R, T, with_h):
    J = inputs.pm1_coupling(n, seed=n + 3)
    h = _int_field(n, seed=n) if with_h else None
    zeta = inputs.zeta_ramp(T, start=0.1, end=0.5)
    dt = inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=77)
    with b.Context(J, h, replicas=R, steps=T, prec="j_fp8_q_bf16", fused_readout=1) as cf:
        qf, pf, sf = cf.run(zeta, dt, q0)
        ef, cf_cut, _ = cf.energy(None)
    with b.Context(J, h, replicas=R, steps=T, prec="j_fp8_q_bf16") as cs:
        qs, ps, ss = cs.run(zeta, dt, q0)
        es, cs_cut, _ = cs.energy(None)
    np.testing.assert_array_equal(qf, qs)
    np.testing.assert_array_equal(pf, ps)
    np.testing.assert_array_equal(sf, ss)
    np.testing.assert_array_equal(ef, es)
    np.testing.assert_array_equal(cf_cut, cs_cut)
    np.testing.assert_array_equal(ef, oracle.energy(J, h, sf).astype(np.int64))
    if h is None:
        np.testing.assert_array_equal(cf_cut, oracle.cut(J, sf).astype(np.int64))


def test_fused_readout_over_continued_segments_equals_one_run():
    n, R, seg, nseg = 2000, 1024, 10, 6
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(seg * nseg), inputs.dt_const(seg * nseg)
    q0 = inputs.positions(n, R, seed0=100)
    with b.Context(J, replicas=R, steps=seg * nseg, prec="j_fp8_q_bf16") as c1:
        q1, p1, s1 = c1.run(zeta, dt, q0)
    with b.Context(J, replicas=R, steps=seg, prec="j_fp8_q_bf16", fused_readout=1) as c:
        for k in range(nseg):
            sl = slice(k * seg, (k + 1) * seg)
            q, p, s = c.run(zeta[sl], dt[sl], q0 if k == 0 else None)
            e, cut, _ = c.energy(None)
            np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
            np.testing.assert_array_equal(cut, oracle.cut(J, s).astype(np.int64))
    np.testing.assert_array_equal(q, q1)
    np.testing.assert_array_equal(p, p1)
    np.testing.assert_array_equal(s, s1)


def test_fused_readout_switched_with_set_params():
    """Switched on and off with si_set_params between runs continued in place."""
    n, R, T = 300, 64, 12
    J = inputs.pm1_coupling(n, seed=9)
    zeta, dt = inputs.zeta_ramp(T, start=0.1, end=0.5), inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=5)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as c:
        c.run(zeta, dt, q0)
        for on in (1, 0, 1):
            c.set_params(fused_readout=on)
            _, _, s = c.run(zeta, dt, None)
            e, cut, _ = c.energy(None)
            np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
            np.testing.assert_array_equal(cut, oracle.cut(J, s).astype(np.int64))
