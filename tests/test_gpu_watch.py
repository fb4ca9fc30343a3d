"""si_run_watch: the run with the exact energy readout every E steps inside
the persistent step kernel, stopping at the first readout at which some
replica reaches the target energy.

The expected stop and state come from si_run itself, advanced segment by
segment (each segment continues from the last; a continued run equals one
run, and the multi-step launches equal chained oracle-checked single
steps), with si_energy of each segment's spins; the energies of the stopping
readout are pinned to the oracle's exact Eq. 1 energy of the final spins."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle

pytestmark = pytest.mark.gpu


def _case(n, R, T, seed, field=False):
    J = inputs.pm1_coupling(n, seed=seed)
    q0 = inputs.positions(n, R, seed0=10 * seed)
    zeta = inputs.zeta_ramp(T)
    dt = inputs.dt_const(T)
    h = None
    if field:
        h = np.random.default_rng(seed + 7).integers(-3, 4, size=n).astype(np.float32)
    return J, h, q0, zeta, dt


def _segments(J, h, q0, zeta, dt, every, prec):
    """si_run over segments of `every` steps (the last may be shorter):
    per segment (steps so far, q, p, spins, energies)."""
    T, (R, n) = len(zeta), q0.shape
    out, t = [], 0
    while t < T:
        L = min(every, T - t)
        with b.Context(J, h=h, replicas=R, steps=L, prec=prec) as c:
            if t == 0:
                q, p, s = c.run(zeta[:L], dt[:L], q0)
            else:
                q, p, s = c.run(zeta[t:t + L], dt[t:t + L], q_prev, p_prev)
            E, _, _ = c.energy(s)
        t += L
        out.append((t, q, p, s, E))
        q_prev, p_prev = q, p
    return out


@pytest.mark.parametrize("n,R,T,every,field,prec", [
    (2000, 256, 60, 10, False, "j_fp8_q_bf16"),
    (2001, 130, 45, 7, True, "j_fp8_q_bf16"),     # ragged n and R, a field, a last readout after 3 steps
    (300, 17, 20, 1, True, "j_bf16_q_bf16"),      # a readout after every step
])
def test_watch_without_a_hit_equals_si_run(n, R, T, every, field, prec):
    """A target no replica reaches: all T steps run, and q, p, spins equal
    si_run's bit for bit; the last readout's energies equal the oracle's."""
    J, h, q0, zeta, dt = _case(n, R, T, seed=3, field=field)
    with b.Context(J, h=h, replicas=R, steps=T, prec=prec) as c:
        q_r, p_r, s_r = c.run(zeta, dt, q0)
        done, q, p, s, E = c.run_watch(zeta, dt, q0, every, -10 ** 12)
        assert "tcgen05" in c.describe()
    assert done == T
    assert np.array_equal(q, q_r) and np.array_equal(p, p_r) and np.array_equal(s, s_r)
    assert np.array_equal(E, oracle.energy(J, h, s).astype(np.int32))


@pytest.mark.parametrize("n,R,T,every,field", [
    (2000, 256, 80, 10, False),
    (2001, 130, 45, 7, True),
])
def test_watch_stops_at_the_first_readout_that_reaches_the_target(n, R, T, every, field):
    """The target is the best energy of a middle readout: the run stops at
    the first readout whose best energy is at most that, with the state of
    that step (bit for bit the segmented run's) and its energies."""
    J, h, q0, zeta, dt = _case(n, R, T, seed=4, field=field)
    prec = "j_fp8_q_bf16"
    segs = _segments(J, h, q0, zeta, dt, every, prec)
    target = int(segs[len(segs) // 2][4].min())
    k_hit = next(k for k, sg in enumerate(segs) if int(sg[4].min()) <= target)
    t_hit, q_e, p_e, s_e, E_e = segs[k_hit]
    with b.Context(J, h=h, replicas=R, steps=T, prec=prec) as c:
        done, q, p, s, E = c.run_watch(zeta, dt, q0, every, target)
    assert done == t_hit
    assert np.array_equal(q, q_e) and np.array_equal(p, p_e) and np.array_equal(s, s_e)
    assert np.array_equal(E, E_e)
    assert np.array_equal(E, oracle.energy(J, h, s).astype(np.int32))
    assert int(E.min()) <= target


def test_watch_then_continue_equals_one_run():
    """After a stop, si_run with q_init NULL continues from the stopping
    state: watch (stopping at step d) + a continued run of T steps equals
    si_run over the schedules' first d steps followed by T more."""
    n, R, T, every = 2000, 128, 40, 10
    J, h, q0, zeta, dt = _case(n, R, T, seed=6)
    segs = _segments(J, h, q0, zeta, dt, every, "j_fp8_q_bf16")
    target = int(segs[1][4].min())
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as c:
        done, *_ = c.run_watch(zeta, dt, q0, every, target)
        q1, p1, s1 = c.run(zeta, dt, None)
    d = done
    assert d < T
    with b.Context(J, replicas=R, steps=d, prec="j_fp8_q_bf16") as ca:
        qa, pa, _ = ca.run(zeta[:d], dt[:d], q0)
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as cb:
        q2, p2, s2 = cb.run(zeta, dt, qa, pa)
    assert np.array_equal(q1, q2) and np.array_equal(p1, p2) and np.array_equal(s1, s2)


def test_watch_rejects_what_it_cannot_serve():
    n, R, T = 96, 4, 10
    J, h, q0, zeta, dt = _case(n, R, T, seed=8)
    with b.Context(J, replicas=R, steps=T, prec="fp32") as c:
        with pytest.raises(b.SpringIsingError):
            c.run_watch(zeta, dt, q0, 5, 0)
    Jg = (inputs.pm1_coupling(n, seed=8) * np.float32(0.5)).astype(np.float32)
    with b.Context(Jg, replicas=R, steps=T, prec="j_bf16_q_bf16") as c:
        with pytest.raises(b.SpringIsingError):
            c.run_watch(zeta, dt, q0, 5, 0)     # J not integer-valued
    with b.Context(J, replicas=R, steps=T, prec="j_fp8_q_bf16") as c:
        with pytest.raises(b.SpringIsingError):
            c.run_watch(zeta, dt, q0, 0, 0)     # every >= 1


def test_watch_at_the_batched_workload():
    """The time-to-target launch as the bench times it: N=2000 +-1, R=1024,
    the T=2000 schedule, a readout every 10 steps.  The target is the best
    energy at the fifth readout of the segmented run, so the watched run
    stops at the first readout (<= 5) that reaches it, with the segmented
    run's state and energies, and the oracle's exact energies of its spins."""
    n, R, T, every = 2000, 1024, 2000, 10
    J, h, q0, zeta, dt = _case(n, R, T, seed=2)
    prec = "j_fp8_q_bf16"
    segs, t = [], 0
    with b.Context(J, replicas=R, steps=every, prec=prec) as c:
        for k in range(5):
            if k == 0:
                q, p, s = c.run(zeta[:every], dt[:every], q0)
            else:
                q, p, s = c.run(zeta[t:t + every], dt[t:t + every], None)
            E, _, _ = c.energy(None)
            t += every
            segs.append((t, q, p, s, E))
    target = int(segs[4][4].min())
    k_hit = next(k for k, sg in enumerate(segs) if int(sg[4].min()) <= target)
    t_hit, q_e, p_e, s_e, E_e = segs[k_hit]
    with b.Context(J, replicas=R, steps=T, prec=prec) as c:
        done, q, p, s, E = c.run_watch(zeta, dt, q0, every, target)
        assert "tile=128x128" in c.describe()
    assert done == t_hit
    assert np.array_equal(q, q_e) and np.array_equal(p, p_e) and np.array_equal(s, s_e)
    assert np.array_equal(E, E_e)
    assert np.array_equal(E, oracle.energy(J, None, s).astype(np.int32))
