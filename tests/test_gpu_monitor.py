"""GPU parity of si_hamiltonian (FP64 Hamiltonian for drift monitoring) and
of the schedule tuner running on si_grad."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle
from paper_2305_07187_gb300 import monitor, schedule

pytestmark = pytest.mark.gpu


def _scale(J, h, q, p, zeta, k, m, q0):
    """Sum of the magnitudes of H's terms per replica: the FP64 rounding scale."""
    s = (0.5 * p * p / m + 0.5 * k * (q - q0) ** 2).sum(1)
    s = s + 0.5 * abs(zeta) * ((np.abs(q) @ np.abs(J)) * np.abs(q)).sum(1)
    if h is not None:
        s = s + abs(zeta) * (np.abs(h) * np.abs(q)).sum(1)
    return s


@pytest.mark.parametrize("prec,kind,n,R,with_h", [
    ("fp32", "gauss", 300, 5, True),
    ("fp64", "gauss", 129, 3, True),
    ("j_bf16_q_bf16", "gauss", 513, 40, False),
    ("j_fp8_q_bf16", "pm1", 2000, 9, False),
])
def test_hamiltonian_matches_oracle(prec, kind, n, R, with_h):
    J = inputs.pm1_coupling(n, seed=51) if kind == "pm1" else inputs.gauss_coupling_bf16(n, seed=51)
    h = inputs.field(n, seed=52, scale=0.3) if with_h else None
    g = np.random.Generator(np.random.PCG64(53))
    q = g.uniform(-1.4, 1.4, (R, n)).astype(np.float32)
    p = g.uniform(-2, 2, (R, n)).astype(np.float32)
    kw = dict(k=0.7, m=1.3, q0=0.02)
    zeta = 0.37
    with b.Context(J, h, replicas=max(R, 1), steps=1, prec=prec, **kw) as c:
        H = c.hamiltonian(q, p, zeta)
    ref = oracle.hamiltonian(J.astype(np.float64), None if h is None else h.astype(np.float64),
                             q.astype(np.float64), p.astype(np.float64), zeta=zeta,
                             k=float(np.float32(0.7)), m=float(np.float32(1.3)), q0=float(np.float32(0.02)))
    tol = 1e-13 * _scale(J.astype(np.float64), h, q.astype(np.float64), p.astype(np.float64), zeta, 0.7, 1.3, 0.02)
    assert (np.abs(H - ref) <= tol).all(), np.abs(H - ref).max()


def test_hamiltonian_device_buffers_and_ragged_replica_counts():
    import torch
    n = 77
    J = inputs.gauss_coupling_bf16(n, seed=54)
    with b.Context(J, replicas=8, steps=1, prec="fp32") as c:
        for R in (0, 1, 4, 7, 13):
            g = np.random.Generator(np.random.PCG64(R))
            q = g.uniform(-1, 1, (R, n)).astype(np.float32)
            p = g.uniform(-1, 1, (R, n)).astype(np.float32)
            out = torch.empty(R, dtype=torch.float64, device="cuda")
            c.hamiltonian(torch.from_numpy(q).cuda(), torch.from_numpy(p).cuda(), 0.1, out=out)
            torch.cuda.synchronize()
            if R:
                ref = oracle.hamiltonian(J.astype(np.float64), None, q, p, zeta=0.1)
                np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)


def test_drift_monitor_bounded_below_the_walls():
    """N=2000 +-1 graph at constant zeta below the instability (zeta * 2
    sqrt(N) < k): H stays within a small band over 100 / 200 FP32 steps, the
    band shrinks with the step size (symplectic, first order), and the GPU's
    H series follows the oracle's FP64 run of the same schedule (the motion
    is linear and stable here, so FP32 and FP64 trajectories stay close)."""
    n, R = 2000, 2
    J = inputs.pm1_coupling(n, seed=1)
    q = inputs.positions(n, R, seed0=100)
    drifts = []
    for dt in (0.2, 0.1):
        T = int(round(20 / dt))
        with b.Context(J, replicas=R, steps=T, prec="fp32") as c:
            H, drift = monitor.hamiltonian_drift(c, 0.002, dt, q, segments=5)
        assert H.shape == (6, R)
        drifts.append(drift.max())
        qo, po = q.astype(np.float64), np.zeros((R, n))
        Ho = [oracle.hamiltonian(J, None, qo, po, zeta=0.002)]
        for _ in range(5):
            qo, po = oracle.run(J, None, np.full(T, 0.002), np.full(T, dt), qo, po)
            Ho.append(oracle.hamiltonian(J, None, qo, po, zeta=0.002))
        np.testing.assert_allclose(H, np.stack(Ho), rtol=1e-4)
    assert drifts[0] < 0.05
    assert 1.5 < drifts[0] / drifts[1] < 3.5


def test_tuned_schedule_lowers_the_relaxed_energy():
    n, R, T = 256, 16, 100
    J = inputs.pm1_coupling(n, seed=61)
    q = inputs.positions(n, R, seed0=6100)
    dt = inputs.dt_const(T)
    k0 = schedule.ramp_knots(5, 0.02, 0.25)
    with schedule.LibraryGrad(J, q, dt) as fn:
        res = schedule.tune_zeta(fn, k0, T, iters=8, lr=0.02)
        # the library gradient of the knots agrees with the oracle's
        W = schedule.knot_matrix(T, k0.size)
        L, gz = fn(schedule.expand(k0, T))
    Lo, gzo, _, _ = oracle.grad(J.astype(np.float64), None, schedule.expand(k0, T).astype(np.float64),
                                dt.astype(np.float64), q.astype(np.float64))
    np.testing.assert_allclose(W.T @ gz, W.T @ gzo, rtol=1e-3, atol=1e-3 * np.abs(W.T @ gzo).max())
    assert abs(L - Lo) <= 1e-4 * abs(Lo)
    assert res.objective < res.initial
