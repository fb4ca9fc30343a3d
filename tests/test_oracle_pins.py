"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's loops: each checks it against a
closed form, an exact invariant, a library routine computing the same quantity
by a different formula, or exhaustive enumeration, chosen so that a dropped
term, a wrong sign, a wrong index or a transposed operand fails at least one.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2305_07187_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ2 = math.sqrt(2.0)


def _linear_map(J, zeta_n, dt_n, k, m, order):
    """State-space matrix of one step of the unclamped iteration (Eq. 8 or
    Eq. 5), acting on z = (q, p) stacked, for a general (not necessarily
    symmetric) J.  Built from blocks with numpy; used to pin the oracle in the
    linear regime (no wall contact)."""
    n = J.shape[0]
    I = np.eye(n)
    G = -k * I + zeta_n * J            # dp/dt as a linear function of q
    if order == 0:
        # p' = p + dt G q ; q' = q + dt/m p'
        top = np.hstack([I + (dt_n * dt_n / m) * G, (dt_n / m) * I])
        bot = np.hstack([dt_n * G, I])
    else:
        # q' = q + dt/m p ; p' = p + dt G q
        top = np.hstack([I, (dt_n / m) * I])
        bot = np.hstack([dt_n * G, I])
    return np.vstack([top, bot])


# ---------------------------------------------------------------- integrator

@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("m", [1.0, 2.5])
def test_free_oscillator_matches_matrix_power(order, m):
    """J = 0, h = 0, no wall contact: q_n is the q-part of M^n z_0 exactly."""
    n, T, k, dt = 5, 40, 0.5, 0.2
    q0 = inputs.positions(n, 1, seed0=11)[0].astype(np.float64)
    J = np.zeros((n, n))
    zeta = np.full(T, 0.3)
    dts = np.full(T, dt)
    q, p = oracle.run(J, None, zeta, dts, q0[None], None, k=k, m=m, order=order)
    M = _linear_map(J, 0.3, dt, k, m, order)
    z = np.linalg.matrix_power(M, T) @ np.concatenate([q0, np.zeros(n)])
    np.testing.assert_allclose(q[0], z[:n], rtol=0, atol=1e-14)
    np.testing.assert_allclose(p[0], z[n:], rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [0, 1])
def test_linear_regime_general_J_matches_product_of_maps(order):
    """Coupled, unclamped dynamics with a NON-symmetric J and per-step zeta
    and dt: the oracle equals the ordered product of the one-step linear maps.
    A transposed J, a wrong zeta/dt index or a wrong sign fails this."""
    n, T, k, m = 6, 25, 0.5, 1.0
    g = np.random.Generator(np.random.PCG64(5))
    J = g.uniform(-1, 1, (n, n))
    np.fill_diagonal(J, 0.0)
    zeta = np.linspace(0.04, 0.5, T)
    dts = 0.05 + 0.2 * g.random(T)
    q0 = g.uniform(-0.01, 0.01, n)
    z = np.concatenate([q0, np.zeros(n)])
    for t in range(T):
        z = _linear_map(J, zeta[t], dts[t], k, m, order) @ z
    assert np.abs(z[:n]).max() < SQ2 and np.abs(z[n:]).max() < 2.0
    q, p = oracle.run(J, None, zeta, dts, q0[None], None, k=k, m=m, order=order)
    np.testing.assert_allclose(q[0], z[:n], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p[0], z[n:], rtol=1e-12, atol=1e-15)


def test_field_shifts_equilibrium():
    """J = 0, constant zeta, field h: the force -k q + zeta h has its
    equilibrium at q* = zeta h / k, and q - q* follows the free map M^n."""
    n, T, k, dt, z = 4, 30, 0.5, 0.2, 0.25
    h = np.array([0.3, -0.2, 0.1, 0.0])
    qs = z * h / k
    q0 = qs + np.array([0.05, -0.02, 0.0, 0.01])
    q, p = oracle.run(np.zeros((n, n)), h, np.full(T, z), np.full(T, dt),
                      q0[None], None, k=k)
    M = _linear_map(np.zeros((n, n)), 0.0, dt, k, 1.0, 0)
    zz = np.linalg.matrix_power(M, T) @ np.concatenate([q0 - qs, np.zeros(n)])
    np.testing.assert_allclose(q[0] - qs, zz[:n], atol=1e-14)


def test_spring_origin_q0():
    """J = 0, h = 0, spring origin c: q - c follows the free map."""
    n, T, k, dt, c = 3, 30, 0.5, 0.2, 0.3
    x0 = np.array([0.35, 0.25, 0.3])
    q, _ = oracle.run(np.zeros((n, n)), None, np.zeros(T), np.full(T, dt),
                      x0[None], None, k=k, q0=c)
    M = _linear_map(np.zeros((n, n)), 0.0, dt, k, 1.0, 0)
    zz = np.linalg.matrix_power(M, T) @ np.concatenate([x0 - c, np.zeros(n)])
    np.testing.assert_allclose(q[0] - c, zz[:n], atol=1e-14)


@pytest.mark.parametrize("m", [1.0, 2.0])
def test_kick_drift_invariant(m):
    """Symplectic Euler (order 0) conserves p^2/m + k q^2 - dt k q p / m
    exactly for the free spring (derived symbolically); FP64 drift ~1e-15."""
    n, T, k, dt = 8, 2000, 0.5, 0.2
    q0 = inputs.positions(n, 3, seed0=21).astype(np.float64)
    q, p = q0.copy(), np.zeros_like(q0)
    I0 = p ** 2 / m + k * q ** 2 - dt * k * q * p / m
    for _ in range(10):
        q, p = oracle.run(np.zeros((n, n)), None, np.zeros(T // 10),
                          np.full(T // 10, dt), q, p, k=k, m=m)
        I1 = p ** 2 / m + k * q ** 2 - dt * k * q * p / m
        np.testing.assert_allclose(I1, I0, rtol=1e-12)


def test_literal_euler_amplitude_growth():
    """Literal Eq. 5 (explicit Euler) multiplies k q^2 + p^2 by exactly
    (1 + dt^2 k) per step (m = 1) for the free spring."""
    n, T, k, dt = 4, 50, 0.5, 0.2
    q0 = np.array([[0.01, -0.02, 0.015, 0.0]])
    q, p = oracle.run(np.zeros((n, n)), None, np.zeros(T), np.full(T, dt),
                      q0, None, k=k, order=1)
    e0 = k * q0 ** 2
    e1 = k * q ** 2 + p ** 2
    np.testing.assert_allclose(e1, e0 * (1 + dt * dt * k) ** T, rtol=1e-12)


def test_first_order_convergence_to_cosine():
    """Continuous limit of the free spring: x(t) = x0 cos(sqrt(k/m) t).  The
    iteration is first order, so halving dt halves the error."""
    k, x0, t_end = 0.5, 0.1, 4.0
    errs = []
    for dt in (0.02, 0.01, 0.005):
        T = int(round(t_end / dt))
        q, _ = oracle.run(np.zeros((1, 1)), None, np.zeros(T), np.full(T, dt),
                          np.array([[x0]]), None, k=k)
        errs.append(abs(q[0, 0] - x0 * math.cos(math.sqrt(k) * t_end)))
    o1 = math.log2(errs[0] / errs[1])
    o2 = math.log2(errs[1] / errs[2])
    assert 0.9 < o1 < 1.1 and 0.9 < o2 < 1.1, (errs, o1, o2)


def test_one_step_golden_fixture():
    """Hand-worked one- and two-step examples (tests/golden/one_step_n2.json)."""
    with open(os.path.join(GOLDEN, "one_step_n2.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        q, p = oracle.run(np.array(case["J"]), None, case["zeta"], case["dt"],
                          np.array([case["q"]]), np.array([case["p"]]),
                          k=case["k"], m=case["m"], order=case["order"])
        np.testing.assert_allclose(q[0], case["q_out"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(p[0], case["p_out"], rtol=0, atol=1e-15)


def test_walls_hold_and_are_hit():
    """Eq. 6 and the constraints after Eq. 8: |q| <= sqrt 2, |p| <= 2 after
    every step, and a strongly coupled run reaches both walls."""
    n, R, T = 40, 4, 60
    J = inputs.pm1_coupling(n, seed=3).astype(np.float64)
    q = inputs.positions(n, R, seed0=300).astype(np.float64)
    p = np.zeros_like(q)
    zeta = np.full(T, 2.0)
    hit_q = hit_p = False
    for t in range(T):
        q, p = oracle.run(J, None, zeta[t:t + 1], [0.3], q, p)
        assert np.abs(q).max() <= SQ2 and np.abs(p).max() <= 2.0
        hit_q |= bool((np.abs(q) == SQ2).any())
        hit_p |= bool((np.abs(p) == 2.0).any())
    assert hit_q and hit_p


def test_inelastic_wall_zeroes_momentum():
    """wall_zero_p: a spin whose position was clipped this step has p = 0;
    without it, the clipped spin keeps its (clamped) momentum."""
    J = np.zeros((1, 1))
    q0, p0 = np.array([[1.40]]), np.array([[0.5]])
    q, p = oracle.run(J, None, [0.0], [0.2], q0, p0, k=0.0, wall_zero_p=True)
    assert q[0, 0] == SQ2 and p[0, 0] == 0.0
    q, p = oracle.run(J, None, [0.0], [0.2], q0, p0, k=0.0, wall_zero_p=False)
    assert q[0, 0] == SQ2 and p[0, 0] == 0.5


def test_negation_symmetry_bit_exact():
    """h = 0: (q, p) -> (-q, -p) negates the whole trajectory exactly."""
    n, R, T = 30, 3, 200
    J = inputs.pm1_coupling(n, seed=4).astype(np.float64)
    q0 = inputs.positions(n, R, seed0=400).astype(np.float64)
    z = inputs.zeta_ramp(T).astype(np.float64)
    d = inputs.dt_const(T).astype(np.float64)
    qa, pa = oracle.run(J, None, z, d, q0)
    qb, pb = oracle.run(J, None, z, d, -q0)
    assert np.array_equal(qa, -qb) and np.array_equal(pa, -pb)


def test_gauge_symmetry_bit_exact():
    """J -> D J D, q -> D q with D = diag(+-1) maps trajectories exactly."""
    n, R, T = 25, 2, 150
    J = inputs.pm1_coupling(n, seed=5).astype(np.float64)
    D = np.where(np.random.Generator(np.random.PCG64(9)).random(n) < 0.5, -1.0, 1.0)
    q0 = inputs.positions(n, R, seed0=500).astype(np.float64)
    z = inputs.zeta_ramp(T).astype(np.float64)
    d = inputs.dt_const(T).astype(np.float64)
    qa, pa = oracle.run(J, None, z, d, q0)
    qb, pb = oracle.run(D[:, None] * J * D[None, :], None, z, d, q0 * D)
    assert np.array_equal(qa * D, qb) and np.array_equal(pa * D, pb)


# ---------------------------------------------------------------- energy/cut

def _np_energy(J, h, s):
    """-1/2 s^T J s - h^T s, valid for symmetric zero-diagonal J."""
    s = s.astype(np.float64)
    e = -0.5 * np.einsum("ri,ij,rj->r", s, J, s)
    if h is not None:
        e -= s @ h
    return e


def test_energy_hand_examples():
    # Two spins, ferromagnetic J = 1: aligned -1, anti-aligned +1 (Eq. 1).
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    s = np.array([[1, 1], [1, -1], [-1, -1]], dtype=np.int8)
    np.testing.assert_array_equal(oracle.energy(J, None, s), [-1.0, 1.0, -1.0])
    # Field only: H = -sum h_i s_i.
    h = np.array([0.5, -2.0])
    np.testing.assert_array_equal(oracle.energy(np.zeros((2, 2)), h, s),
                                  [1.5, -2.5, -1.5])
    # Only the upper triangle enters Eq. 1 (sum over i < j).
    Ju = np.array([[0.0, 3.0], [100.0, 0.0]])
    np.testing.assert_array_equal(oracle.energy(Ju, None, s[:1]), [-3.0])


def test_energy_matches_quadratic_form():
    n, R = 50, 20
    J = inputs.gauss_coupling_bf16(n, seed=8).astype(np.float64)
    h = inputs.field(n).astype(np.float64)
    s = np.where(np.random.Generator(np.random.PCG64(3)).random((R, n)) < 0.5, -1, 1).astype(np.int8)
    np.testing.assert_allclose(oracle.energy(J, h, s), _np_energy(J, h, s), rtol=1e-12, atol=1e-9)
    np.testing.assert_array_equal(oracle.energy(J, None, s), oracle.energy(J, None, -s))


def test_ferromagnet_closed_form():
    """Complete graph with J_ij = 1: H = -(M^2 - n)/2 with M = sum s."""
    n = 13
    J = np.ones((n, n)) - np.eye(n)
    g = np.random.Generator(np.random.PCG64(1))
    s = np.where(g.random((30, n)) < 0.5, -1, 1).astype(np.int8)
    M = s.astype(np.int64).sum(axis=1)
    np.testing.assert_array_equal(oracle.energy(J, None, s), -(M * M - n) / 2.0)
    E, _ = oracle.bruteforce(J)
    assert E == -n * (n - 1) / 2


@pytest.mark.parametrize("n", [5, 8, 11])
def test_antiferromagnet_max_cut(n):
    """J_ij = -1 on K_n is MAX-CUT with unit weights: max cut = floor(n^2/4)."""
    J = -(np.ones((n, n)) - np.eye(n))
    E, s = oracle.bruteforce(J)
    assert oracle.cut(J, s[None])[0] == (n * n) // 4


def test_cut_identity_and_definition():
    """cut = sum_{i<j} w_ij (1 - s_i s_j)/2 with w = -J (numpy), and
    cut = -(sum_{i<j} J_ij + E)/2 at h = 0."""
    n, R = 60, 25
    J = inputs.pm1_coupling(n, seed=12).astype(np.float64)
    s = np.where(np.random.Generator(np.random.PCG64(2)).random((R, n)) < 0.5, -1, 1).astype(np.int8)
    c = oracle.cut(J, s)
    ss = s.astype(np.float64)
    w = -np.triu(J, 1)
    ref = np.einsum("ij,rij->r", w, (1 - ss[:, :, None] * ss[:, None, :]) / 2)
    np.testing.assert_array_equal(c, ref)
    E = oracle.energy(J, None, s)
    np.testing.assert_array_equal(c, -(np.triu(J, 1).sum() + E) / 2)


def test_bruteforce_against_itertools():
    n = 9
    J = inputs.gauss_coupling_bf16(n, seed=13).astype(np.float64)
    h = inputs.field(n, seed=14).astype(np.float64)
    states = np.array(list(itertools.product([-1, 1], repeat=n)), dtype=np.int8)
    Emin_ref = _np_energy(J, h, states).min()
    E, s = oracle.bruteforce(J, h)
    assert abs(E - Emin_ref) < 1e-9
    assert abs(_np_energy(J, h, s[None])[0] - E) < 1e-9


def test_relaxed_energy_and_hamiltonian():
    n, R = 20, 4
    J = inputs.gauss_coupling_bf16(n, seed=15).astype(np.float64)
    h = inputs.field(n, seed=16).astype(np.float64)
    g = np.random.Generator(np.random.PCG64(4))
    q = g.uniform(-1, 1, (R, n))
    p = g.uniform(-1, 1, (R, n))
    ref = -0.5 * np.einsum("ri,ij,rj->r", q, J, q) - q @ h
    np.testing.assert_allclose(oracle.relaxed_energy(J, h, q), ref, rtol=1e-12)
    s = np.sign(q).astype(np.int8)
    np.testing.assert_allclose(oracle.relaxed_energy(J, h, s.astype(np.float64)),
                               oracle.energy(J, h, s), rtol=1e-12)
    H = oracle.hamiltonian(J, h, q, p, zeta=0.3, k=0.5, m=2.0, q0=0.1)
    ref = (0.5 * p ** 2 / 2.0).sum(1) + (0.25 * (q - 0.1) ** 2).sum(1) + 0.3 * ref
    np.testing.assert_allclose(H, ref, rtol=1e-12)


def test_hamiltonian_generates_the_oracle_step():
    """Hamilton's equations pin H to the integrator (a different function of
    the oracle): one kick-drift step of length dt from (q, p) moves p by
    -dt dH/dq and then q by dt dH/dp at the new p.  dH/dq and dH/dp are taken
    by FP64 central differences of the oracle's H, the step from or_run, with
    walls far away; a dropped term, a wrong sign or a transposed J fails."""
    n, R = 12, 2
    J = inputs.gauss_coupling_bf16(n, seed=21).astype(np.float64)
    h = inputs.field(n, seed=22).astype(np.float64)
    g = np.random.Generator(np.random.PCG64(5))
    q = g.uniform(-0.3, 0.3, (R, n))
    p = g.uniform(-0.3, 0.3, (R, n))
    kw = dict(zeta=0.37, k=0.6, m=1.7, q0=0.05)
    eps = 1e-6
    dHdq = np.empty_like(q)
    dHdp1 = np.empty_like(p)
    dt = 1e-3
    q1, p1 = oracle.run(J, h, np.array([kw["zeta"]]), np.array([dt]), q, p, k=kw["k"], m=kw["m"],
                        q0=kw["q0"], q_max=10.0, p_max=10.0)
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        dHdq[:, i] = (oracle.hamiltonian(J, h, q + e, p, **kw) - oracle.hamiltonian(J, h, q - e, p, **kw)) / (2 * eps)
        dHdp1[:, i] = (oracle.hamiltonian(J, h, q, p1 + e, **kw) - oracle.hamiltonian(J, h, q, p1 - e, **kw)) / (2 * eps)
    np.testing.assert_allclose((p1 - p) / dt, -dHdq, rtol=0, atol=1e-7)
    np.testing.assert_allclose((q1 - q) / dt, dHdp1, rtol=0, atol=1e-7)


def test_hamiltonian_nearly_conserved_at_constant_zeta():
    """Symplectic Euler keeps H within O(dt) of its start with no secular
    drift at constant zeta: over 4000 steps, the spread at dt = 0.01 is about
    half that at dt = 0.02 and stays small (walls out of reach)."""
    n, R = 10, 2
    J = inputs.gauss_coupling_bf16(n, seed=23).astype(np.float64) * 0.05
    q = inputs.positions(n, R, seed0=300).astype(np.float64)
    spreads = []
    for dt in (0.02, 0.01):
        T = int(round(40.0 / dt))
        qc, pc = q.copy(), np.zeros_like(q)
        H0 = oracle.hamiltonian(J, None, qc, pc, zeta=0.2)
        worst = 0.0
        for _ in range(20):
            qc, pc = oracle.run(J, None, np.full(T // 20, 0.2), np.full(T // 20, dt), qc, pc,
                                q_max=10.0, p_max=10.0)
            worst = max(worst, np.abs(oracle.hamiltonian(J, None, qc, pc, zeta=0.2) - H0).max())
        spreads.append(worst / np.abs(H0).max())
    assert spreads[0] < 0.05
    assert 1.6 < spreads[0] / spreads[1] < 2.4


def test_sign_readout():
    q = np.array([0.5, -0.5, 0.0, -0.0, 1e-300, -1e-300])
    np.testing.assert_array_equal(oracle.sign(q), [1, -1, 1, 1, 1, -1])


def test_sia_never_beats_ground_state_and_usually_finds_it():
    """For small n the best-of-R energy of the iteration can never be below
    the exhaustive minimum, and with the paper's ramp it usually equals it."""
    found = 0
    trials = 6
    for seed in range(trials):
        n, R, T = 14, 32, 400
        J = inputs.pm1_coupling(n, seed=100 + seed).astype(np.float64)
        Emin, _ = oracle.bruteforce(J)
        q0 = inputs.positions(n, R, seed0=1000 * seed).astype(np.float64)
        q, _ = oracle.run(J, None, inputs.zeta_ramp(T), inputs.dt_const(T), q0)
        E = oracle.energy(J, None, oracle.sign(q))
        assert E.min() >= Emin - 1e-12
        found += int(E.min() == Emin)
    assert found >= trials - 2, found


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("order", [0, 1])
def test_reverse_mode_matches_central_differences(order):
    """The oracle's hand-derived adjoint agrees with FP64 central differences
    (small case, walls active for some spins)."""
    n, R, T = 6, 3, 30
    J = inputs.pm1_coupling(n, seed=31).astype(np.float64)
    h = inputs.field(n, seed=32, scale=0.1).astype(np.float64)
    q0 = inputs.positions(n, R, seed0=3100).astype(np.float64) * 2
    zeta = np.linspace(0.2, 0.3, T)
    dt = np.full(T, 0.25)
    obj, gz, gd, gk = oracle.grad(J, h, zeta, dt, q0, order=order)
    assert abs(obj - oracle.objective(J, h, zeta, dt, q0, order=order)) < 1e-12
    fd = oracle.fd_grad(J, h, zeta, dt, q0, eps=1e-6, order=order)
    scale = max(np.abs(fd["zeta"]).max(), np.abs(fd["dt"]).max(), abs(fd["k"]))
    np.testing.assert_allclose(gz, fd["zeta"], atol=1e-6 * scale)
    np.testing.assert_allclose(gd, fd["dt"], atol=1e-6 * scale)
    assert abs(gk - fd["k"]) < 1e-6 * scale
    # the walls must actually have been touched for this to test the masks
    qT, pT = oracle.run(J, h, zeta, dt, q0, order=order)
    assert (np.abs(qT) == SQ2).any() and not (np.abs(qT) == SQ2).all()
    assert abs(gk) > 1.0
