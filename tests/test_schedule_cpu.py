"""Host logic of the schedule tuner (knot interpolation, chain rule, the
projected Adam loop), driven by the FP64 oracle's gradient on the CPU."""
import numpy as np

import oracle
from paper_2305_07187_gb300 import inputs, schedule


def test_knot_matrix_reproduces_the_linear_ramp():
    for T, K in ((1, 2), (7, 2), (100, 5), (2000, 9), (33, 33)):
        W = schedule.knot_matrix(T, K)
        np.testing.assert_allclose(W.sum(1), 1.0, rtol=0, atol=1e-15)
        assert (W >= 0).all()
        z = schedule.expand(schedule.ramp_knots(K, inputs.ZETA_START, inputs.ZETA_END), T)
        np.testing.assert_allclose(z, inputs.zeta_ramp(T), rtol=0, atol=2e-7)
    # knots are hit exactly where they sit on a step
    W = schedule.knot_matrix(9, 5)
    np.testing.assert_array_equal(W[::2], np.eye(5))


def _problem():
    n, R, T = 12, 3, 40
    J = inputs.pm1_coupling(n, seed=41).astype(np.float64)
    q = inputs.positions(n, R, seed0=700).astype(np.float64)
    dt = np.full(T, 0.2)
    return J, q, dt, T


def test_knot_gradient_matches_finite_differences_of_the_objective():
    J, q, dt, T = _problem()
    knots = np.array([0.05, 0.2, 0.1, 0.3])
    W = schedule.knot_matrix(T, knots.size)
    _, gz, _, _ = oracle.grad(J, None, W @ knots, dt, q)
    gk = W.T @ gz
    eps = 1e-6
    fd = np.empty_like(knots)
    for k in range(knots.size):
        e = np.zeros_like(knots); e[k] = eps
        fd[k] = (oracle.objective(J, None, W @ (knots + e), dt, q)
                 - oracle.objective(J, None, W @ (knots - e), dt, q)) / (2 * eps)
    np.testing.assert_allclose(gk, fd, rtol=1e-5, atol=1e-8)


def test_tuner_lowers_the_objective_and_respects_bounds():
    J, q, dt, T = _problem()

    def grad_fn(z):
        L, gz, _, _ = oracle.grad(J, None, np.asarray(z, np.float64), dt, q)
        return L, gz

    k0 = schedule.ramp_knots(4, 0.04, 0.5)
    res = schedule.tune_zeta(grad_fn, k0, T, iters=15, lr=0.03, zeta_max=0.6)
    assert res.initial == res.history[0]
    assert res.objective <= min(res.history) + 1e-12
    assert res.objective < res.initial
    assert (res.knots >= 0).all() and (res.knots <= 0.6).all()


def test_transfer_scales_by_sqrt_of_size_ratio():
    k = np.array([0.04, 0.5])
    np.testing.assert_allclose(schedule.transfer(k, 2000, 8000), k / 2)
