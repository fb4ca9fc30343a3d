"""The persistent adjoint sweep (k_adj_run: one launch per segment, the
recomputation of segment s-1 beside the reverse sweep of segment s) against
the per-step sweep (one launch per product, SI_ADJOINT_PERSISTENT=0) and the
oracle's FP64 reverse mode.

Both sweeps compute every product, integrator step and adjoint step with
the same arithmetic, so the forward trajectory (hence the objective and the
final state) is equal bit for bit; the gradients differ only in the order
in which the per-step sums are added (per CTA slice instead of per block
of a grid-stride loop, both compensated), held to 1e-5 of the largest
component."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle, params_f64

pytestmark = pytest.mark.gpu


def _case(n, R, T, seed, field=False):
    J = inputs.pm1_coupling(n, seed=seed)
    q0 = inputs.positions(n, R, seed0=10 * seed)
    zeta = inputs.zeta_ramp(T)
    dt = inputs.dt_const(T)
    h = None
    if field:
        rng = np.random.default_rng(seed + 100)
        h = rng.integers(-2, 3, size=n).astype(np.float32)
    return J, h, q0, zeta, dt


def _rel(a, b_):
    a, b_ = np.asarray(a, np.float64), np.asarray(b_, np.float64)
    return np.abs(a - b_).max() / max(np.abs(b_).max(), 1e-30)


def _grad(J, h, q0, zeta, dt, K, env, monkeypatch):
    for k in ("SI_ADJOINT_PERSISTENT", "SI_ADJOINT_PAIR"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    n, R = q0.shape[1], q0.shape[0]
    with b.Context(J, h=h, replicas=R, steps=len(zeta), prec="fp32", ckpt_every=K) as ctx:
        res = ctx.grad(zeta, dt, q0)
        q, p = ctx.get_state()
        desc = ctx.describe()
    return res, q, p, desc


@pytest.mark.parametrize("n,R,T,K,field", [
    (2000, 64, 60, 10, False),    # the gradient workload's tiles and clusters, 6 segments
    (300, 70, 31, 10, True),      # two replica blocks, ragged n, R, last segment of 1 step, a field
    (120, 5, 47, 7, False),       # one M tile, clusters of 2
    (129, 64, 9, 1, False),       # one-step segments
    (2000, 64, 500, 50, False),   # the gradient workload itself (10 segments of 50)
])
def test_persistent_sweep_equals_per_step_sweep(n, R, T, K, field, monkeypatch):
    J, h, q0, zeta, dt = _case(n, R, T, seed=5, field=field)
    ref, qr, pr, dr = _grad(J, h, q0, zeta, dt, K, {"SI_ADJOINT_PERSISTENT": "0"}, monkeypatch)
    assert "sweep=per-step" in dr
    variants = [({}, "sweep=persistent"), ({"SI_ADJOINT_PAIR": "0"}, "sweep=persistent ")]
    for env, tag in variants:
        res, q, p, d = _grad(J, h, q0, zeta, dt, K, env, monkeypatch)
        assert tag in d + " ", d
        assert res[0] == ref[0]
        assert np.array_equal(q, qr) and np.array_equal(p, pr)
        scale = max(np.abs(ref[2]).max(), abs(ref[3]))
        assert _rel(res[1], ref[1]) <= 1e-5 and _rel(res[2], ref[2]) <= 1e-5
        assert abs(res[3] - ref[3]) <= 1e-5 * scale


def test_persistent_sweep_pairs_at_the_workload_shape():
    """At N=2000, R=64 the recomputation and the reverse sweep run side by
    side (asserted through si_describe); R=4, T=20 against the oracle's FP64
    reverse mode at the FP32 bar, g_k included."""
    n, R, T = 2000, 4, 20
    J, h, q0, zeta, dt = _case(n, R, T, seed=1)
    with b.Context(J, replicas=64, steps=T, prec="fp32", ckpt_every=10) as cw:
        cw.grad(zeta, dt, inputs.positions(n, 64, seed0=10))
        assert "sweep=persistent-side-by-side" in cw.describe()
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=10) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        assert "sweep=persistent" in ctx.describe()
        kw = params_f64(ctx)
    kw.pop("wall_zero_p")
    o_obj, o_gz, o_gd, o_gk = oracle.grad(J, None, zeta, dt, q0, **kw)
    assert abs(obj - o_obj) <= 1e-4 * abs(o_obj)
    assert _rel(gz, o_gz) <= 1e-3 and _rel(gd, o_gd) <= 1e-3
    assert abs(gk - o_gk) <= 1e-3 * max(abs(o_gk), np.abs(o_gd).max())


def test_persistent_sweep_repeats_bit_for_bit():
    """Two calls (the second replays the captured graph) give the same
    gradient bit for bit: the per-CTA partials are added in a fixed order."""
    n, R, T = 2000, 64, 40
    J, h, q0, zeta, dt = _case(n, R, T, seed=2)
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=10) as ctx:
        r1 = ctx.grad(zeta, dt, q0)
        r2 = ctx.grad(zeta, dt, q0)
    assert r1[0] == r2[0] and r1[3] == r2[3]
    assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
