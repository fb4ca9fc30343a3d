"""GPU adjoint (si_grad) against the oracle's FP64 reverse mode and FP64
central finite differences, through the C ABI."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle, params_f64

pytestmark = pytest.mark.gpu


def _case(n, R, T, seed, scale=1.0):
    J = inputs.pm1_coupling(n, seed=seed)
    q0 = inputs.positions(n, R, seed0=10 * seed) * scale
    zeta = inputs.zeta_ramp(T)
    dt = inputs.dt_const(T)
    return J, q0, zeta, dt


def _rel(a, b_):
    a, b_ = np.asarray(a, np.float64), np.asarray(b_, np.float64)
    return np.abs(a - b_).max() / max(np.abs(b_).max(), 1e-30)


@pytest.mark.parametrize("n,R,T,K", [(64, 4, 100, 50), (33, 7, 61, 8), (64, 1, 40, 40)])
def test_fp64_adjoint_matches_oracle_reverse_mode(n, R, T, K):
    J, q0, zeta, dt = _case(n, R, T, seed=n)
    with b.Context(J, replicas=R, steps=T, prec="fp64", ckpt_every=K) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        kw = params_f64(ctx)
    kw.pop("wall_zero_p")
    o_obj, o_gz, o_gd, o_gk = oracle.grad(J, None, zeta, dt, q0, **kw)
    # outputs are float32: compare at float32 resolution of the largest entry
    assert abs(obj - o_obj) <= 1e-6 * abs(o_obj)
    assert _rel(gz, o_gz) <= 1e-6 and _rel(gd, o_gd) <= 1e-6
    assert abs(gk - o_gk) <= 1e-6 * max(abs(o_gk), np.abs(o_gd).max())


def test_fp64_adjoint_against_central_differences():
    """FP64 central differences of the FP64 oracle at n=64 on a sample of
    components: relative error <= 1e-4 (components whose wall pattern changes
    within +-eps are excluded, as the clamp makes the objective non-smooth)."""
    n, R, T = 64, 4, 60
    J, q0, zeta, dt = _case(n, R, T, seed=5)
    with b.Context(J, replicas=R, steps=T, prec="fp64") as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        kw = params_f64(ctx)
    kw.pop("wall_zero_p")
    zeta64, dt64 = zeta.astype(np.float64), dt.astype(np.float64)
    eps = 1e-6
    scale = max(np.abs(gz).max(), np.abs(gd).max(), abs(gk))
    for t in (0, 7, 19, 33, 48, 59):
        zp, zm = zeta64.copy(), zeta64.copy()
        zp[t] += eps
        zm[t] -= eps
        fd = (oracle.objective(J, None, zp, dt64, q0, **kw) - oracle.objective(J, None, zm, dt64, q0, **kw)) / (2 * eps)
        assert abs(gz[t] - fd) <= 1e-4 * scale, (t, gz[t], fd)
        dp, dm = dt64.copy(), dt64.copy()
        dp[t] += eps
        dm[t] -= eps
        fd = (oracle.objective(J, None, zeta64, dp, q0, **kw) - oracle.objective(J, None, zeta64, dm, q0, **kw)) / (2 * eps)
        assert abs(gd[t] - fd) <= 1e-4 * scale, (t, gd[t], fd)
    kp = dict(kw, k=kw["k"] + eps)
    km = dict(kw, k=kw["k"] - eps)
    fd = (oracle.objective(J, None, zeta64, dt64, q0, **kp) - oracle.objective(J, None, zeta64, dt64, q0, **km)) / (2 * eps)
    assert abs(gk - fd) <= 1e-4 * scale


def test_fp64_adjoint_against_gpu_central_differences():
    """The same check with the differences taken on the GPU: FP64 forward
    runs of the library at perturbed schedules (and spring constants), the
    relaxed energy of their FP64 final states (si_get_state), against the
    FP64 adjoint.  The perturbation is the one the float32 schedule entries
    actually received."""
    n, R, T = 64, 4, 60
    J, q0, zeta, dt = _case(n, R, T, seed=5)
    J64 = J.astype(np.float64)
    eps = 1e-5
    with b.Context(J, replicas=R, steps=T, prec="fp64") as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)

        def L(z, d):
            ctx.run(z, d, q0)
            q, _ = ctx.get_state()
            return float(oracle.relaxed_energy(J64, None, q).sum())

        scale = max(np.abs(gz).max(), np.abs(gd).max(), abs(gk))
        for t in (0, 7, 19, 33, 48, 59):
            zp, zm = zeta.copy(), zeta.copy()
            zp[t] = np.float32(zeta[t] + eps)
            zm[t] = np.float32(zeta[t] - eps)
            fd = (L(zp, dt) - L(zm, dt)) / (float(zp[t]) - float(zm[t]))
            assert abs(gz[t] - fd) <= 1e-4 * scale, (t, gz[t], fd)
            dp, dm = dt.copy(), dt.copy()
            dp[t] = np.float32(dt[t] + eps)
            dm[t] = np.float32(dt[t] - eps)
            fd = (L(zeta, dp) - L(zeta, dm)) / (float(dp[t]) - float(dm[t]))
            assert abs(gd[t] - fd) <= 1e-4 * scale, (t, gd[t], fd)
    k0 = float(b.default_params().k)
    kp, km = np.float32(k0 + eps), np.float32(k0 - eps)
    Ls = []
    for kk in (kp, km):
        with b.Context(J, replicas=R, steps=T, prec="fp64", k=float(kk)) as ck:
            ck.run(zeta, dt, q0)
            q, _ = ck.get_state()
            Ls.append(float(oracle.relaxed_energy(J64, None, q).sum()))
    fd = (Ls[0] - Ls[1]) / (float(kp) - float(km))
    assert abs(gk - fd) <= 1e-4 * scale


@pytest.mark.parametrize("kind,n,R", [("tensor", 96, 8), ("tensor", 300, 70), ("simt-env", 96, 8),
                                      ("simt-j", 96, 8)])
def test_fp32_adjoint_close_to_oracle(kind, n, R, monkeypatch):
    """FP32 adjoint vs the FP64 reverse mode on a short horizon: the FP32
    forward drifts from the FP64 one by rounding, amplified by the dynamics,
    so the bar is 1e-3 relative to the largest component.  Both product
    paths: tensor cores (J exact in bf16; three-piece operand split, ragged
    n and R > 64) and CUDA cores (forced, or J not exact in bf16)."""
    T = 30
    J, q0, zeta, dt = _case(n, R, T, seed=9)
    if kind == "simt-env":
        monkeypatch.setenv("SI_ADJOINT_SIMT", "1")
    if kind == "simt-j":
        J = (J / np.float32(3.0)).astype(np.float32)
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=10) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        kw = params_f64(ctx)
        assert ("grad=tcgen05-bf16x3" if kind == "tensor" else "grad=cuda-core") in ctx.describe()
    kw.pop("wall_zero_p")
    o_obj, o_gz, o_gd, o_gk = oracle.grad(J, None, zeta, dt, q0, **kw)
    assert abs(obj - o_obj) <= 1e-4 * abs(o_obj)
    assert _rel(gz, o_gz) <= 1e-3 and _rel(gd, o_gd) <= 1e-3
    assert abs(gk - o_gk) <= 1e-3 * max(abs(o_gk), np.abs(o_gd).max())


def test_fp32_tensor_adjoint_at_the_timed_shape():
    """The shape the gradient workload times: N=2000 +-1 couplings, so the
    products run on the tensor cores with K split over the same thread-block
    cluster size as the R=64 workload (asserted through si_describe), here
    with R=4 replicas and T=20 steps so that the oracle's FP64 reverse mode
    finishes in seconds.  Every output is compared, g_k included, at the
    FP32 bar of 1e-3 relative."""
    n, R, T = 2000, 4, 20
    J, q0, zeta, dt = _case(n, R, T, seed=1)
    with b.Context(J, replicas=64, steps=T, prec="fp32", ckpt_every=10) as cw:
        cw.grad(zeta, dt, inputs.positions(n, 64, seed0=10))
        split_workload = cw.describe().split("ksplit=")[1].split()[0]
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=10) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        desc = ctx.describe()
        kw = params_f64(ctx)
    assert "grad=tcgen05-bf16x3" in desc
    assert desc.split("ksplit=")[1].split()[0] == split_workload and int(split_workload) > 1
    kw.pop("wall_zero_p")
    o_obj, o_gz, o_gd, o_gk = oracle.grad(J, None, zeta, dt, q0, **kw)
    assert abs(obj - o_obj) <= 1e-4 * abs(o_obj)
    assert _rel(gz, o_gz) <= 1e-3 and _rel(gd, o_gd) <= 1e-3
    assert abs(gk - o_gk) <= 1e-3 * max(abs(o_gk), np.abs(o_gd).max())


def test_set_params_changes_k_without_a_new_context():
    """si_set_params on a live context: the gradient under the new spring
    constant equals that of a context created with it, bit for bit."""
    n, R, T = 96, 8, 30
    J, q0, zeta, dt = _case(n, R, T, seed=12)
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=10) as ctx:
        ctx.grad(zeta, dt, q0)
        ctx.set_params(k=0.7, ckpt_every=7)
        r1 = ctx.grad(zeta, dt, q0)
        q1, p1, _ = ctx.run(zeta, dt, q0)
        with pytest.raises(b.SpringIsingError):
            ctx.set_params(replicas=R + 1)
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=7, k=0.7) as cx:
        r2 = cx.grad(zeta, dt, q0)
        q2, p2, _ = cx.run(zeta, dt, q0)
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2]) and r1[3] == r2[3]
    assert np.array_equal(q1, q2) and np.array_equal(p1, p2)


def test_autograd_device_binding_reuses_one_context():
    """relaxed_energy with CUDA tensors: J is copied into a library context
    once; later forward/backward passes (with a new k each time, set through
    si_set_params) reuse it, keep every tensor on the device, and equal
    si_grad bit for bit."""
    import torch
    from paper_2305_07187_gb300 import autograd as ag
    ag.clear_cache()
    dev = torch.device("cuda")
    n, R, T = 96, 8, 30
    J, q0, zeta, dt = _case(n, R, T, seed=13)
    Jd, qd = torch.from_numpy(J).to(dev), torch.from_numpy(q0).to(dev)
    created0, reused0 = ag.stats["created"], ag.stats["reused"]
    for it in range(3):
        kval = float(np.float32(0.5 + 0.01 * it))
        z = torch.tensor(zeta, device=dev, requires_grad=True)
        d = torch.tensor(dt, device=dev, requires_grad=True)
        k = torch.tensor(kval, device=dev, requires_grad=True)
        E = ag.relaxed_energy(Jd, z, d, k, qd)
        E.backward()
        assert E.is_cuda and z.grad.is_cuda and d.grad.is_cuda and k.grad.is_cuda
        with b.Context(J, replicas=R, steps=T, k=kval) as ctx:
            obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        assert E.item() == obj
        assert np.array_equal(z.grad.cpu().numpy(), gz) and np.array_equal(d.grad.cpu().numpy(), gd)
        assert k.grad.item() == np.float32(gk)
    assert ag.stats["created"] - created0 == 1 and ag.stats["reused"] - reused0 == 2
    ag.clear_cache()


def test_checkpoint_interval_does_not_change_the_gradient():
    n, R, T = 120, 5, 47
    J, q0, zeta, dt = _case(n, R, T, seed=3)
    res = []
    for K in (1, 7, 50):
        with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=K) as ctx:
            res.append(ctx.grad(zeta, dt, q0))
    for r in res[1:]:
        assert r[0] == res[0][0] and np.array_equal(r[1], res[0][1]) and np.array_equal(r[2], res[0][2])
        assert r[3] == res[0][3]


def test_gradient_workload_n2000_r64_t500():
    """The gradient workload: N=2000 +-1, R=64, T=500, checkpoints every 50.
    The objective equals the relaxed energy, evaluated by the oracle, of the
    final state of the gradient's own forward sweep (si_get_state after
    si_grad); that state keeps the walls and stays close to si_run's."""
    n, R, T = 2000, 64, 500
    J, q0, zeta, dt = _case(n, R, T, seed=1)
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=50) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
        assert "grad=tcgen05-bf16x3" in ctx.describe()
        qT, pT = ctx.get_state()
        q, p, s = ctx.run(zeta, dt, q0)
    assert np.isfinite(gz).all() and np.isfinite(gd).all() and np.isfinite(gk)
    assert np.abs(qT).max() <= b.SQRT2_F32 and np.abs(pT).max() <= 2.0
    ref = oracle.relaxed_energy(J, None, qT).sum()
    assert abs(obj - ref) <= 1e-5 * abs(ref)
    # chaotic divergence from si_run's trajectory stays a small fraction
    run_E = oracle.relaxed_energy(J, None, q).sum()
    assert abs(ref - run_E) <= 1e-2 * abs(run_E)


def test_autograd_function_and_schedule_tuning():
    import torch
    from paper_2305_07187_gb300.autograd import relaxed_energy
    n, R, T = 64, 4, 40
    J, q0, zeta, dt = _case(n, R, T, seed=11)
    z = torch.tensor(zeta, requires_grad=True)
    d = torch.tensor(dt, requires_grad=True)
    k = torch.tensor(0.5, requires_grad=True)
    E = relaxed_energy(J, z, d, k, q0)
    E.backward()
    with b.Context(J, replicas=R, steps=T) as ctx:
        obj, gz, gd, gk = ctx.grad(zeta, dt, q0)
    assert abs(E.item() - obj) == 0
    assert np.array_equal(z.grad.numpy(), gz) and np.array_equal(d.grad.numpy(), gd)
    assert k.grad.item() == np.float32(gk)
    # a few gradient steps on the coupling schedule lower the relaxed energy
    z = torch.tensor(zeta, requires_grad=True)
    opt = torch.optim.SGD([z], lr=1e-4)
    first = None
    for _ in range(5):
        opt.zero_grad()
        E = relaxed_energy(J, z, torch.tensor(dt), 0.5, q0)
        if first is None:
            first = E.item()
        E.backward()
        opt.step()
    assert relaxed_energy(J, z.detach(), torch.tensor(dt), 0.5, q0).item() < first
