"""The allocation-free entry point si_run_noalloc, through the C ABI.

It serves callers that cannot allocate device memory (their host owns every
allocation, or they must not enter the allocator), using the library's fixed
scratch array.  Checked against the ordinary FP32 single-replica run
(si_create + si_run) on two calls in a row, so that the reused scratch is
shown to start clean each time.  Collected last on purpose.
"""
import numpy as np
import pytest

from _helpers import b, inputs, normwise_rel, oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,T,exact", [(2000, 300, True), (1000, 40, False), (37, 25, False)])
def test_noalloc_matches_context_run_twice(n, T, exact):
    import torch
    dev = torch.device("cuda")
    J = inputs.pm1_coupling(n, seed=n + 3)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    q0 = inputs.positions(n, 1, seed0=77)
    with b.Context(J, replicas=1, steps=T, prec="fp32") as ctx:
        q_ref, p_ref, s_ref = ctx.run(zeta, dt, q0)
    Jd = torch.from_numpy(J).to(dev)
    zd, dd = torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev)
    for call in range(2):
        qd = torch.from_numpy(q0[0].copy()).to(dev)
        pd = torch.zeros(n, dtype=torch.float32, device=dev)
        sd = torch.empty(n, dtype=torch.int8, device=dev)
        b.run_noalloc(Jd, None, zd, dd, qd, pd, sd)
        q, p, s = qd.cpu().numpy(), pd.cpu().numpy(), sd.cpu().numpy()
        if exact:
            assert np.array_equal(q, q_ref[0]) and np.array_equal(p, p_ref[0]), call
            assert np.array_equal(s, s_ref[0]), call
        else:
            assert normwise_rel(q, p, q_ref[0], p_ref[0]) <= 1e-6, call


@pytest.mark.parametrize("n", [8192, b.NOALLOC_MAX_N])
def test_noalloc_global_coupling_rows_against_oracle(n):
    """Sizes whose rows of J no longer fit in a CTA's shared memory, so the
    kernel reads J from global memory every step (the largest allowed n
    included): per step from an identical state against the FP64 oracle
    (1e-6 normwise, the FP32 bar), and a three-step call equal bit for bit to
    three one-step calls."""
    import torch
    dev = torch.device("cuda")
    T = 3
    J = inputs.pm1_coupling(n, seed=n + 11)
    zeta = inputs.zeta_ramp(2000)[1500:1500 + T]
    dt = inputs.dt_const(T)
    q = (inputs.positions(n, 1, seed0=91) * 8).astype(np.float32)
    p = np.zeros_like(q)
    Jd = torch.from_numpy(J).to(dev)
    zd, dd = torch.from_numpy(zeta).to(dev), torch.from_numpy(dt).to(dev)
    kw = dict(k=0.5, m=1.0, q0=0.0, q_max=float(np.float32(b.SQRT2_F32)), p_max=2.0)
    qd = torch.from_numpy(q[0].copy()).to(dev)
    pd = torch.from_numpy(p[0].copy()).to(dev)
    for t in range(T):
        b.run_noalloc(Jd, None, zd[t:t + 1], dd[t:t + 1], qd, pd)
        qg, pg = qd.cpu().numpy()[None, :], pd.cpu().numpy()[None, :]
        qo, po = oracle.run(J, None, zeta[t:t + 1], dt[t:t + 1], q, p, **kw)
        assert normwise_rel(qg, pg, qo, po) <= 1e-6, t
        q, p = qg, pg
    q3 = torch.from_numpy((inputs.positions(n, 1, seed0=91) * 8).astype(np.float32)[0]).to(dev)
    p3 = torch.zeros(n, dtype=torch.float32, device=dev)
    b.run_noalloc(Jd, None, zd, dd, q3, p3)
    assert np.array_equal(q3.cpu().numpy(), q[0]) and np.array_equal(p3.cpu().numpy(), p[0])


def test_noalloc_rejects_too_large_n():
    import torch
    n = b.NOALLOC_MAX_N + 1
    dev = torch.device("cuda")
    q = torch.zeros(n, dtype=torch.float32, device=dev)
    p = torch.zeros(n, dtype=torch.float32, device=dev)
    J = torch.zeros(1, dtype=torch.float32, device=dev)   # never read: rejected first
    z = torch.zeros(1, dtype=torch.float32, device=dev)
    with pytest.raises(b.SpringIsingError) as ei:
        lib = b.load()
        import ctypes
        prm = b.default_params(n=n, replicas=1, steps=1)
        st = lib.si_run_noalloc(ctypes.byref(prm), ctypes.c_void_p(J.data_ptr()), None,
                                ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p.data_ptr()), None, None)
        b._check(st)
    assert ei.value.status == b.SI_ERR_INVALID_ARG
    assert "SI_NOALLOC_MAX_N" in str(ei.value)
