"""Allocation failures injected on the host (SI_DEBUG_FAIL_ALLOC=k fails the
k-th device allocation after the last create call): every failure comes
back as SI_ERR_OOM, nothing leaks, and the library works afterwards.  No
GPU fault is involved: the failing cudaMalloc is never issued."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle

pytestmark = pytest.mark.gpu

SI_ERR_OOM = 3


def _run_once(kind, J, q0, T):
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    if kind == "group":
        with b.Group([J, J[:100, :100].copy()], None, replicas=[70, 16], steps=T, precs="j_fp8_q_bf16") as g:
            _, _, s = g.run(zeta, dt, [q0, q0[:16, :100].copy()])
            g.energy(0, s[0])
        return
    prec = {"fp32": "fp32", "tensor": "j_fp8_q_bf16", "grad": "fp32"}[kind]
    with b.Context(J, replicas=q0.shape[0], steps=T, prec=prec) as c:
        if kind == "grad":
            c.grad(zeta, dt, q0)
        else:
            _, _, s = c.run(zeta, dt, q0)
            c.energy(s)


@pytest.mark.parametrize("kind", ["fp32", "tensor", "group", "grad"])
def test_injected_allocation_failures(kind, monkeypatch):
    import torch
    n, R, T = 300, 70, 6
    J = inputs.pm1_coupling(n, seed=41)
    q0 = inputs.positions(n, R, seed0=4100)
    _run_once(kind, J, q0, T)                 # warm: lazy workspaces, caches
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 200):
        monkeypatch.setenv("SI_DEBUG_FAIL_ALLOC", str(k))
        try:
            _run_once(kind, J, q0, T)
        except b.SpringIsingError as e:
            assert e.status == SI_ERR_OOM, str(e)
            failures += 1
            continue
        break                                 # k is past the last allocation
    else:
        pytest.fail("the injected failure never stopped")
    assert failures >= 5
    monkeypatch.delenv("SI_DEBUG_FAIL_ALLOC")
    # repeated failing creates leak nothing
    for _ in range(30):
        monkeypatch.setenv("SI_DEBUG_FAIL_ALLOC", str(max(1, failures - 1)))
        with pytest.raises(b.SpringIsingError):
            _run_once(kind, J, q0, T)
    monkeypatch.delenv("SI_DEBUG_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 32 * 2 ** 20
    # and the library still computes correctly
    with b.Context(J, replicas=4, steps=T, prec="fp32") as c:
        _, _, s = c.run(inputs.zeta_ramp(T), inputs.dt_const(T), q0[:4])
        e, _, _ = c.energy(s)
    np.testing.assert_array_equal(e, oracle.energy(J, None, s).astype(np.int64))
