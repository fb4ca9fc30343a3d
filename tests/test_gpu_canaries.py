"""Guard regions around every device output of the C ABI (compute-sanitizer
is closed on this machine): each output is the middle of a larger device
buffer filled with a sentinel; after the call the guards are unchanged and
the output holds no sentinel.  Ragged sizes on every path."""
import numpy as np
import pytest

from _helpers import b, inputs

pytestmark = pytest.mark.gpu

G = 4096  # guard elements on each side


def _guarded(torch, numel, dtype):
    sent = {torch.int8: 0x5A, torch.int32: 0x5A5A5A5A}.get(dtype, -12345.25)
    buf = torch.full((numel + 2 * G,), sent, dtype=dtype, device="cuda")
    return buf, buf[G:G + numel], sent


def _check(torch, buf, numel, sent, written=True):
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert (h[:G] == sent).all() and (h[G + numel:] == sent).all(), "guard overwritten"
    if written and numel:
        assert not (h[G:G + numel] == sent).any(), "output not fully written"


@pytest.mark.parametrize("prec,n,R", [("fp32", 129, 3), ("fp32", 77, 17), ("j_fp8_q_bf16", 129, 17),
                                      ("j_fp8_q_bf16", 300, 70), ("fp64", 33, 5)])
def test_run_energy_hamiltonian_outputs(prec, n, R):
    import torch
    T = 4
    J = inputs.pm1_coupling(n, seed=51)
    q0 = torch.from_numpy(inputs.positions(n, R, seed0=5100)).cuda()
    z = torch.from_numpy(inputs.zeta_ramp(T)).cuda()
    d = torch.from_numpy(inputs.dt_const(T)).cuda()
    with b.Context(J, replicas=R, steps=T, prec=prec) as c:
        qb, qv, qs = _guarded(torch, n * R, torch.float32)
        pb, pv, ps = _guarded(torch, n * R, torch.float32)
        sb, sv, ss = _guarded(torch, n * R, torch.int8)
        c.run_into(z, d, q0, None, qv, pv, sv)
        for buf, sent in ((qb, qs), (pb, ps), (sb, ss)):
            _check(torch, buf, n * R, sent)
        eb, ev, es = _guarded(torch, R, torch.int32)
        cb, cv, cs = _guarded(torch, R, torch.int32)
        fb, fv, fs = _guarded(torch, R, torch.float64)
        c.energy_into(sv, R, ev, cv, fv)
        for buf, sent in ((eb, es), (cb, cs), (fb, fs)):
            _check(torch, buf, R, sent)
        hb, hv, hs = _guarded(torch, R, torch.float64)
        c.hamiltonian(qv, pv, 0.3, out=hv)
        _check(torch, hb, R, hs)


def test_grad_outputs():
    import torch
    n, R, T = 129, 70, 9
    J = inputs.pm1_coupling(n, seed=52)
    q0 = torch.from_numpy(inputs.positions(n, R, seed0=5200)).cuda()
    z = torch.from_numpy(inputs.zeta_ramp(T)).cuda()
    d = torch.from_numpy(inputs.dt_const(T)).cuda()
    with b.Context(J, replicas=R, steps=T, prec="fp32", ckpt_every=4) as c:
        outs = [_guarded(torch, T, torch.float32), _guarded(torch, T, torch.float32),
                _guarded(torch, 1, torch.float32), _guarded(torch, 1, torch.float32)]
        c.grad_into(z, d, q0, None, *[o[1] for o in outs])
        for (buf, _, sent), numel in zip(outs, (T, T, 1, 1)):
            _check(torch, buf, numel, sent)


def test_group_outputs():
    import torch
    members = [(129, 17), (77, 48), (300, 70)]
    T = 3
    Js = [inputs.pm1_coupling(n, seed=53 + k) for k, (n, _) in enumerate(members)]
    qs = [torch.from_numpy(inputs.positions(n, R, seed0=5300 + k)).cuda() for k, (n, R) in enumerate(members)]
    z = torch.from_numpy(inputs.zeta_ramp(T)).cuda()
    d = torch.from_numpy(inputs.dt_const(T)).cuda()
    with b.Group(Js, None, replicas=[R for _, R in members], steps=T, precs="j_fp8_q_bf16") as g:
        bufs = [(_guarded(torch, n * R, torch.float32), _guarded(torch, n * R, torch.float32),
                 _guarded(torch, n * R, torch.int8)) for n, R in members]
        g.run_into(z, d, qs, None, [x[0][1] for x in bufs], [x[1][1] for x in bufs], [x[2][1] for x in bufs])
        for (n, R), trio in zip(members, bufs):
            for buf, _, sent in trio:
                _check(torch, buf, n * R, sent)
