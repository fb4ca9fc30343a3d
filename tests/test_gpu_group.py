"""GPU parity of the grouped batch path (si_create_group / si_run_group):
many independent instances of uneven size in one launch per step."""
import numpy as np
import pytest

from _helpers import b, bf16_step_bound, inputs, oracle

pytestmark = pytest.mark.gpu


def _members():
    # (n, R, kind): ragged sizes, both tile widths, +-1 and Gaussian couplings
    return [(17, 16, "pm1"), (128, 48, "gauss"), (300, 64, "pm1"), (513, 130, "gauss"),
            (1000, 200, "pm1"), (64, 1, "pm1"), (257, 96, "gauss"), (130, 300, "pm1")]


def _build(members, seed=0):
    Js, hs, qs = [], [], []
    for k, (n, R, kind) in enumerate(members):
        J = inputs.pm1_coupling(n, seed=100 + k) if kind == "pm1" else inputs.gauss_coupling_bf16(n, seed=100 + k)
        Js.append(J)
        hs.append(inputs.field(n, seed=200 + k, scale=0.3) if kind == "gauss" else None)
        qs.append(inputs.positions(n, R, seed0=1000 * (k + 1) + seed))
    return Js, hs, qs


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4])
def test_group_per_step_within_bf16_bound(policy, monkeypatch):
    """Every tile policy (replica blocks of 64 / 128, whole-instance tiles in
    one accumulator) takes the same step within the bf16 bound."""
    monkeypatch.setenv("SI_GROUP_POLICY", str(policy))
    members = _members()
    Js, hs, qs = _build(members)
    ps = [np.zeros_like(q) for q in qs]
    T = 8
    zeta, dt = inputs.zeta_ramp(T, end=0.5), inputs.dt_const(T)
    precs = ["j_fp8_q_bf16" if kind == "pm1" else "j_bf16_q_bf16" for (_, _, kind) in members]
    with b.Group(Js, hs, replicas=[R for (_, R, _) in members], steps=1, precs=precs) as g:
        assert "grouped" in g.describe()
        names = ["bn64-if-R<=64-else-128", "all-64", "all-128", "whole-instance", "whole-instance-tmem-a"]
        p0 = b.default_params()
        kw = dict(k=float(p0.k), m=float(p0.m), q0=float(p0.q0), q_max=float(np.float32(p0.q_max)),
                  p_max=float(p0.p_max))
        for t in range(T):
            qg, pg, _ = g.run(zeta[t:t + 1], dt[t:t + 1], qs, ps)
            for k, (n, R, kind) in enumerate(members):
                qo, po = oracle.run(Js[k], hs[k], zeta[t:t + 1], dt[t:t + 1], qs[k], ps[k], **kw)
                eq, ep = bf16_step_bound(Js[k], qs[k].astype(np.float64), ps[k].astype(np.float64),
                                         float(zeta[t]), float(dt[t]), kw, h=hs[k])
                assert (np.abs(qg[k] - qo) <= eq).all(), (t, k)
                assert (np.abs(pg[k] - po) <= ep).all(), (t, k)
            qs, ps = qg, pg
        assert "policy=" + names[policy] in g.describe()


@pytest.mark.parametrize("policy", [-1, 3])
def test_group_free_run_energies_and_determinism(policy, monkeypatch):
    if policy >= 0:
        monkeypatch.setenv("SI_GROUP_POLICY", str(policy))
    members = _members()
    Js, hs, qs = _build(members, seed=5)
    T = 60
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    with b.Group(Js, hs, replicas=[R for (_, R, _) in members], steps=T) as g:
        q1, p1, s1 = g.run(zeta, dt, qs)
        q2, p2, s2 = g.run(zeta, dt, qs)
        for k, (n, R, kind) in enumerate(members):
            assert np.array_equal(q1[k], q2[k]) and np.array_equal(s1[k], s2[k])
            assert np.abs(q1[k]).max() <= b.SQRT2_F32 and np.abs(p1[k]).max() <= 2.0
            np.testing.assert_array_equal(s1[k], oracle.sign(q1[k]))
            if kind == "pm1":
                e, c, _ = g.energy(k, s1[k])
                np.testing.assert_array_equal(e, oracle.energy(Js[k], None, s1[k]).astype(np.int64))
                np.testing.assert_array_equal(c, oracle.cut(Js[k], s1[k]).astype(np.int64))
            else:
                _, _, f = g.energy(k, s1[k], exact=False)
                ref = oracle.energy(Js[k], hs[k], s1[k])
                bound = 1e-5 * (np.abs(Js[k]).sum() + np.abs(hs[k]).sum())
                np.testing.assert_allclose(f, ref, rtol=0, atol=bound)


def test_group_uneven_sample_of_the_batched_workload():
    """A slice of the uneven batch (instances with n <= 3000 from the seeded
    recipe), 30 steps: every member keeps its walls and exact energies."""
    import torch
    specs = [s for s in inputs.uneven_instances(256) if s.n <= 3000][:24]
    Js = [inputs.instance_coupling_torch(s) for s in specs]
    qs = [inputs.positions_torch(s.n, s.replicas, seed=9000 + s.index) for s in specs]
    T = 30
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    precs = ["j_fp8_q_bf16" if s.kind == "pm1" else "j_bf16_q_bf16" for s in specs]
    with b.Group(Js, None, replicas=[s.replicas for s in specs], steps=T, precs=precs) as g:
        sp = [torch.empty((s.replicas, s.n), dtype=torch.int8, device="cuda") for s in specs]
        g.run_into(torch.from_numpy(zeta).cuda(), torch.from_numpy(dt).cuda(), qs, None, None, None, sp)
        torch.cuda.synchronize()
        for k in (0, 1, 2, 3):
            s = sp[k].cpu().numpy()
            Jh = Js[k].cpu().numpy()
            if specs[k].kind == "pm1":
                e, c, _ = g.energy(k, s)
                np.testing.assert_array_equal(e, oracle.energy(Jh, None, s).astype(np.int64))
            else:
                _, _, f = g.energy(k, s, exact=False)
                np.testing.assert_allclose(f, oracle.energy(Jh, None, s), rtol=0, atol=1e-5 * np.abs(Jh).sum())


def test_group_rejects_mismatched_parameters():
    J = inputs.pm1_coupling(32, seed=1)
    with pytest.raises(b.SpringIsingError):
        b.Group([J, J], replicas=[4, 4], steps=5, precs=["fp32", "fp32"])


def test_group_block_sparse_king_graphs():
    """King graphs (banded J) in a group with a dense member: all-zero
    128 x 64 blocks of J are skipped, the step stays within the bf16 bound,
    energies are exact, and the J bytes per step drop."""
    import re
    members = [("king", 32, 64), ("king", 13, 16), ("dense", 300, 32)]
    Js = [inputs.king_graph_coupling(a, seed=70 + k) if kind == "king" else inputs.pm1_coupling(a, seed=70 + k)
          for k, (kind, a, _) in enumerate(members)]
    Rs = [R for (_, _, R) in members]
    qs = [inputs.positions(J.shape[0], R, seed0=7000 + 100 * k) * 4 for k, (J, R) in enumerate(zip(Js, Rs))]
    ps = [np.zeros_like(q) for q in qs]
    T = 5
    zeta, dt = inputs.zeta_ramp(T, start=0.3, end=0.5), inputs.dt_const(T)
    p0 = b.default_params()
    kw = dict(k=float(p0.k), m=float(p0.m), q0=float(p0.q0), q_max=float(np.float32(p0.q_max)), p_max=float(p0.p_max))
    with b.Group(Js, None, replicas=Rs, steps=1, precs="j_fp8_q_bf16") as g:
        for t in range(T):
            qg, pg, _ = g.run(zeta[t:t + 1], dt[t:t + 1], qs, ps)
            for k in range(len(members)):
                qo, po = oracle.run(Js[k], None, zeta[t:t + 1], dt[t:t + 1], qs[k], ps[k], **kw)
                eq, ep = bf16_step_bound(Js[k], qs[k].astype(np.float64), ps[k].astype(np.float64),
                                         float(zeta[t]), float(dt[t]), kw)
                assert (np.abs(qg[k] - qo) <= eq).all() and (np.abs(pg[k] - po) <= ep).all(), (t, k)
            qs, ps = qg, pg
        jbytes = int(re.search(r"jbytes/step=(\d+)", g.describe()).group(1))
    dense = sum(-(-J.shape[0] // 128) * 128 * -(-J.shape[0] // 64) * 64 * 2 * -(-R // 64)
                for J, R in zip(Js, Rs))
    assert jbytes < 0.6 * dense
    with b.Group(Js, None, replicas=Rs, steps=30, precs="j_fp8_q_bf16") as g:
        _, _, s = g.run(inputs.zeta_ramp(30), inputs.dt_const(30), qs)
        for k in range(len(members)):
            e, c, _ = g.energy(k, s[k])
            np.testing.assert_array_equal(e, oracle.energy(Js[k], None, s[k]).astype(np.int64))
            np.testing.assert_array_equal(c, oracle.cut(Js[k], s[k]).astype(np.int64))


def test_autotune_cache_persists_across_processes(tmp_path):
    """SI_TUNE_CACHE: the autotuner's choice is written to the file and a
    later process takes the policy from it without timing (here a policy
    edited into the file, which the second process must use)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    code = (
        "import sys, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2305_07187_gb300 import _binding as b, inputs\n"
        "Js = [inputs.pm1_coupling(n, seed=5) for n in (96, 160)]\n"
        "with b.Group(Js, None, replicas=[48, 80], steps=4, precs='j_fp8_q_bf16') as g:\n"
        "    g.run(inputs.zeta_ramp(4), inputs.dt_const(4), [inputs.positions(96, 48), inputs.positions(160, 80)])\n"
        "    print(g.describe())\n" % root)
    env = dict(os.environ, SI_TUNE_CACHE=str(cache))
    env.pop("SI_GROUP_POLICY", None)
    out1 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out1.returncode == 0, out1.stderr
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1
    key, pol = lines[0].rsplit(" ", 1)
    assert "96x48" in key and "160x80" in key
    names = ["bn64-if-R<=64-else-128", "all-64", "all-128", "whole-instance", "whole-instance-tmem-a"]
    assert "policy=" + names[int(pol)] in out1.stdout
    other = (int(pol) + 1) % 4
    cache.write_text("%s %d\n" % (key, other))
    out2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out2.returncode == 0, out2.stderr
    assert "policy=" + names[other] in out2.stdout
    assert cache.read_text().strip().splitlines() == ["%s %d" % (key, other)]


@pytest.mark.parametrize("policy,n,R", [(1, 3072, 512), (2, 1280, 256), (3, 12288, 512)])
def test_group_split_tiles_per_step(policy, n, R, monkeypatch):
    """Tile lists with more tiles than CTAs: some tiles are split into two of
    half the replicas (the describe string's tile count exceeds the plain
    count).  One step from the same state, checked against the oracle on a
    sample of replicas spread over every tile (replicas are independent)."""
    import re
    import torch
    monkeypatch.setenv("SI_GROUP_POLICY", str(policy))
    J = inputs.pm1_coupling_torch(n, seed=60 + policy, device="cuda")
    q = inputs.positions_torch(n, R, seed=6000 + policy, device="cuda")
    z = torch.tensor([0.3], device="cuda")
    d = torch.tensor([0.2], device="cuda")
    with b.Group([J], None, replicas=[R], steps=1, precs="j_fp8_q_bf16") as g:
        qo_d = torch.empty_like(q)
        po_d = torch.empty_like(q)
        g.run_into(z, d, [q], None, [qo_d], [po_d], None)
        torch.cuda.synchronize()
        desc = g.describe()
    bn = {1: 64, 2: 128, 3: 256}[policy]
    plain_tiles = (-(-n // 128)) * (-(-R // bn))
    assert int(re.search(r"tiles=(\d+)", desc).group(1)) > plain_tiles, desc
    sample = np.arange(3, R, 37)
    Jh = J.cpu().numpy().astype(np.float64)
    qh = q.cpu().numpy()[sample].astype(np.float64)
    p0 = b.default_params()
    kw = dict(k=float(p0.k), m=float(p0.m), q0=float(p0.q0), q_max=float(np.float32(p0.q_max)), p_max=float(p0.p_max))
    qo, po = oracle.run(Jh, None, np.array([0.3]), np.array([0.2]), qh, None, **kw)
    eq, ep = bf16_step_bound(Jh, qh, np.zeros_like(qh), 0.3, 0.2, kw)
    qg = qo_d.cpu().numpy()[sample]
    pg = po_d.cpu().numpy()[sample]
    assert (np.abs(qg - qo) <= eq).all() and (np.abs(pg - po) <= ep).all()
