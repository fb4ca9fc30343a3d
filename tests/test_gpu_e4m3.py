"""FP8 e4m3 storage of J (SI_PREC_J_FP8_Q_BF16).

The grouped per-step kernel (and every context it serves) keeps J in HBM as
1-byte e4m3 and widens each 128 x 64 tile to bf16 before the tensor cores
read it (in shared memory, or in tensor memory as the MMA's A operand); the
persistent kernel does the same into tensor memory when SI_TC_J_E4M3=1 (by
default it keeps a bf16 copy, its J tiles being L2-resident).  Every finite
e4m3 value is exact in bf16, so a context that stores J as e4m3 must compute
exactly what a context storing the same J as bf16 computes: bit-identical
states, spins and energies.  J here takes every finite e4m3 value (both signs, subnormals
included), so a wrong swizzle position, byte order or exponent mapping of
the widening shows up as a difference.  The per-step parity of both against
the oracle is in test_gpu_tc / test_gpu_group.
"""
import numpy as np
import pytest

from _helpers import b, inputs, oracle, random_spins

pytestmark = pytest.mark.gpu


def _e4m3_values():
    """All finite e4m3 values, decoded from the format's definition (sign,
    4-bit exponent with bias 7, 3-bit mantissa; exponent 0 is subnormal;
    code 0x7F / 0xFF is NaN)."""
    vals = []
    for code in range(256):
        if code & 0x7F == 0x7F:
            continue
        s = -1.0 if code & 0x80 else 1.0
        e, m = (code >> 3) & 0xF, code & 0x7
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        vals.append(s * v)
    return np.array(vals, np.float32)


def _all_codes_coupling(n, seed):
    vals = _e4m3_values()
    g = np.random.Generator(np.random.PCG64(seed))
    U = vals[g.integers(0, vals.size, size=(n, n))]
    # every code appears at least once in the upper triangle
    iu = np.triu_indices(n, 1)
    k = min(vals.size, iu[0].size)
    U[iu[0][:k], iu[1][:k]] = vals[:k]
    J = np.triu(U, 1)
    return (J + J.T).astype(np.float32)


def test_e4m3_values_are_the_format():
    v = _e4m3_values()
    assert v.size == 254 and np.unique(v).size == 253   # +0 and -0 compare equal
    assert v.max() == 448.0 and np.abs(v[v != 0]).min() == 2.0 ** -9
    assert np.array_equal(inputs.round_to_bf16(v), v)   # all exact in bf16


ZETA_SMALL = 2.0 ** -8   # keeps zeta * dt * |J| < p_max for |J| <= 448: no momentum saturates


@pytest.fixture
def e4m3_operand(monkeypatch):
    """The persistent kernel with the e4m3 operand widened per tile."""
    monkeypatch.setenv("SI_TC_J_E4M3", "1")


@pytest.mark.parametrize("tile_n", [64, 128])
def test_widened_coupling_read_back_through_one_step(tile_n, e4m3_operand):
    """One step from q_r = e_r / 2 (replica r displaced at spin r only, exact
    in bf16): F_ir = J_ir / 2 exactly, so the new momenta read J back column
    by column.  FP8 storage must give the bf16-storage result bit for bit,
    and both the value that FP32 arithmetic gives for J_ir."""
    n = 300
    J = _all_codes_coupling(n, seed=3)
    R = n
    q0 = np.eye(n, dtype=np.float32) * np.float32(0.5)
    zeta = np.full(1, ZETA_SMALL, np.float32)
    dt = inputs.dt_const(1)
    out = {}
    for prec in ("j_fp8_q_bf16", "j_bf16_q_bf16"):
        with b.Context(J, replicas=R, steps=1, prec=prec, tile_n=tile_n) as c:
            out[prec] = c.run(zeta, dt, q0)
    for a_, b_ in zip(out["j_fp8_q_bf16"], out["j_bf16_q_bf16"]):
        np.testing.assert_array_equal(a_, b_)
    p = out["j_fp8_q_bf16"][1]
    # p_ri = dt (-k q_ri + zeta F_ri), F_ri = J_ir / 2 (J symmetric)
    want = np.float32(0.2) * (np.float32(-0.5) * q0 + np.float32(ZETA_SMALL) * (J.T * np.float32(0.5)))
    np.testing.assert_allclose(p, want, rtol=4 * 2.0 ** -24, atol=0)


@pytest.mark.parametrize("n,R,tile_n", [(300, 40, 64), (300, 40, 128), (129, 17, 0)])
def test_fp8_storage_equals_bf16_storage_every_code(n, R, tile_n, e4m3_operand):
    J = _all_codes_coupling(n, seed=n)
    T = 15
    zeta, dt = np.full(T, ZETA_SMALL, np.float32), inputs.dt_const(T)
    q0 = (inputs.positions(n, R, seed0=5100) * 8).astype(np.float32)
    out = {}
    for prec in ("j_fp8_q_bf16", "j_bf16_q_bf16"):
        with b.Context(J, replicas=R, steps=T, prec=prec, tile_n=tile_n) as c:
            desc = c.describe()
            assert ("J=e4m3(1B)" if prec == "j_fp8_q_bf16" else "J=bf16(2B)") in desc
            q, p, s = c.run(zeta, dt, q0)
            _, _, ef = c.energy(s, exact=False)
            H = c.hamiltonian(q, p, 0.3)
        out[prec] = (q, p, s, ef, H)
    for a_, b_ in zip(out["j_fp8_q_bf16"], out["j_bf16_q_bf16"]):
        np.testing.assert_array_equal(a_, b_)


def test_fp8_storage_equals_bf16_storage_full_workload_shape(e4m3_operand):
    """N=2000, R=1024 (the batched workload's shape and tile), 50 steps."""
    n, R, T = 2000, 1024, 50
    J = inputs.pm1_coupling(n, seed=1)
    zeta, dt = inputs.zeta_ramp(2000)[:T], inputs.dt_const(T)
    q0 = inputs.positions(n, R, seed0=100)
    out = {}
    for prec in ("j_fp8_q_bf16", "j_bf16_q_bf16"):
        with b.Context(J, replicas=R, steps=T, prec=prec) as c:
            assert "tile=128x128" in c.describe()
            q, p, s = c.run(zeta, dt, q0)
            e, cut, _ = c.energy(None)
        out[prec] = (q, p, s, e, cut)
    for a_, b_ in zip(out["j_fp8_q_bf16"], out["j_bf16_q_bf16"]):
        np.testing.assert_array_equal(a_, b_)


@pytest.mark.parametrize("n,R", [(17, 1), (300, 100), (2001, 130)])
def test_exact_readout_from_e4m3_storage(n, R, e4m3_operand):
    """The tensor-core exact readout widens the e4m3 tiles too: integer J
    (values +-3, e4m3-exact) with an integer field, against the oracle."""
    J = inputs.pm1_coupling(n, seed=n) * 3
    h = np.round(inputs.field(n, seed=n + 1) * 10).astype(np.float32)
    s = random_spins(R, n, seed=n + 2)
    with b.Context(J, h, replicas=1, steps=1, prec="j_fp8_q_bf16") as ctx:
        assert "J=e4m3(1B)" in ctx.describe()
        e, c, _ = ctx.energy(s)
    np.testing.assert_array_equal(e, oracle.energy(J, h, s).astype(np.int64))
    np.testing.assert_array_equal(c, oracle.cut(J, s).astype(np.int64))


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4])
def test_group_fp8_members_equal_bf16_members(policy, monkeypatch):
    """Grouped kernel: the same members stored as e4m3 and as bf16 give
    bit-identical runs under every tile policy (mixed with a Gaussian bf16
    member that passes through the converters untouched)."""
    monkeypatch.setenv("SI_GROUP_POLICY", str(policy))
    sizes = [(300, 64), (513, 130), (64, 16), (1000, 200)]
    Js = [_all_codes_coupling(n, seed=700 + k) for k, (n, _) in enumerate(sizes)]
    Jg = inputs.gauss_coupling_bf16(200, seed=77)
    Rs = [R for _, R in sizes] + [48]
    qs = [(inputs.positions(J.shape[0], R, seed0=7100 + k) * 8).astype(np.float32)
          for k, (J, R) in enumerate(zip(Js + [Jg], Rs))]
    T = 9
    zeta, dt = np.full(T, ZETA_SMALL, np.float32), inputs.dt_const(T)
    res = {}
    for prec in ("j_fp8_q_bf16", "j_bf16_q_bf16"):
        with b.Group(Js + [Jg], None, replicas=Rs, steps=T, precs=[prec] * len(sizes) + ["j_bf16_q_bf16"]) as g:
            res[prec] = g.run(zeta, dt, qs)
    for arrs_a, arrs_b in zip(res["j_fp8_q_bf16"], res["j_bf16_q_bf16"]):
        for x, y in zip(arrs_a, arrs_b):
            np.testing.assert_array_equal(x, y)


def test_persistent_kernel_keeps_a_bf16_operand_by_default():
    J = inputs.pm1_coupling(300, seed=4)
    with b.Context(J, replicas=64, steps=1, prec="j_fp8_q_bf16") as c:
        assert "J=bf16(2B)" in c.describe()
    with b.Group([J], None, replicas=[64], steps=1, precs=["j_fp8_q_bf16"]) as g:
        assert "jbytes/step" in g.describe()
