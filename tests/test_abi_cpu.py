"""CPU checks of the boundary: the library loads and exports every function
that include/spring_ising.h declares; host-side parameter logic; inputs."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2305_07187_gb300 import _binding as b
from paper_2305_07187_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(si_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = b.load()
    declared = _declared_functions()
    assert {"si_create", "si_run", "si_energy", "si_grad", "si_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(b.EXPORTS) <= declared


def test_params_struct_layout_and_defaults():
    assert ctypes.sizeof(b.SiParams) == 4 * 17
    p = b.default_params(n=10, replicas=3, steps=7)
    assert (p.k, p.m, p.q0, p.p_max) == (0.5, 1.0, 0.0, 2.0)
    assert p.q_max == np.float32(np.sqrt(2.0))
    assert p.prec == 0 and p.update_order == 0 and p.wall_zero_p == 0
    assert (p.n, p.replicas, p.steps) == (10, 3, 7)


def test_last_error_is_a_string_without_gpu():
    assert isinstance(b.load().si_last_error(), bytes)


def test_pm1_coupling_shape():
    J = inputs.pm1_coupling(50, seed=1)
    assert J.dtype == np.float32 and J.shape == (50, 50)
    assert np.array_equal(J, J.T) and not np.diag(J).any()
    off = J[~np.eye(50, dtype=bool)]
    assert set(np.unique(off)) == {-1.0, 1.0}
    assert np.array_equal(J, inputs.pm1_coupling(50, seed=1))
    assert not np.array_equal(J, inputs.pm1_coupling(50, seed=2))


def test_gauss_coupling_is_bf16_exact():
    J = inputs.gauss_coupling_bf16(64, seed=3)
    assert np.array_equal(J, J.T) and not np.diag(J).any()
    assert np.array_equal(J, inputs.round_to_bf16(J))
    # rounding is to nearest: error below half a bf16 ulp
    x = np.float32([1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159])
    r = inputs.round_to_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 + 2 ** -7 and abs(r[2] + 3.140625) < 1e-7


def test_zeta_ramp():
    z = inputs.zeta_ramp(1000)
    assert z[0] == np.float32(0.04) and z[-1] == np.float32(0.5)
    assert np.all(np.diff(z) > 0)
    z = inputs.zeta_ramp(1000, plateau=200)
    assert len(np.unique(z)) == 5 and z[0] == np.float32(0.04) and z[-1] == np.float32(0.5)


def test_positions_per_replica_seed():
    q = inputs.positions(30, 4, seed0=100)
    assert q.shape == (4, 30) and np.abs(q).max() <= 0.1
    assert np.array_equal(q[2], inputs.positions(30, 1, seed0=102)[0])


def test_uneven_instances():
    s = inputs.uneven_instances(256)
    ns = np.array([x.n for x in s])
    rs = np.array([x.replicas for x in s])
    assert ns.min() >= 256 and ns.max() <= 8192
    assert rs.min() >= 16 and rs.max() <= 256 and np.all(rs % 16 == 0)
    assert [x.kind for x in s[:4]] == ["pm1", "gauss", "pm1", "gauss"]
