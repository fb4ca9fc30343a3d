"""The seeded generators that the large workloads draw on the device (the
grouped batch, the N=32768 scale run, the king graph), run here on the CPU
with torch's CPU generator: the couplings they hand to si_create must be
symmetric with a zero diagonal and exact in the storage precision (+-1 in
e4m3 and bf16, Gaussian rounded once to bf16), positions must follow the
stated U[-0.1, 0.1] recipe, and a seed must fix the draw."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_07187_gb300 import inputs


def _np(t):
    return t.cpu().numpy()


def test_pm1_torch_is_symmetric_pm1_with_zero_diagonal():
    J = _np(inputs.pm1_coupling_torch(257, seed=11, device="cpu"))
    assert J.shape == (257, 257) and J.dtype == np.float32
    assert np.array_equal(J, J.T)
    assert not np.diag(J).any()
    off = J[~np.eye(257, dtype=bool)]
    assert set(np.unique(off).tolist()) == {-1.0, 1.0}
    # about half of each sign (binomial, 65792 draws: 5 sigma is under 1 %)
    assert abs((off > 0).mean() - 0.5) < 0.01


def test_gauss_torch_is_symmetric_and_bf16_exact():
    J = _np(inputs.gauss_coupling_bf16_torch(300, seed=12, device="cpu"))
    assert np.array_equal(J, J.T)
    assert not np.diag(J).any()
    assert np.array_equal(J, inputs.round_to_bf16(J))
    off = J[np.triu_indices(300, 1)]
    assert abs(off.mean()) < 0.02 and abs(off.std() - 1.0) < 0.02


def test_positions_torch_recipe_and_seed():
    q = _np(inputs.positions_torch(2000, 64, seed=5, device="cpu"))
    assert q.shape == (64, 2000) and q.dtype == np.float32
    assert q.min() >= -0.1 and q.max() < 0.1
    assert abs(q.mean()) < 0.002
    again = _np(inputs.positions_torch(2000, 64, seed=5, device="cpu"))
    other = _np(inputs.positions_torch(2000, 64, seed=6, device="cpu"))
    assert np.array_equal(q, again) and not np.array_equal(q, other)


def test_king_graph_torch_has_the_king_graph_pattern():
    L = 9
    Jt = _np(inputs.king_graph_coupling_torch(L, seed=3, device="cpu"))
    Jn = inputs.king_graph_coupling(L, seed=3)
    assert np.array_equal(Jt, Jt.T) and not np.diag(Jt).any()
    # same edges as the NumPy king graph (the signs come from another stream)
    assert np.array_equal(Jt != 0, Jn != 0)
    assert set(np.unique(Jt[Jt != 0]).tolist()) <= {-1.0, 1.0}
    deg = (Jt != 0).sum(axis=1).reshape(L, L)
    assert deg[1:-1, 1:-1].min() == 8 and deg[0, 0] == 3 and deg[0, L // 2] == 5
    # every edge joins cells at most one row and one column apart
    i, j = np.nonzero(Jt)
    assert (np.abs(i // L - j // L) <= 1).all() and (np.abs(i % L - j % L) <= 1).all()


def test_instance_coupling_torch_follows_the_kind():
    specs = inputs.uneven_instances(count=4)
    for s in specs[:2]:
        small = inputs.InstanceSpec(s.index, 64, s.replicas, s.kind, s.seed)
        J = _np(inputs.instance_coupling_torch(small, device="cpu"))
        off = J[np.triu_indices(64, 1)]
        if s.kind == "pm1":
            assert set(np.unique(off).tolist()) <= {-1.0, 1.0}
        else:
            assert np.array_equal(J, inputs.round_to_bf16(J)) and len(np.unique(off)) > 100
