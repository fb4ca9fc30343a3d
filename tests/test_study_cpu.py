"""Host logic of the synthetic studies (schedules, CDFs, summaries)."""
import numpy as np

from paper_2305_07187_gb300 import inputs, schedule, study


def test_zeta_strategies():
    T = 2000
    z = study.zeta_strategies(T, tuned_knots=np.array([0.01, 0.3, 0.6]))
    assert set(z) == set(study.STRATEGIES) | {"tuned"}
    for v in z.values():
        assert v.shape == (T,) and v.dtype == np.float32
    assert (z["fixed-0.8z0"] == np.float32(0.04)).all() and (z["fixed-10z0"] == np.float32(0.5)).all()
    np.testing.assert_array_equal(z["ramp-L1"], inputs.zeta_ramp(T))
    for L in (200, 1000):
        v = z["ramp-L%d" % L]
        levels = np.unique(v)
        assert levels.size == -(-T // L)
        assert v[0] == np.float32(0.04) and v[-1] == np.float32(0.5)
        assert (np.diff(v) >= 0).all() and (v[:L] == v[0]).all()
    np.testing.assert_array_equal(z["tuned"], schedule.expand([0.01, 0.3, 0.6], T))


def test_empirical_cdf_and_summary():
    x, F = study.empirical_cdf([3, 1, 2, 2])
    np.testing.assert_array_equal(x, [1, 2, 2, 3])
    np.testing.assert_allclose(F, [0.25, 0.5, 0.75, 1.0])
    s = study.summarize(np.arange(1, 102))
    assert s["best"] == 101 and s["median"] == 51 and s["count"] == 101
    assert s["p10"] == 11 and s["p90"] == 91


def test_king_graph_generator():
    L = 7
    J = inputs.king_graph_coupling(L, seed=3)
    assert np.array_equal(J, J.T) and not np.diag(J).any()
    assert set(np.unique(J)) <= {-1.0, 0.0, 1.0}
    deg = (J != 0).sum(1).reshape(L, L)
    assert deg[0, 0] == 3 and deg[0, 3] == 5 and deg[3, 3] == 8
    # couplings only between king-move neighbours
    i, j = np.nonzero(J)
    assert (np.maximum(np.abs(i // L - j // L), np.abs(i % L - j % L)) == 1).all()
