"""The study helpers on the GPU: final cuts are the exact cuts of the GPU's
own spins, and the segmented energy trajectory ends in the same state as a
single run (resuming from the full FP32 state changes nothing)."""
import numpy as np
import pytest

from _helpers import b, inputs, oracle
from paper_2305_07187_gb300 import study

pytestmark = pytest.mark.gpu


def test_final_cuts_are_exact_cuts_of_the_spins():
    n, R, T = 200, 32, 100
    J = inputs.pm1_coupling(n, seed=90)
    q0 = inputs.positions(n, R, seed0=9000)
    for name, z in study.zeta_strategies(T).items():
        cuts, s = study.final_cuts(J, q0, z, inputs.dt_const(T))
        np.testing.assert_array_equal(cuts, oracle.cut(J, s).astype(np.int64))


@pytest.mark.parametrize("variant", [{}, {"update_order": 1}, {"wall_zero_p": 1}, {"q_max": 1.0}])
def test_segmented_trajectory_matches_one_run(variant):
    n, R, T, every = 257, 20, 60, 20
    J = inputs.pm1_coupling(n, seed=91)
    q0 = inputs.positions(n, R, seed0=9100)
    zeta, dt = inputs.zeta_ramp(T), inputs.dt_const(T)
    steps, E, s_seg = study.energy_trajectory(J, q0, zeta, dt, every, **variant)
    assert list(steps) == [20, 40, 60] and E.shape == (3, R)
    _, s_one = study.final_cuts(J, q0, zeta, dt, **variant)
    np.testing.assert_array_equal(s_seg, s_one)
    np.testing.assert_array_equal(E[-1], oracle.energy(J, None, s_one).astype(np.int64))
