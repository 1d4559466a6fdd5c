"""The paper's orbital-error statements (Sec. 5.1) through the CUDA tracker:
the tracked runs on the GPU, the references on the oracle, and the one-turn
errors equal to the oracle's own up to rounding (a relative Delta X of 5e-9
is about 5e-12 m on this 1 mm beam, the FP64 noise of a turn through 1728
bend slices)."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
from orbit_error_claims import (check_amplitude_dependence, check_errors_over_turns, check_one_turn_errors,
                               check_tunes)

pytestmark = pytest.mark.gpu


def test_one_turn_orbit_errors_on_the_gpu():
    g = check_one_turn_errors(st.track)
    o = check_one_turn_errors(oracle.track)
    for k in g:
        assert abs(g[k] - o[k]) < 1e-6 * o[k] + 5e-9, k


def test_orbit_errors_over_turns_on_the_gpu():
    check_errors_over_turns(st.track)


def test_orbit_error_amplitude_dependence_on_the_gpu():
    check_amplitude_dependence(st.track)


def _gpu_jacobian(ring, h=1e-7):
    """One-turn Jacobian at z = 0 by central differences of CUDA-tracked
    orbits (12 particles, one turn)."""
    n = 12
    z = np.zeros((6, n))
    for j in range(6):
        z[j, 2 * j], z[j, 2 * j + 1] = h, -h
    S = np.tile(np.array([[0.0], [1.0], [0.0]]), (1, n))
    z1, _, lost = st.track(ring, z, S, 1, 0)
    assert not lost.any()
    return np.stack([(z1[:, 2 * j] - z1[:, 2 * j + 1]) / (2 * h) for j in range(6)], axis=1)


def test_tunes_need_no_fit_with_bend_kick_matrix_kick_on_the_gpu():
    check_tunes(_gpu_jacobian, 1e-7)
