"""The paper's orbital-error statements (Sec. 5.1) through the CUDA tracker:
the tracked runs on the GPU, the references on the oracle, and the one-turn
errors equal to the oracle's own up to rounding (a relative Delta X of 5e-9
is about 5e-12 m on this 1 mm beam, the FP64 noise of a turn through 1728
bend slices)."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
from orbit_error_claims import check_amplitude_dependence, check_errors_over_turns, check_one_turn_errors

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
