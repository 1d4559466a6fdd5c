"""The paper's orbital-error statements (Sec. 5.1, Figs. oneTurnErrsX and
xErrVsTurnNo) reproduced with the oracle on the RHIC-scale ring with thin
sextupoles (claims in tests/orbit_error_claims.py)."""
import oracle
import numpy as np

from orbit_error_claims import (check_amplitude_dependence, check_errors_over_turns, check_one_turn_errors,
                               check_tunes)


def test_one_turn_orbit_errors():
    check_one_turn_errors(oracle.track)


def test_orbit_errors_over_turns():
    check_errors_over_turns(oracle.track)


def test_orbit_error_amplitude_dependence():
    check_amplitude_dependence(oracle.track)


def _oracle_jacobian(ring):
    """Exact one-turn Jacobian at z = 0 by complex-step differentiation."""
    J = np.zeros((6, 6))
    for j in range(6):
        zc = np.zeros(6, dtype=np.complex128)
        zc[j] = 1e-30j
        for e in ring["elements"]:
            zc, rc = oracle.orbit_map(e, ring["G"], ring["Ggamma0"], zc, variant="c128")
            assert rc == 0
        J[:, j] = zc.imag / 1e-30
    return J


def test_tunes_need_no_fit_with_bend_kick_matrix_kick():
    check_tunes(_oracle_jacobian, 1e-12)
