"""The paper's orbital-error statements (Sec. 5.1, Figs. oneTurnErrsX and
xErrVsTurnNo) reproduced with the oracle on the RHIC-scale ring with thin
sextupoles (claims in tests/orbit_error_claims.py)."""
import oracle
from orbit_error_claims import check_amplitude_dependence, check_errors_over_turns, check_one_turn_errors


def test_one_turn_orbit_errors():
    check_one_turn_errors(oracle.track)


def test_orbit_errors_over_turns():
    check_errors_over_turns(oracle.track)


def test_orbit_error_amplitude_dependence():
    check_amplitude_dependence(oracle.track)
