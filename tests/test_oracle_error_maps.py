"""The paper's single-element error maps (Sec. 5.2.1, Figs. sbendErrsQ/R,
sbendErrsQR4M/QR8M, quadErrs48QR) reproduced with the oracle: the
statements the paper makes about them (ranges, Romberg lowering the error
throughout phase space, the PWC valley on the locus of Eq. (dpx0), the
vertical-spin pattern of the IR quadrupole) hold for the oracle's results."""
import pytest

import oracle
from error_map_claims import check_dipole_maps, check_quad_maps


@pytest.mark.parametrize("Py,Pt", [(0.0, 0.0), (2e-4, 0.0), (0.0, 2e-4), (-2e-4, -2e-4)])
def test_dipole_error_maps(Py, Pt):
    check_dipole_maps(oracle.track, Py, Pt)


@pytest.mark.parametrize("alpha", [0, 20, 180])
def test_ir_quad_error_maps(alpha):
    check_quad_maps(oracle.track, alpha)
