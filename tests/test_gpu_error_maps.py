"""The paper's single-element error maps (Sec. 5.2.1) through the CUDA
tracker: the same statements as tests/test_oracle_error_maps.py with the
maps' runs on the GPU (the reference runs stay on the oracle), and the maps
equal to the oracle's own maps to 1e-11."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
from error_map_claims import check_dipole_maps, check_quad_maps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Py,Pt", [(0.0, 0.0), (2e-4, 0.0), (0.0, 2e-4)])
def test_dipole_error_maps_on_the_gpu(Py, Pt):
    g = check_dipole_maps(st.track, Py, Pt)
    o = check_dipole_maps(oracle.track, Py, Pt)
    for key in g:
        assert np.abs(g[key] - o[key]).max() < 1e-11


@pytest.mark.parametrize("alpha", [0, 20, 180])
def test_ir_quad_error_maps_on_the_gpu(alpha):
    g = check_quad_maps(st.track, alpha)
    o = check_quad_maps(oracle.track, alpha)
    for key in g:
        assert np.abs(g[key] - o[key]).max() < 1e-11
