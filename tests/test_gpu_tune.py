"""The slice-count tuner (st_tune_slicing): the fastest discretisation whose
one-turn spin error Delta S (Sec. 5.3) on a sample stays within a bound, as
the paper chooses n_b and the Romberg order against a finely sliced
reference (Sec. 5.2.1, 5.3).  Checked against the oracle: the chosen
candidate's error recomputed by the oracle is within the bound, every
candidate row's error matches the oracle's, and no faster candidate in the
table meets the bound."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

pytestmark = pytest.mark.gpu


def oracle_dS(ring, z, S, nb, K, Sref):
    _, S1, l1 = oracle.track(W.with_slices(ring, nb), z, S, 1, K)
    ok = ~l1.astype(bool)
    return np.linalg.norm(S1 - Sref, axis=0)[ok].mean()


@pytest.mark.parametrize("bound", [1e-6, 1e-8])
def test_tuner_meets_the_bound_at_the_fastest_candidate(bound):
    gg = 45.5
    ring = W.rhic_like_ring(gg, n_cells=12)
    z, S = W.gaussian_particles(256, gg, seed=21)
    r = st.st_tune_slicing(ring, z, S, bound)
    table = r["table"]
    assert table.shape == (st.ST_TUNE_MAX_CANDIDATES, 4)
    _, Sref, _ = oracle.track(W.with_slices(ring, st.ST_TUNE_REF_SLICES), z, S, 1, st.ST_TUNE_REF_ORDER)
    for nb, K, dS, ms in table[::5]:
        assert abs(dS - oracle_dS(ring, z, S, int(nb), int(K), Sref)) < 1e-11 + 1e-9 * dS
    assert r["dS"] <= bound
    assert oracle_dS(ring, z, S, r["n_slices"], r["spin_order"], Sref) <= bound * (1 + 1e-6) + 1e-12
    ok = table[:, 2] <= bound
    assert ok.any() and np.all(table[ok, 3] >= r["ms"])
    # with Romberg iterations the bound is met with fewer slices than by the
    # trapezoid rule alone
    pwc = table[(table[:, 1] == 0) & ok]
    assert r["spin_order"] > 0
    assert pwc.size == 0 or r["n_slices"] < pwc[:, 0].min()


def test_tuner_rejects_bad_arguments():
    ring = W.toy_ring(45.5)
    z, S = W.gaussian_particles(16, 45.5, seed=1)
    with pytest.raises(st.SpinTrackError):
        st.st_tune_slicing(ring, z, S, 0.0)
