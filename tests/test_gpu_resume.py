"""Checkpoint/resume and the failure path of the device-side bounded waits.

Resume: the state between launches is the FP64 orbit, the spins and the lost
flags; downloading it after n1 turns and uploading it (lost flags included)
into a fresh context gives, after n2 more turns, bit for bit the state of
n1 + n2 turns tracked in one context.

Bounded waits: a block waits on a barrier that nothing completes; the wait
gives up after its limit, the call returns ST_ETIMEOUT, and the GPU context
stays usable (no fault, no hang)."""
import numpy as np
import pytest

import oracle
import paper_1501_03450_b300 as st
import workloads as W

pytestmark = pytest.mark.gpu


def _ensemble():
    z, S = W.gaussian_particles(300, 45.5, seed=41)
    z[1, 11] = 0.9      # lost in the first quadrupole of the first turn
    z[3, 200] = -0.95
    return z, S


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_is_bit_identical(precision):
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = _ensemble()
    lat = st.Lattice(ring)
    full = st.Tracker(lat, z.shape[1], precision)
    full.set_launch(turns_per_launch=1)
    full.upload(z, S)
    full.track(7, 2)
    zf, Sf, lf = full.download()
    full.close()

    a = st.Tracker(lat, z.shape[1], precision)
    a.set_launch(turns_per_launch=1)
    a.upload(z, S)
    a.track(3, 2)
    zc, Sc, lc = a.download()
    a.close()
    assert lc[11] == 1 and lc[200] == 1
    b = st.Tracker(lat, z.shape[1], precision)
    b.set_launch(turns_per_launch=1)
    b.upload(zc, Sc)
    b.upload_lost(lc)
    b.track(4, 2)
    zr, Sr, lr = b.download()
    b.close()
    assert np.array_equal(lr, lf)
    assert np.array_equal(zr, zf) and np.array_equal(Sr, Sf)

    # uploaded flags take effect: a healthy particle flagged lost stays frozen
    flags = lc.copy()
    flags[5] = 1
    c = st.Tracker(lat, z.shape[1], precision)
    c.set_launch(turns_per_launch=1)
    c.upload(zc, Sc)
    c.upload_lost(flags)
    c.track(4, 2)
    zn, Sn, ln = c.download()
    c.close()
    lat.close()
    assert ln[5] == 1 and np.array_equal(zn[:, 5], zc[:, 5]) and np.array_equal(Sn[:, 5], Sc[:, 5])
    assert not np.array_equal(zf[:, 5], zc[:, 5])


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    rc, elapsed = st.st_selftest_bounded_wait(0.02)
    assert rc == st.ST_ETIMEOUT
    assert 0.02 <= elapsed < 0.5, elapsed
    assert "gave up" in st.last_error()
    # the GPU context still tracks correctly afterwards
    ring = W.with_spin_order(W.toy_ring(45.5), 2)
    z, S = W.gaussian_particles(64, 45.5, seed=42)
    zg, Sg, lg = st.track(ring, z, S, 3, 2)
    zo, So, lo = oracle.track(ring, z, S, 3, 2)
    assert np.array_equal(lg, lo)
    assert np.abs(zg - zo).max() < 1e-11 and np.abs(Sg - So).max() < 1e-11


def test_lost_upload_needs_an_upload_first():
    lat = st.Lattice(W.with_spin_order(W.toy_ring(45.5), 2))
    t = st.Tracker(lat, 8)
    with pytest.raises(st.SpinTrackError):
        t.upload_lost(np.zeros(8, np.uint8))
    t.close()
    lat.close()
