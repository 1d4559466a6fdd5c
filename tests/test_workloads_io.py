"""The lattice description file (JSON) round-trips every element kind and
field, rejects unknown types and fields, and a loaded ring tracks exactly as
the ring it was written from (CPU oracle)."""
import json

import numpy as np
import pytest

import oracle
import workloads as W


def _mixed_ring():
    ring = W.with_fringes(W.with_split_order(W.with_spin_order(W.toy_ring(45.5, n_cells=2), 2), 4))
    ring["elements"] += [W.element("solenoid", L=2.0, n_slices=4, k1=0.05),
                         W.element("rbend", L=2.5, n_slices=4, angle=0.05, e1=0.01, fringe=1),
                         W.element("snake", snake_phi=0.7, snake_mu=np.pi),
                         W.element("teapot", L=3.0, n_slices=4, angle=0.05, eta=0.99, split_order=4),
                         W.element("thin_mult", n_slices=4, k1=0.01, k2=0.4)]
    return ring


def test_round_trip_and_identical_tracking(tmp_path):
    ring = _mixed_ring()
    p = tmp_path / "ring.json"
    W.save_ring(ring, str(p))
    back = W.load_ring(str(p))
    assert back["G"] == ring["G"] and back["Ggamma0"] == ring["Ggamma0"]
    assert back["elements"] == ring["elements"]
    z, S = W.gaussian_particles(20, 45.5, seed=9)
    a = oracle.track(ring, z, S, 2, 2)
    b = oracle.track(back, z, S, 2, 2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_hand_written_file_with_defaults(tmp_path):
    p = tmp_path / "ring.json"
    p.write_text(json.dumps({"format": W.RING_FORMAT, "G": W.G_PROTON, "Ggamma0": 45.5,
                             "elements": [{"type": "drift", "L": 1.0},
                                          {"type": "quad_mk", "L": 1.0, "n_slices": 4, "k1": 0.03}]}))
    r = W.load_ring(str(p))
    assert r["elements"][1]["split_order"] == 2 and r["elements"][0]["fringe"] == 0


@pytest.mark.parametrize("bad", [{"type": "wiggler", "L": 1.0}, {"type": "drift", "L": 1.0, "colour": "red"}])
def test_rejects_unknown_types_and_fields(tmp_path, bad):
    p = tmp_path / "ring.json"
    p.write_text(json.dumps({"format": W.RING_FORMAT, "G": W.G_PROTON, "Ggamma0": 45.5, "elements": [bad]}))
    with pytest.raises((ValueError, TypeError)):
        W.load_ring(str(p))
