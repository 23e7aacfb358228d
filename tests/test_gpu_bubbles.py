"""GPU vs oracle: bubble regions (§3.1) and the jet pulse.

lbdps_bubbles labels the regions of high voidage on the device (union-find);
the oracle floods them on the host.  Both start from the same particle
positions, so the cell counts and therefore the regions are identical:
compared exactly.  The pulse check runs a Table 1 bed with the jet on, turns
it off with lbdps_set_inlet, and compares the state with the oracle's.
"""
import math
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from oracle import oracle as O                      # noqa: E402
from paper_1303_2653_gb300 import workloads as W    # noqa: E402
from test_oracle_pins import _counted_bed, _counted_bed3d  # noqa: E402

pytestmark = pytest.mark.gpu


def _lb():
    from paper_1303_2653_gb300 import lbdps as L
    return L


def test_bubbles_of_a_designed_bed_on_gpu():
    L = _lb()
    counts = np.full((24, 12), 16)
    counts[-5:, :] = 0
    counts[6:9, 4:7] = 0
    counts[0, 9:11] = 0
    bed = L.Bed(_counted_bed(counts, storage=W.STORE_F32))
    assert bed.bubbles(0.85, L.VOIDAGE_2D) == {"largest": 9, "count": 2, "cells": 11}
    bed.close()


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_bubbles_match_oracle(seed):
    L = _lb()
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 17, size=(40, 20))
    counts[rng.random(counts.shape) < 0.4] = 0
    w = _counted_bed(counts, storage=W.STORE_F32)
    bed = L.Bed(w)
    ob = O.OracleBed(w)
    for thr, v in [(0.85, L.VOIDAGE_2D), (0.6, L.VOIDAGE_2D), (0.97, L.VOIDAGE_G)]:
        assert bed.bubbles(thr, v) == ob.bubbles(thr, v)
    bed.close()


@pytest.mark.parametrize("seed,periodic_x", [(4, False), (6, True), (7, True)])
def test_bubbles_3d_match_oracle(seed, periodic_x):
    # 3D: face neighbours along x, y and z, z vertical, the x face wrapping
    L = _lb()
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 28, size=(12, 10, 11))
    counts[rng.random(counts.shape) < 0.1] = 0
    w = _counted_bed3d(counts, periodic_x, storage=W.STORE_F32)
    bed = L.Bed(w)
    ob = O.OracleBed(w)
    for thr in (0.99, 0.985, 0.975, 0.9):
        got = bed.bubbles(thr, L.VOIDAGE_G)
        assert got == ob.bubbles(thr, L.VOIDAGE_G)
    bed.close()


def test_bubbles_after_steps_match_oracle():
    # a moving bed: the regions of the GPU cell list equal the oracle's
    L = _lb()
    w = W.bubbling_table1(nx=25, ny=40, n_particles=1500, bed_rows=18, storage=W.STORE_F64)
    bed = L.Bed(w, storage=W.STORE_F64)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    P, v = bed.particles()
    ob.set_particles(P, v)
    for _ in range(3):
        bed.step(2)
        ob.step(2)
        for thr in (0.85, 0.7):
            assert bed.bubbles(thr, L.VOIDAGE_2D) == ob.bubbles(thr, L.VOIDAGE_2D)
    bed.close()


def test_jet_pulse_with_set_inlet_matches_oracle():
    # §3.1: the jet lasts a while, then the inlet returns to the background
    # velocity; the change must reach the captured step graphs
    L = _lb()
    w = W.bubbling_table1(nx=25, ny=40, n_particles=1500, bed_rows=18, storage=W.STORE_F64,
                          v_inj=4.0)
    bed = L.Bed(w, storage=W.STORE_F64)
    ob = O.OracleBed(w)
    ob.set_populations(bed.populations())
    P, v = bed.particles()
    ob.set_particles(P, v)
    bed.step(4)
    ob.step(4)
    bg = W.background_inlet(w)
    bed.set_inlet(bg)
    ob.set_inlet(bg)
    bed.step(4)
    ob.step(4)
    fo, fg = ob.populations(), bed.populations()
    assert np.abs(fg - fo).max() <= 1e-13
    Pg, _ = bed.particles()
    Po, _ = ob.particles()
    assert np.abs(Pg - Po).max() <= 1e-10
    # and the pulse did change the state: a bed kept on the jet differs
    keep = L.Bed(w, storage=W.STORE_F64)
    keep.step(8)
    assert np.abs(keep.populations() - fg).max() > 1e-8
    keep.close()
    bed.close()


def test_set_inlet_rejects_bad_input():
    L = _lb()
    w = W.bubbling_table1(nx=25, ny=40, n_particles=100, bed_rows=18)
    bed = L.Bed(w)
    with pytest.raises(L.LbdpsError):
        bed.set_inlet(np.full_like(w.inlet_u, 1e3))   # far above 0.3 in lattice units
    riser = L.Bed(W.scaled_riser2d(nx=32, ny=64))
    with pytest.raises(L.LbdpsError):
        riser.set_inlet(np.zeros((32, 2)))           # no inlet face
    with pytest.raises(L.LbdpsError):
        bed.bubbles(1.5)
    riser.close()
    bed.close()
