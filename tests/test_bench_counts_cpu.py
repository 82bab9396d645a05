"""The benchmark's algorithmic work count (the roofline's numerator) on the CPU: the per-(atom,
candidate) formula written out by hand for one cubic cell, its half-space k count against the
oracle's full-sphere enumeration, and the count of a sheared cell equal to that of the orthorhombic
cell it is a unimodular transform of (same density, same wave vectors)."""
import math
import os
import sys

import numpy as np

from oracle import ewald
from paper_2601_19034_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_batch_flop_by_hand_for_one_cell():
    systems, hp, _, elec = wl.config_llzo_batch(n_struct=1, n_candidates=1)
    s = systems[0]
    lengths = np.diag(s.box)
    rho = s.n_atoms / float(np.prod(lengths))
    n_r = 4.0 / 3.0 * math.pi * 6.0 ** 3 * rho
    n_a = 4.0 / 3.0 * math.pi * 4.0 ** 3 * rho
    nk = len(ewald.kspace_integers(s.box, elec.kmax)) // 2
    per = (2 * 4 * (9 * 5 + 9 * 5 * 24) + 6 * 30 * 30 + 24 * n_r + 840 * n_a + 8 * n_r + 14 * nk)
    assert abs(bench._batch_flop(systems, hp, elec, 64) - s.n_atoms * 64 * per) < 1e-6 * s.n_atoms * 64 * per
    assert bench._ewald_kcount(s.box, elec.kmax) == nk


def test_batch_flop_of_a_unimodular_cell_equals_the_orthorhombic_one():
    systems, hp, _, elec = wl.config_llzo_batch(n_struct=1, n_candidates=1)
    s = systems[0]
    sheared = s.box.copy()
    sheared[1] = s.box[1] + s.box[0]
    sheared[2] = s.box[2] + s.box[1]
    t = wl.System(s.positions, s.types, sheared, s.species)
    assert bench._ewald_kcount(sheared, elec.kmax) == bench._ewald_kcount(s.box, elec.kmax)
    a = bench._batch_flop([s], hp, elec, 64)
    b = bench._batch_flop([t], hp, elec, 64)
    assert abs(a - b) < 1e-9 * a
