"""Pins of the oracle on sheared (triclinic) cells, ahead of a triclinic GPU path.

* The NaCl Madelung constant (golden file) from the two-ion rhombohedral primitive
  cell of rock salt, whose lattice vectors are not orthogonal.
* The same crystal described by two cells related by a unimodular change of basis
  (rows a1, a2 + a1, a3 instead of a1, a2, a3) gives the same force call: energy,
  forces, virial, charges and Born effective charges, Ewald in modes 1 and 2.
"""
import math
import os

import numpy as np
import pytest

from oracle import ewald, forcecall, geometry
from paper_2601_19034_gb300 import workloads as wl

KE = 14.3996454784
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_madelung_constant_from_the_primitive_rhombohedral_cell():
    rows = [ln for ln in open(os.path.join(GOLDEN, "madelung_nacl.txt")) if ln.strip() and not ln.startswith("#")]
    m_ref = float(rows[0].split()[0])
    a = 5.64
    box = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])   # fcc primitive vectors
    pos = np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.0, 0.0]])
    q = np.array([1.0, -1.0])
    alpha, rc = 0.8, 6.0
    elec = wl.Elec(mode=1, alpha=alpha, rc_real=rc, kmax=2 * alpha * math.sqrt(math.log(1e18)))
    ent = geometry.neighbor_entries(pos, box, rc)
    out = ewald.ewald_static(pos, box, q, ent, elec)
    e = out["e_real"] + out["e_kspace"] + out["e_self"]
    madelung = -e / (KE / (a / 2))
    assert abs(madelung - m_ref) < 2e-6
    assert np.abs(out["force"]).max() < 1e-9


@pytest.mark.parametrize("mode", [1, 2])
def test_unimodular_change_of_cell_leaves_the_force_call_unchanged(mode):
    s = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(32))[0]
    elec = wl.Elec(mode=mode, kind="ewald")
    pos = s.positions.astype(np.float64)
    ortho = s.box
    sheared = ortho.copy()
    sheared[1] = ortho[1] + ortho[0]          # same lattice, non-orthogonal rows
    a = forcecall.force_call(pos, ortho, s.types, hp, blob, elec)
    b = forcecall.force_call(pos, sheared, s.types, hp, blob, elec)
    assert abs(a["energy"] - b["energy"]) < 1e-9 * max(1.0, abs(a["energy"]))
    for key, tol in (("forces", 1e-9), ("charges", 1e-12), ("bec", 1e-9), ("virial", 1e-8)):
        np.testing.assert_allclose(b[key], a[key], atol=tol * max(1.0, np.abs(a[key]).max()))
