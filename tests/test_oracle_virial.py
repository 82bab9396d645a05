"""Pins of the oracle's per-atom virial (Eq. per-atom_virial, Sec. II.C; the mesh form of Sec. II.F).

The sum over atoms equals the force call's total virial, which test_oracle_forces.py
pins by finite differences of the energy under strain; the per-atom virial is
unchanged by a uniform translation; and a 2 x 2 x 2 replica of a cell has, atom by
atom, the virials of the cell (the split among atoms is local).
"""
import numpy as np
import pytest

from oracle import virial
from paper_2601_19034_gb300 import workloads as wl


@pytest.fixture(scope="module")
def cell():
    s = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(32))[0]
    return s.positions.astype(np.float64), s.box, s.types, hp, blob


@pytest.mark.parametrize("elec", [wl.Elec(mode=1, kind="ewald"), wl.Elec(mode=2, kind="ewald"),
                                  wl.Elec(mode=1, kind="pppm", mesh=(16, 16, 16), order=5)],
                         ids=["ewald-mode1", "ewald-mode2", "pppm"])
def test_per_atom_virial_sums_to_the_total(cell, elec):
    pos, box, types, hp, blob = cell
    w, out = virial.per_atom_virial(pos, box, types, hp, blob, elec)
    scale = max(1.0, np.abs(out["virial"]).max())
    np.testing.assert_allclose(w.sum(0), out["virial"], atol=1e-9 * scale)
    assert np.abs(w).max() > 1e-3            # not trivially zero


def test_kspace_per_atom_sums_to_the_mesh_and_ewald_totals(cell):
    pos, box, types, hp, blob = cell
    q = np.random.default_rng(5).normal(size=len(pos))
    q -= q.mean()
    from oracle import ewald, pppm
    el = wl.Elec(mode=2, kind="ewald")
    tot = ewald.ewald_static(pos, box, q, None, el)["virial"]
    np.testing.assert_allclose(virial.kspace_static_ewald(pos, box, q, el.alpha, el.kmax).sum(0), tot,
                               atol=1e-10 * np.abs(tot).max())
    pm = pppm.pppm(pos, box, q, (16, 16, 16), 5, 0.3)
    np.testing.assert_allclose(virial.kspace_static_pppm(pos, box, q, (16, 16, 16), 5, 0.3).sum(0), pm["virial"],
                               atol=1e-10 * np.abs(pm["virial"]).max())


def test_translation_invariance(cell):
    pos, box, types, hp, blob = cell
    elec = wl.Elec(mode=1, kind="ewald")
    w, _ = virial.per_atom_virial(pos, box, types, hp, blob, elec)
    shifted = (pos + np.array([1.37, -2.11, 0.53])) % 8.0
    w2, _ = virial.per_atom_virial(shifted, box, types, hp, blob, elec)
    np.testing.assert_allclose(w2, w, atol=1e-9 * np.abs(w).max())


def test_replica_has_the_cells_per_atom_virials(cell):
    pos, box, types, hp, blob = cell
    elec = wl.Elec(mode=1, kind="ewald")
    w1, _ = virial.per_atom_virial(pos, box, types, hp, blob, elec)
    shifts = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    big = (pos[None] + shifts[:, None, :] * 8.0).reshape(-1, 3)
    w8, _ = virial.per_atom_virial(big, box * 2, np.tile(types, 8), hp, blob, elec)
    np.testing.assert_allclose(w8, np.tile(w1, (8, 1, 1)), atol=1e-8 * np.abs(w1).max())


def test_energy_moment_identity_fixes_the_convention():
    """Cluster, NEP only (charge head zero): along velocities v,
    d/dt sum_i r_i U_i = sum_i v_i U_i - sum_i r_i (F_i . v_i) + sum_i W_i v_i
    holds exactly for W_i = sum_j r_ij (x) F_ji (it follows from F_i = sum_j (F_ij - F_ji) and
    dU_i/dt = sum_j F_ij . (v_j - v_i)); giving the entry term to atom i instead of j breaks it."""
    from oracle import forcecall
    rng = np.random.default_rng(17)
    pos = rng.uniform(-2.5, 2.5, size=(9, 3)) + 30.0
    types = rng.integers(0, 3, size=9)
    box = np.diag([60.0] * 3)
    hp = wl.HParams(n_species=3)
    blob = wl.scale_charge_head(wl.random_params(hp, np.random.default_rng(18))[0], hp, 0.0).astype(np.float64)
    elec = wl.Elec(mode=2, kind="ewald")
    v = rng.normal(size=pos.shape) * 0.01
    w, out = virial.per_atom_virial(pos, box, types, hp, blob, elec)
    assert np.abs(out["charges"]).max() == 0.0

    def moment(x):
        o = forcecall.force_call(x, box, types, hp, blob, elec, want_bec=False)
        return (x * o["site_energy"][:, None]).sum(0)

    h = 1e-4
    lhs = (moment(pos + h * v) - moment(pos - h * v)) / (2 * h)
    u, f = out["site_energy"], out["forces"]
    rhs = (v * u[:, None]).sum(0) - (pos * (f * v).sum(1)[:, None]).sum(0) + np.einsum("iab,ib->a", w, v)
    np.testing.assert_allclose(rhs, lhs, atol=1e-7)
    # the other assignment of the entry terms (to the central atom) fails the identity
    w_wrong = np.zeros_like(w)
    for ent, g in out["partials"]:
        np.add.at(w_wrong, ent.i, -np.einsum("ea,eb->eab", ent.vec, g))
    rhs_wrong = (v * u[:, None]).sum(0) - (pos * (f * v).sum(1)[:, None]).sum(0) + np.einsum("iab,ib->a", w_wrong, v)
    assert np.abs(rhs_wrong - lhs).max() > 1e-4
