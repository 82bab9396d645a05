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
import torch

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


def _sheared_water(seed=2):
    """64 H2O at the fractional coordinates of the cubic box in a cell with every off-diagonal
    element non-zero, partial charges summing to zero."""
    s = wl.water_box(4, seed=seed)
    length = s.box[0, 0]
    box = length * np.array([[1.0, 0.05, -0.04], [0.2, 1.0, 0.06], [-0.1, 0.15, 1.0]])
    pos = (s.positions.astype(np.float64) / length) @ box
    rng = np.random.default_rng(seed)
    q = np.tile([0.8, -0.4, -0.4], len(pos) // 3) + rng.normal(0, 0.05, len(pos))
    return pos, box, q - q.mean()


def test_pppm_in_a_general_cell_converges_to_ewald():
    """The fractional-mesh PPPM of a sheared cell against the general-cell Ewald sum (pinned above
    by the rhombohedral Madelung constant and the unimodular change of cell): mesh spacing below
    0.9 A along every lattice vector with P = 5 reaches the ~1e-4 relative accuracy of Sec. II.F,
    for the forces, U^k and the k-space virial."""
    from oracle import pppm
    pos, box, q = _sheared_water()
    alpha = 0.3
    ent = geometry.neighbor_entries(pos, box, 6.0)
    full = ewald.ewald_static(pos, box, q, ent, wl.Elec(mode=1, alpha=alpha,
                                                        kmax=2 * alpha * math.sqrt(math.log(1e14))))
    real = ewald.ewald_static(pos, box, q, ent, wl.Elec(mode=1, alpha=alpha), with_kspace=False)
    mesh = [int(math.ceil(np.linalg.norm(box[d]) / 0.9)) for d in range(3)]
    mesh = tuple(m + m % 2 for m in mesh)
    out = pppm.pppm(pos, box, q, mesh, 5, alpha)
    k_force = full["force"] - real["force"]
    fnorm = np.sqrt((full["force"] ** 2).sum(1).mean())
    err = np.sqrt(((out["force"] - k_force) ** 2).sum(1).mean())
    assert err / fnorm < 3e-4, err / fnorm
    assert abs(out["e_kspace"] - full["e_kspace"]) < 1e-4 * abs(full["e_real"] + full["e_kspace"])
    np.testing.assert_allclose(out["virial"], full["virial"] - real["virial"], atol=2e-3 * np.abs(full["virial"]).max())
    # the diagonal special case of the general code is the orthorhombic one
    cube = np.diag(np.diag(box))
    pc = pos @ np.linalg.inv(box) @ cube
    a = pppm.pppm(pc, cube, q, mesh, 5, alpha)
    b = pppm.pppm_general(pc, cube, q, mesh, 5, alpha)
    for key in ("e_kspace", "phi", "force", "virial"):
        np.testing.assert_allclose(b[key], a[key], rtol=1e-10, atol=1e-10)


def test_pppm_in_a_general_cell_energy_identity_and_mesh_virial():
    """U^k = 1/2 sum q phi, phi = dU^k/dq by finite differences, and the per-atom mesh virial of
    the six inverse FFTs sums to the total k-space virial, in the sheared cell."""
    from oracle import pppm, virial
    pos, box, q = _sheared_water(seed=3)
    mesh = (16, 16, 16)
    out = pppm.pppm(pos, box, q, mesh, 5, 0.3)
    assert abs(out["e_kspace"] - 0.5 * (q * out["phi"]).sum()) < 1e-10 * abs(out["e_kspace"])
    h = 1e-5
    for i in (0, 7, 100):
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (pppm.pppm(pos, box, qp, mesh, 5, 0.3)["e_kspace"] - pppm.pppm(pos, box, qm, mesh, 5, 0.3)["e_kspace"]) / (2 * h)
        assert abs(fd - out["phi"][i]) < 1e-6
    w = virial.kspace_static_pppm(pos, box, q, mesh, 5, 0.3)
    np.testing.assert_allclose(w.sum(0), out["virial"], rtol=1e-10, atol=1e-10 * np.abs(out["virial"]).max())


@pytest.mark.parametrize("mode", [1, 2])
def test_virial_and_forces_in_a_general_cell_match_finite_differences(mode):
    """In a fully sheared cell the force call's virial is -dU/d eps under the homogeneous strain of
    positions and cell (central differences, +-1e-6) and its forces are -dU/dr (central
    differences, 1e-4 A), Ewald modes 1 and 2: the general-cell images, k = 2 pi H^-1 n and the
    volume enter both."""
    s0 = wl.batio3_supercell(2, seed=41)
    box = s0.box + np.array([[0.0, 0.4, -0.3], [0.7, 0.0, 0.5], [-0.6, 0.8, 0.0]])
    pos = (s0.positions.astype(np.float64) @ np.linalg.inv(s0.box)) @ box
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(42))[0]
    elec = wl.Elec(mode=mode, kind="ewald", q_total=0.2)
    out = forcecall.force_call(pos, box, s0.types, hp, blob, elec, want_bec=False)

    def energy(p, b):
        with torch.no_grad():
            e, _, _ = forcecall.total_energy_autograd(p, b, s0.types, hp, blob, elec)
        return float(e)

    h = 1e-6
    for a, b in ((0, 0), (2, 2), (0, 1), (1, 2), (2, 0)):
        eps = np.zeros((3, 3))
        eps[a, b] = h
        dp, dm = np.eye(3) + eps, np.eye(3) - eps
        w = -(energy(pos @ dp.T, box @ dp.T) - energy(pos @ dm.T, box @ dm.T)) / (2 * h)
        assert abs(w - out["virial"][b, a]) < 1e-4 * max(1.0, abs(out["virial"][b, a])), (a, b)
    hr = 1e-4
    for i, d in ((0, 0), (7, 1), (23, 2)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += hr
        pm[i, d] -= hr
        f = -(energy(pp, box) - energy(pm, box)) / (2 * hr)
        assert abs(f - out["forces"][i, d]) < 1e-5 * max(1.0, abs(f)), (i, d)


@pytest.mark.parametrize("kind,mode", [("ewald", 1), ("ewald", 2), ("pppm", 1)])
def test_turning_the_structure_with_its_cell_turns_every_output(kind, mode):
    """Rotation covariance of the whole force call, a fact of the physics rather than of any code:
    turning the atoms and the cell's rows by one rotation R leaves the energy and the charges as
    they were and turns the forces (R F_i), the virial (R W R^T), the Born effective charges
    (R Z_i R^T) and the polarization (R P).  The turned cell has no zero entry, so the general-cell
    k-set (Ewald) and the mesh along the lattice vectors (PPPM) run in full; Q != 0 keeps the
    charge correction in play."""
    s = wl.batio3_supercell(2, seed=35)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(36))[0]
    extra = {"mesh": (12, 12, 12)} if kind == "pppm" else {}
    elec = wl.Elec(mode=mode, kind=kind, q_total=0.3, **extra)
    box = s.box.copy()
    box[1, 0], box[2, 0], box[2, 1] = 0.9, -0.6, 0.7          # a sheared cell in the restricted form
    pos = (s.positions.astype(np.float64) / s.box[0, 0]) @ box
    rng = np.random.default_rng(37)
    r, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(r) < 0:
        r[:, 0] = -r[:, 0]                                     # a proper rotation
    a = forcecall.force_call(pos, box, s.types, hp, blob, elec)
    b = forcecall.force_call(pos @ r.T, box @ r.T, s.types, hp, blob, elec)
    assert np.abs(box @ r.T).min() > 1e-3                      # every entry of the turned cell non-zero
    assert abs(b["energy"] - a["energy"]) < 1e-9 * max(1.0, abs(a["energy"]))
    np.testing.assert_allclose(b["charges"], a["charges"], atol=1e-12)
    scale = lambda x: max(1.0, np.abs(x).max())               # noqa: E731
    np.testing.assert_allclose(b["forces"], a["forces"] @ r.T, atol=1e-9 * scale(a["forces"]))
    np.testing.assert_allclose(b["virial"], r @ a["virial"] @ r.T, atol=1e-9 * scale(a["virial"]))
    np.testing.assert_allclose(b["bec"], np.einsum("ab,ibc,dc->iad", r, a["bec"], r), atol=1e-9 * scale(a["bec"]))
    np.testing.assert_allclose(b["polarization"], r @ a["polarization"], atol=1e-9 * scale(a["polarization"]))
