"""GPU force call in general (triclinic) cells, Ewald electrostatics (Sec. II.B with k = 2 pi H^-1 n).

* A sheared 3 x 3 x 3 BaTiO3 cell (every off-diagonal element non-zero) against the FP64 oracle,
  which handles general cells (tests/test_oracle_triclinic.py pins it): energy, forces, charges,
  virial, Born effective charges and polarization at the FP32-path tolerances, modes 1 and 2,
  both kernel families, and the per-atom virial.
* The same crystal described by a unimodularly transformed cell (rows a1, a2 + a1, a3 + a2)
  against the orthorhombic call of the 5 x 5 x 5 cell: the same outputs to FP32 rounding.
* PPPM in general cells (mesh along the lattice vectors, fractional gradients mapped by H^-1):
  the sheared BaTiO3 cell and a sheared 64-water box against the oracle's general-cell PPPM,
  every output including the per-atom virial's mesh term, both kernel families.
* Boxes the library does not take are refused: a left-handed cell, a cell narrower than the
  cutoff, a cell whose Ewald k-set needs more phase factors per atom than the kernels hold; the
  model keeps computing the cell it had.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall, virial  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = dict(e=1e-6, f=1e-4, q=2e-6, w=1e-5, z=1e-4, p=1e-5)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _sheared_batio3(n=3, seed=61):
    """n^3 perovskite cells mapped into a sheared lattice, N(0, 0.05 A) displacements."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0.5], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    frac = ((cells[:, None, :] + basis[None]) / n).reshape(-1, 3)
    a = 4.0 * n
    box = np.array([[a, 0.0, 0.0], [0.9, a, 0.0], [-0.7, 1.1, a]]) + np.array([[0, 0.4, -0.3], [0, 0, 0.5],
                                                                               [0, 0, 0]])
    pos = frac @ box + rng.normal(0.0, 0.05, size=frac.shape)
    types = np.tile(np.array([0, 1, 2, 2, 2], np.int32), n ** 3)
    return wl.System(pos.astype(np.float32), types, box, ("Ba", "Ti", "O"))


def _compute(dev, sysm, hp, params, elec, path="auto", atom_virial=False, potential=False):
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    model = QNEP(hp, params, elec)
    model.set_path(path)
    out = model.compute(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev), sysm.box,
                        atom_virial=atom_virial, potential=potential)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}
    res["sc"] = parse_scalars(out["scalars"])
    model.close()
    return res


@pytest.mark.parametrize("mode,path", [(1, "warp"), (2, "warp"), (1, "thread")])
def test_sheared_cell_against_oracle(dev, mode, path):
    sysm = _sheared_batio3()
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(62))[0]
    elec = wl.Elec(mode=mode, kind="ewald", q_total=0.2)
    g = _compute(dev, sysm, hp, params, elec, path)
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    n = sysm.n_atoms
    de = abs(g["sc"]["energy"] - ref["energy"]) / n
    df = np.abs(g["forces"] - ref["forces"]).max()
    print(f"\nsheared {n} atoms mode {mode} {path}: |dE|/N {de:.3g}, max|dF| {df:.3g}")
    assert de <= TOL["e"], de
    assert df <= TOL["f"], df
    assert np.abs(g["charges"] - ref["charges"]).max() <= TOL["q"]
    assert np.abs(g["sc"]["virial"] - ref["virial"]).max() / n <= TOL["w"]
    assert np.abs(g["bec"] - ref["bec"]).max() <= TOL["z"]
    assert np.abs(g["sc"]["polarization"] - ref["polarization"]).max() / n <= TOL["p"]


def test_sheared_cell_per_atom_virial(dev):
    sysm = _sheared_batio3(seed=63)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(64))[0]
    elec = wl.Elec(mode=1, kind="ewald")
    g = _compute(dev, sysm, hp, params, elec, atom_virial=True)
    ref, _ = virial.per_atom_virial(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    assert np.abs(g["atom_virial"] - ref).max() <= 1e-4


def test_unimodular_change_of_cell_on_the_gpu(dev):
    sysm = wl.batio3_supercell(5, seed=65)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(66))[0]
    for mode in (1, 2):
        elec = wl.Elec(mode=mode, kind="ewald")
        a = _compute(dev, sysm, hp, params, elec)
        sheared = sysm.box.copy()
        sheared[1] = sysm.box[1] + sysm.box[0]
        sheared[2] = sysm.box[2] + sysm.box[1]
        b = _compute(dev, wl.System(sysm.positions, sysm.types, sheared, sysm.species), hp, params, elec)
        n = sysm.n_atoms
        assert abs(a["sc"]["energy"] - b["sc"]["energy"]) / n <= 1e-6
        assert np.abs(a["forces"] - b["forces"]).max() <= 1e-4
        assert np.abs(a["charges"] - b["charges"]).max() <= 2e-6
        assert np.abs(a["sc"]["virial"] - b["sc"]["virial"]).max() / n <= 1e-5
        assert np.abs(a["bec"] - b["bec"]).max() <= 1e-4


def test_boxes_that_are_refused(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    sysm = _sheared_batio3()
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(67))[0]
    pos, typ = torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev)
    m = QNEP(hp, params, wl.Elec(mode=1, kind="ewald"))
    before = parse_scalars(m.compute(pos, typ, sysm.box)["scalars"])["energy"]
    left = sysm.box[[1, 0, 2]]                     # rows swapped: left-handed
    with pytest.raises(_lib.QnepError) as e:
        m.compute(pos, typ, left)
    assert e.value.status == _lib.QNEP_ERR_ARG
    thin = sysm.box.copy()
    thin[1] = sysm.box[1] + 3.0 * sysm.box[0]      # the same volume, a width below 6 A
    with pytest.raises(_lib.QnepError) as e:
        m.compute(pos, typ, thin)
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    big = 12.0 * sysm.box                          # k_max |a_d| / 2 pi ~ 50: over 159 phase factors per atom
    with pytest.raises(_lib.QnepError) as e:
        m.compute(pos, typ, big)
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    # the refusals leave the model's tables alone: the cell it had still computes the same energy
    after = parse_scalars(m.compute(pos, typ, sysm.box)["scalars"])["energy"]
    assert abs(after - before) / sysm.n_atoms <= 1e-6
    m.close()


def _sheared_water(seed=71):
    """64 H2O at the fractional coordinates of the 12.42 A cube in a cell with every off-diagonal
    element non-zero."""
    s = wl.water_box(4, seed=seed)
    length = s.box[0, 0]
    box = length * np.array([[1.0, 0.05, -0.04], [0.2, 1.0, 0.06], [-0.1, 0.15, 1.0]])
    pos = (s.positions.astype(np.float64) / length) @ box
    return wl.System(pos.astype(np.float32), s.types, box, s.species)


@pytest.mark.parametrize("case,mode,path", [("batio3", 1, "warp"), ("batio3", 2, "thread"), ("water", 1, "warp")])
def test_pppm_in_a_general_cell_against_oracle(dev, case, mode, path):
    """The PPPM call in a sheared cell against the oracle's general-cell PPPM (the same scheme):
    energy, forces, charges, virial, BEC, polarization and the potential at the FP32-path
    tolerances (the potential to 1e-5 of its largest value, as for orthorhombic PPPM)."""
    if case == "batio3":
        sysm = _sheared_batio3(seed=72)
        hp = wl.HParams(n_species=3)
        mesh = (16, 16, 16)
    else:
        sysm = _sheared_water()
        hp = wl.HParams(n_species=2)
        mesh = (16, 18, 14)
    params = wl.random_params(hp, np.random.default_rng(73))[0]
    elec = wl.Elec(mode=mode, kind="pppm", mesh=mesh, order=5, q_total=0.2)
    g = _compute(dev, sysm, hp, params, elec, path, potential=True)
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    n = sysm.n_atoms
    de = abs(g["sc"]["energy"] - ref["energy"]) / n
    df = np.abs(g["forces"] - ref["forces"]).max()
    print(f"\nPPPM sheared {case} {n} atoms mode {mode} {path}: |dE|/N {de:.3g}, max|dF| {df:.3g}")
    assert de <= TOL["e"], de
    assert df <= TOL["f"], df
    assert np.abs(g["charges"] - ref["charges"]).max() <= TOL["q"]
    assert np.abs(g["sc"]["virial"] - ref["virial"]).max() / n <= TOL["w"]
    assert np.abs(g["bec"] - ref["bec"]).max() <= TOL["z"]
    assert np.abs(g["sc"]["polarization"] - ref["polarization"]).max() / n <= TOL["p"]
    phi_scale = max(1.0, float(np.abs(ref["phi"]).max()))
    assert np.abs(g["potential"] - ref["phi"]).max() <= 1e-5 * phi_scale


def test_pppm_in_a_general_cell_per_atom_virial(dev):
    """The per-atom virial with the mesh term of the six extra inverse FFTs in a sheared cell."""
    sysm = _sheared_batio3(seed=74)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(75))[0]
    elec = wl.Elec(mode=1, kind="pppm", mesh=(16, 16, 16), order=5)
    g = _compute(dev, sysm, hp, params, elec, atom_virial=True)
    ref, _ = virial.per_atom_virial(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    assert np.abs(g["atom_virial"] - ref).max() <= 1e-4
