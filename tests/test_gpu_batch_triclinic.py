"""The batched force call in general cells (Sec. II.B with k = 2 pi H^-1 n).  The kernels run the
restricted form a = (a_x, 0, 0), b = (b_x, b_y, 0), c = (c_x, c_y, c_z); other cells are rotated into
it inside the call and their outputs rotated back.

* Sheared LLZO cells of three sizes and sheared BaTiO3 cells (mode 2, Q != 0) against the FP64
  oracle (which handles general cells; tests/test_oracle_triclinic.py pins it), pair by pair:
  energy, forces, charges, the virial, BEC and the uncorrected total charge at the FP32-path
  tolerances, both descriptor contractions, orthorhombic cells in the same batch.
* The same crystal in a general cell and in the orthorhombic cell it is a unimodular transform
  of (rows a1, a2 + a1, a3 + a2 of an orthorhombic box, with its x and y shears kept in the
  restricted form): the same energies, and the forces and charges per atom, to FP32 rounding.
* Fully general cells (every off-diagonal element non-zero) against the oracle pair by pair, and a
  structure turned by a random rotation: energies and charges unchanged, forces, virial and BEC
  turned with it.
* Cells the batched call does not take are refused before any GPU work: a left-handed cell, one
  narrower than the cutoff.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_19034_gb300 import workloads as wl  # noqa: E402
from tests.test_gpu_batch import _check_pair, _check_virial, _llzo  # noqa: E402
from tests.test_gpu_batch_bec import _check_bec, _run, _sum_rule  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _sheared(system, shear, seed):
    """The cell's atoms at the same fractional coordinates in the lower-triangular cell
    diag(L) + shear (shear: b_x, c_x, c_y as fractions of the edges), plus N(0, 0.05 A) moves."""
    rng = np.random.default_rng(seed)
    lengths = np.diag(system.box).astype(np.float64)
    box = np.diag(lengths)
    box[1, 0] = shear[0] * lengths[1]
    box[2, 0] = shear[1] * lengths[2]
    box[2, 1] = shear[2] * lengths[2]
    frac = system.positions.astype(np.float64) / lengths[None]
    pos = frac @ box + rng.normal(0.0, 0.05, size=frac.shape)
    return wl.System(pos.astype(np.float32), system.types, box, system.species)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_sheared_llzo_and_orthorhombic_cells_against_oracle(dev, contract):
    systems = [_sheared(_llzo((1, 1, 1), 101), (0.12, -0.08, 0.1), 102), _llzo((1, 1, 1), 103),
               _sheared(_llzo((2, 1, 1), 104), (-0.05, 0.15, -0.11), 105),
               _sheared(_llzo((1, 2, 2), 106), (0.2, 0.0, 0.07), 107)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(108), n_candidates=33)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.2)
    res, off = _run(systems, hp, params, elec, dev, contract, virial=True, bec=True, total_charge=True,
                    polarization=True)
    for s, c in ((0, 0), (1, 3), (2, 32), (3, 17), (0, 31)):
        _check_pair(res, off, systems, s, c, hp, params, elec)
        _check_virial(res, off, systems, s, c, hp, params, elec)
        _check_bec(res, off, systems, s, c, hp, params, elec)
    _sum_rule(res, off, 0.2)


def test_sheared_perovskite_mode2(dev):
    systems = [_sheared(wl.batio3_supercell(2, seed=111), (0.1, 0.1, -0.1), 112),
               _sheared(wl.batio3_supercell(3, seed=113), (-0.15, 0.05, 0.12), 114)]
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(115), n_candidates=3)
    elec = wl.Elec(mode=2, kind="ewald", q_total=-0.3)
    res, off = _run(systems, hp, params, elec, dev, "bf16x3", virial=True, bec=True, total_charge=True,
                    polarization=True)
    for s in range(2):
        for c in range(3):
            _check_pair(res, off, systems, s, c, hp, params, elec)
            _check_virial(res, off, systems, s, c, hp, params, elec)
        _check_bec(res, off, systems, s, s, hp, params, elec)


def test_unimodular_cell_gives_the_orthorhombic_outputs(dev):
    """A 2 x 2 x 2 LLZO supercell (25.9 A cube) described by the cell with rows a1, a2 + a1, a3 + a2
    (lower triangular, its volume and lattice unchanged): every output per atom equals the
    orthorhombic call's to FP32 rounding, and the energy per atom to 1e-6 eV."""
    ortho = _llzo((2, 2, 2), 121)
    lat = np.diag(ortho.box).astype(np.float64)
    box = np.diag(lat)
    box[1, 0] = lat[0]   # a2 + a1
    box[2, 1] = lat[1]   # a3 + a2
    tri = wl.System(ortho.positions, ortho.types, box, ortho.species)
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(122), n_candidates=2)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.1)
    a, off = _run([ortho, tri], hp, params, elec, dev, "bf16x3", virial=True)
    n = int(off[1])
    assert np.abs(a["energy"][:, 0] - a["energy"][:, 1]).max() / n <= 1e-6
    assert np.abs(a["forces"][:, :n] - a["forces"][:, n:]).max() <= 1e-4
    assert np.abs(a["charges"][:, :n] - a["charges"][:, n:]).max() <= 2e-6
    assert np.abs(a["virial"][:, 0] - a["virial"][:, 1]).max() / n <= 1e-5


def test_cells_the_batched_call_refuses(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEPBatch
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(131), n_candidates=2)
    b = QNEPBatch(hp, params, wl.Elec(mode=1, kind="ewald"))
    pos = torch.rand(10, 3, device=dev) * 10.0
    typ = torch.zeros(10, dtype=torch.int32, device=dev)
    for box, status in ((np.array([[20.0, 0, 0], [1.0, 20.0, 0], [0, 2.0, -20.0]]), _lib.QNEP_ERR_ARG),
                        (np.array([[20.0, 0.3, 0.2], [1.0, 20.0, 0.5], [0.4, 2.0, -20.0]]), _lib.QNEP_ERR_ARG),
                        (np.array([[20.0, 0, 0], [19.0, 5.5, 0], [0, 0, 20.0]]), _lib.QNEP_ERR_UNSUPPORTED)):
        with pytest.raises(_lib.QnepError) as e:
            b.compute(pos, typ, [0, 10], box[None])
        assert e.value.status == status, box
    b.close()


def _general(system, shear, seed):
    """The cell's atoms at the same fractional coordinates in diag(L) + shear x L (every entry of
    the 3 x 3 shear non-zero off the diagonal), plus N(0, 0.05 A) moves."""
    rng = np.random.default_rng(seed)
    lengths = np.diag(system.box).astype(np.float64)
    box = np.diag(lengths) + np.asarray(shear) * lengths[:, None]
    frac = system.positions.astype(np.float64) / lengths[None]
    pos = frac @ box + rng.normal(0.0, 0.05, size=frac.shape)
    return wl.System(pos.astype(np.float32), system.types, box, system.species)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_fully_general_cells_against_oracle(dev, contract):
    shear1 = [[0.0, 0.06, -0.05], [0.12, 0.0, 0.08], [-0.1, 0.09, 0.0]]
    shear2 = [[0.0, -0.04, 0.07], [0.05, 0.0, -0.06], [0.11, -0.08, 0.0]]
    systems = [_general(_llzo((1, 1, 1), 151), shear1, 152), _llzo((1, 1, 1), 153),
               _general(_llzo((2, 1, 1), 154), shear2, 155)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(156), n_candidates=33)
    elec = wl.Elec(mode=1, kind="ewald", q_total=-0.2)
    res, off = _run(systems, hp, params, elec, dev, contract, virial=True, bec=True, total_charge=True,
                    polarization=True)
    for s, c in ((0, 0), (0, 32), (1, 5), (2, 17)):
        _check_pair(res, off, systems, s, c, hp, params, elec)
        _check_virial(res, off, systems, s, c, hp, params, elec)
        _check_bec(res, off, systems, s, c, hp, params, elec)
    _sum_rule(res, off, -0.2)


def test_a_rotated_structure_turns_its_outputs(dev):
    """A sheared BaTiO3 cell and the same crystal turned by a random rotation Q (cell rows and
    positions r -> Q r): energies and charges equal, forces Q F, virial and BEC Q X Q^T."""
    base = _sheared(wl.batio3_supercell(3, seed=161), (0.1, -0.08, 0.12), 162)
    q_, _ = np.linalg.qr(np.random.default_rng(163).normal(size=(3, 3)))
    if np.linalg.det(q_) < 0:
        q_[:, 0] = -q_[:, 0]
    turned = wl.System((base.positions.astype(np.float64) @ q_.T).astype(np.float32), base.types,
                       base.box @ q_.T, base.species)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(164), n_candidates=2)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.3)
    a, off = _run([base, turned], hp, params, elec, dev, "bf16x3", virial=True, bec=True, polarization=True)
    n = int(off[1])
    assert np.abs(a["energy"][:, 0] - a["energy"][:, 1]).max() / n <= 1e-6
    assert np.abs(a["charges"][:, :n] - a["charges"][:, n:]).max() <= 2e-6
    assert np.abs(a["forces"][:, :n] @ q_.T - a["forces"][:, n:]).max() <= 1e-4
    w0 = np.einsum("ab,cbd,ed->cae", q_, a["virial"][:, 0], q_)
    assert np.abs(w0 - a["virial"][:, 1]).max() / n <= 1e-5
    z0 = np.einsum("ab,cibd,ed->ciae", q_, a["bec"][:, :n], q_)
    assert np.abs(z0 - a["bec"][:, n:]).max() <= 1e-4
    assert np.abs(a["polarization"][:, 0] @ q_.T - a["polarization"][:, 1]).max() / n <= 1e-5
