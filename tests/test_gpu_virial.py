"""GPU parity of the per-atom virial W_i (Sec. II.C, Eq. per-atom_virial; the mesh form of Sec. II.F).

Element by element against the FP64 oracle (oracle/virial.py): the neighbour-entry
terms (descriptor and dynamic-charge partial forces, -r_ij (x) F_ij given to W_j), the
static real-space pair terms and the static reciprocal-space term (Heyes form for Ewald,
six more inverse FFTs for PPPM).  Bounds: max |dW_i| <= 1e-4 eV (per-atom terms of
~O(1-10) eV summed in FP32) and the sum over the atoms equal to the call's total
virial within the total-virial tolerance (1e-5 eV per atom).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import virial  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _run(dev, sysm, hp, params, elec, tol=1e-4):
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    model = QNEP(hp, params, elec)
    out = model.compute(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev), sysm.box,
                        bec=False, atom_virial=True)
    torch.cuda.synchronize()
    w = out["atom_virial"].double().cpu().numpy()
    tot = parse_scalars(out["scalars"])["virial"]
    model.close()
    ref, _ = virial.per_atom_virial(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    n = sysm.n_atoms
    dw = np.abs(w - ref).max()
    print(f"\n{n} atoms {elec.kind} mode {elec.mode}: max|dW_i| {dw:.3g} eV (max|W_i| {np.abs(ref).max():.3g}), "
          f"|sum W_i - W|/N {np.abs(w.sum(0) - tot).max() / n:.3g}")
    assert dw <= tol, dw
    assert np.abs(w.sum(0) - tot).max() / n <= 1e-5
    assert np.abs(w.sum(0) - ref.sum(0)).max() / n <= 1e-5


@pytest.mark.parametrize("elec", [wl.Elec(mode=1, kind="ewald"), wl.Elec(mode=2, kind="ewald", q_total=0.3),
                                  wl.Elec(mode=1, kind="pppm", mesh=(16, 16, 16), order=5)],
                         ids=["ewald-mode1", "ewald-mode2-charged", "pppm-16"])
def test_batio3_40_atoms(dev, elec):
    sysm = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(32))[0]
    _run(dev, sysm, hp, params, elec)


def test_water_192_ewald(dev):
    sysm, hp, params, elec = wl.config_water_small()
    _run(dev, sysm, hp, params, elec)


def test_mg_water_slab_pppm(dev):
    sysm = wl.mg_water_interface(6, 4, seed=77)
    _, hp, params, _ = wl.config_mg_water(nx=6, ny=4)
    elec = wl.Elec(mode=1, kind="pppm", mesh=(20, 24, 100), order=5)
    _run(dev, sysm, hp, params, elec)


def test_batio3_5000_atoms_ewald(dev):
    sysm, hp, params, elec = wl.config_batio3()
    _run(dev, sysm, hp, params, elec)


def test_per_atom_virial_leaves_the_other_outputs_unchanged(dev):
    from paper_2601_19034_gb300.qnep import QNEP
    sysm, hp, params, elec = wl.config_water_small()
    model = QNEP(hp, params, elec)
    pos, typ = torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev)
    a = model.compute(pos, typ, sysm.box, atom_virial=True)
    b = model.compute(pos, typ, sysm.box)
    torch.cuda.synchronize()
    for k in ("forces", "bec", "charges"):
        assert (a[k] - b[k]).abs().max().item() <= 1e-5, k
    # the scalars up to the order of the FP32 partial sums and FP64 atomics (the backward kernels
    # with and without the per-atom virial run at different occupancies): energies to FP64
    # rounding, the virial to FP32 rounding of its per-thread partial sums
    sa, sb = a["scalars"].cpu().numpy(), b["scalars"].cpu().numpy()
    assert np.all(np.abs(sa[:5] - sb[:5]) <= 1e-9 * np.maximum(1.0, np.abs(sb[:5])))
    assert np.abs(sa[5:14] - sb[5:14]).max() / sysm.n_atoms <= 1e-8
    model.set_path("thread")
    from paper_2601_19034_gb300 import _lib
    with pytest.raises(_lib.QnepError) as e:
        model.compute(pos, typ, sysm.box, atom_virial=True)
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    model.close()
