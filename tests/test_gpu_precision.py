"""Precision form: the network on the tensor cores (BF16 or TF32 operands, FP32 accumulation).

Everything else stays on the FP32 path (descriptor, Ewald / PPPM, backward) with FP64
reductions.  Bounds against the FP64 oracle (force RMSE <= 5e-3 eV/A for the mixed path
is the stated target; the other bounds follow from the operand rounding, 2^-9 relative
for BF16 and 2^-12 for TF32, propagated through the 30-wide network):
  BF16  force RMSE <= 5e-3 eV/A, max <= 3e-2; |dE|/N <= 2e-3 eV/atom; max |dq| <= 5e-3 e
  TF32  force RMSE <= 5e-4 eV/A, max <= 4e-3; |dE|/N <= 3e-4 eV/atom; max |dq| <= 6e-4 e
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu

BOUNDS = {
    "bf16": dict(f_rmse=5e-3, f_max=3e-2, e=2e-3, q=5e-3),
    "tf32": dict(f_rmse=5e-4, f_max=4e-3, e=3e-4, q=6e-4),
}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _errors(sysm, hp, params, elec, dev, precision, path="auto"):
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    model = QNEP(hp, params, elec, precision=precision)
    model.set_path(path)
    out = model.compute(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev), sysm.box)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}
    g.update(parse_scalars(out["scalars"]))
    model.close()
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    n = sysm.n_atoms
    df = g["forces"] - ref["forces"]
    return {
        "energy_per_atom": abs(g["energy"] - ref["energy"]) / n,
        "force_rmse": float(np.sqrt((df ** 2).mean())),
        "force_max": float(np.abs(df).max()),
        "charge_max": float(np.abs(g["charges"] - ref["charges"]).max()),
        "virial_per_atom": float(np.abs(g["virial"] - ref["virial"]).max() / n),
        "bec_max": float(np.abs(g["bec"] - ref["bec"]).max()),
        "polarization_per_atom": float(np.abs(g["polarization"] - ref["polarization"]).max() / n),
    }


def _one_species_water():
    """The 64-water box with every atom of one species (a single network; the tensor-core
    kernel then writes dU/dD and dq/dD row by row instead of through shared memory)."""
    sysm, _, _, elec = wl.config_water_small()
    sysm = wl.System(positions=sysm.positions, types=np.zeros_like(sysm.types), box=sysm.box, species=("O",))
    hp = wl.HParams(n_species=1)
    return sysm, hp, wl.random_params(hp, np.random.default_rng(43))[0], elec


CASES = {
    "water64": lambda: wl.config_water_small(),
    "water64_one_species": _one_species_water,
    "llzo192": lambda: (wl.llzo_base_cell(), wl.HParams(n_species=4),
                        wl.random_params(wl.HParams(n_species=4), np.random.default_rng(41))[0],
                        wl.Elec(mode=1, kind="ewald")),
    "batio3_40_pppm": lambda: (wl.batio3_supercell(2, seed=31), wl.HParams(n_species=3),
                               wl.random_params(wl.HParams(n_species=3), np.random.default_rng(42))[0],
                               wl.Elec(mode=1, kind="pppm", mesh=(16, 16, 16), order=5)),
}


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("path", ["warp", "thread"])
def test_mixed_precision_errors_within_bounds(dev, precision, case, path):
    sysm, hp, params, elec = CASES[case]()
    err = _errors(sysm, hp, params, elec, dev, precision, path)
    print(f"\n{case} {precision} {path}: " + ", ".join(f"{k}={v:.3g}" for k, v in err.items()))
    b = BOUNDS[precision]
    assert err["force_rmse"] <= b["f_rmse"], err
    assert err["force_max"] <= b["f_max"], err
    assert err["energy_per_atom"] <= b["e"], err
    assert err["charge_max"] <= b["q"], err


def test_mixed_path_is_closer_to_fp32_than_operand_rounding(dev):
    """TF32 and FP32 paths on the same input differ by about the TF32 rounding, not more."""
    from paper_2601_19034_gb300.qnep import QNEP
    sysm, hp, params, elec = wl.config_water_small()
    pos, typ = torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev)
    res = {}
    for prec in ("fp32", "tf32", "bf16"):
        m = QNEP(hp, params, elec, precision=prec)
        o = m.compute(pos, typ, sysm.box)
        res[prec] = o["forces"].cpu().numpy()
        m.close()
    d_tf = np.sqrt(((res["tf32"] - res["fp32"]) ** 2).mean())
    d_bf = np.sqrt(((res["bf16"] - res["fp32"]) ** 2).mean())
    scale = np.sqrt((res["fp32"] ** 2).mean())
    assert d_tf < d_bf, (d_tf, d_bf)
    assert d_tf / scale < 2e-3 and d_bf / scale < 2e-2, (d_tf / scale, d_bf / scale)


def test_vjp_rejected_on_mixed_path(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEP
    sysm, hp, params, elec = wl.config_water_small()
    m = QNEP(hp, params, elec, precision="bf16")
    with pytest.raises(_lib.QnepError) as e:
        m.vjp(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev), sysm.box, 1.0)
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    m.close()
