"""Large-scale form: velocity-Verlet NVE around the force call, Mg-water interface with PPPM.

* a 3297-atom Mg-water slab (same construction as the 1 M-atom system) against the FP64
  oracle, FP32 and BF16 network;
* one velocity-Verlet step against the oracle's update (oracle/md.py) with the GPU's forces;
* energy conservation of a short NVE run;
* the full ~1.0 M-atom system (PPPM 256 x 256 x 384): BF16 against the FP32 path
  (force RMSE <= 5e-3 eV/A), the charge constraint, and an NVE segment.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall, md  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _small():
    """3297-atom slab of the large system's construction and parameter recipe (PPPM h ~ 1 A)."""
    sysm = wl.mg_water_interface(6, 4, seed=77)
    _, hp, params, _ = wl.config_mg_water(nx=6, ny=4)
    elec = wl.Elec(mode=1, kind="pppm", mesh=(20, 24, 100), order=5)
    return sysm, hp, params, elec


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_small_mg_water_against_oracle(dev, precision):
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    sysm, hp, params, elec = _small()
    model = QNEP(hp, params, elec, precision=precision)
    out = model.compute(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev), sysm.box,
                        bec=False)
    torch.cuda.synchronize()
    sc = parse_scalars(out["scalars"])
    f = out["forces"].cpu().numpy()
    q = out["charges"].cpu().numpy()
    model.close()
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec,
                               want_bec=False)
    n = sysm.n_atoms
    de = abs(sc["energy"] - ref["energy"]) / n
    rmse = np.sqrt(((f - ref["forces"]) ** 2).mean())
    dfmax = np.abs(f - ref["forces"]).max()
    fmax = np.abs(ref["forces"]).max()
    print(f"\n{precision}: dE/N {de:.3g}, U^k/N {ref['e_kspace'] / n:.3g} eV, F max diff {dfmax:.3g}, "
          f"max|F| {fmax:.3g}, F RMSE {rmse:.3g}")
    if precision == "fp32":
        assert de <= 1e-6 and dfmax <= 1e-4 and np.abs(q - ref["charges"]).max() <= 2e-6, (de, dfmax)
    else:
        assert rmse <= 5e-3 and de <= 2e-3, (rmse, de)


def test_velocity_verlet_step_is_the_textbook_update(dev):
    from paper_2601_19034_gb300.qnep import QNEP, nve
    sysm, hp, params, elec = _small()
    masses = wl.species_masses(wl.MGWATER_SPECIES)
    m_atom = masses[sysm.types]
    v0 = wl.maxwell_boltzmann(m_atom, 300.0, seed=5).astype(np.float32)
    model = QNEP(hp, params, elec)
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    f0 = model.compute(pos, typ, sysm.box, bec=False)["forces"].cpu().numpy().astype(np.float64)
    vel = torch.tensor(v0, device=dev)
    dt = 0.5
    f1, en = nve(model, pos, vel, typ, masses, sysm.box, dt, 1)
    torch.cuda.synchronize()
    # the oracle's velocity-Verlet update, with the GPU's forces at both ends of the step
    x1 = md.positions_after_step(sysm.positions, v0, f0, m_atom, dt)
    np.testing.assert_allclose(pos.cpu().numpy(), x1, atol=2e-5)
    v1 = md.velocities_after_step(v0, f0, f1.cpu().numpy(), m_atom, dt)
    np.testing.assert_allclose(vel.cpu().numpy(), v1, atol=1e-6)
    e = en.cpu().numpy()
    k0, k1 = md.kinetic_energy(v0, m_atom), md.kinetic_energy(v1, m_atom)
    assert abs(e[0, 1] - k0) <= 1e-5 * k0 and abs(e[1, 1] - k1) <= 1e-5 * k1
    model.close()


def test_nve_energy_conservation_small(dev):
    from paper_2601_19034_gb300.qnep import QNEP, nve
    sysm, hp, params, elec = _small()
    masses = wl.species_masses(wl.MGWATER_SPECIES)
    v0 = wl.maxwell_boltzmann(masses[sysm.types], 300.0, seed=6).astype(np.float32)
    model = QNEP(hp, params, elec, precision="bf16")
    pos = torch.tensor(sysm.positions, device=dev)
    vel = torch.tensor(v0, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    _, en = nve(model, pos, vel, typ, masses, sysm.box, 0.5, 200)
    assert model.sync_status() == 0
    e = en.cpu().numpy()
    etot = e.sum(1)
    assert np.isfinite(etot).all()
    n = sysm.n_atoms
    t = np.arange(len(etot)) * 0.5e-3                       # ps
    slope = np.polyfit(t, (etot - etot[0]) / n, 1)[0] * 1e3  # meV/atom/ps
    print(f"\nNVE 3297 atoms, 200 x 0.5 fs: drift {slope:.3g} meV/atom/ps, "
          f"max |dE|/N {np.abs(etot - etot[0]).max() / n:.3g} eV, K0/N {e[0, 1] / n:.4f} eV")
    assert np.abs(etot - etot[0]).max() / n <= 2e-3
    model.close()


def test_full_size_mg_water(dev):
    """~1.0 M atoms, PPPM 256 x 256 x 384: mixed vs FP32 forces, charge constraint, NVE segment."""
    from paper_2601_19034_gb300.qnep import QNEP, nve, parse_scalars
    sysm, hp, params, elec = wl.config_mg_water()
    assert 0.98e6 <= sysm.n_atoms <= 1.02e6
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    res = {}
    for prec in ("fp32", "bf16"):
        model = QNEP(hp, params, elec, precision=prec)
        out = model.compute(pos, typ, sysm.box, bec=False)
        torch.cuda.synchronize()
        res[prec] = (out["forces"].clone(), parse_scalars(out["scalars"]), out["charges"].clone())
        model.close()
    f32, s32, q32 = res["fp32"]
    fbf, sbf, _ = res["bf16"]
    rmse = torch.sqrt(((fbf - f32) ** 2).mean()).item()
    assert rmse <= 5e-3, rmse
    assert abs(sbf["energy"] - s32["energy"]) / sysm.n_atoms <= 2e-3
    assert abs(q32.double().sum().item() - 0.0) <= 1e-3                # Q = 0
    assert torch.isfinite(f32).all()
    masses = wl.species_masses(wl.MGWATER_SPECIES)
    vel = torch.tensor(wl.maxwell_boltzmann(masses[sysm.types], 300.0).astype(np.float32), device=dev)
    model = QNEP(hp, params, elec, precision="bf16")
    _, en = nve(model, pos, vel, typ, masses, sysm.box, 0.5, 10)
    assert model.sync_status() == 0
    e = en.cpu().numpy()
    assert np.isfinite(e).all()
    assert np.abs(e.sum(1) - e[0].sum()).max() / sysm.n_atoms <= 1e-3
    model.close()


def _skin_pair(dev, sysm, hp, params, elec, skin=1.0):
    from paper_2601_19034_gb300.qnep import QNEP
    a = QNEP(hp, params, elec)
    a.set_skin(skin)
    b = QNEP(hp, params, elec)
    return a, b


def _compare_calls(dev, a, b, pos, typ, box, n):
    from paper_2601_19034_gb300.qnep import parse_scalars
    pa = torch.tensor(pos, device=dev)
    ta = torch.tensor(typ, device=dev)
    oa = a.compute(pa, ta, box, bec=False)
    ob = b.compute(pa, ta, box, bec=False)
    torch.cuda.synchronize()
    sa, sb = parse_scalars(oa["scalars"]), parse_scalars(ob["scalars"])
    assert abs(sa["energy"] - sb["energy"]) / n <= 1e-6
    assert (oa["forces"] - ob["forces"]).abs().max().item() <= 1e-4
    assert (oa["charges"] - ob["charges"]).abs().max().item() <= 2e-6
    assert np.abs(sa["virial"] - sb["virial"]).max() / n <= 1e-5


@pytest.mark.parametrize("case", ["mg_water_pppm", "water_ewald"])
def test_skin_lists_give_the_fresh_search_result(dev, case):
    """A kept candidate list (skin 1 A) gives the force call of a fresh cell search: at the build,
    after moves below skin / 2 (no rebuild) and after one atom moved beyond it (a rebuild)."""
    if case == "mg_water_pppm":
        sysm, hp, params, elec = _small()
    else:
        sysm, hp, params, elec = wl.config_water_small()
    a, b = _skin_pair(dev, sysm, hp, params, elec)
    rng = np.random.default_rng(3)
    x0 = sysm.positions.astype(np.float32)
    n = sysm.n_atoms
    _compare_calls(dev, a, b, x0, sysm.types, sysm.box, n)
    assert a.skin_rebuilds() == 1
    for _ in range(3):   # moves of at most 0.4 A (below skin / 2): the list is kept
        d = rng.normal(size=x0.shape)
        d *= 0.4 * rng.uniform(size=(n, 1)) / np.linalg.norm(d, axis=1, keepdims=True)
        _compare_calls(dev, a, b, (x0 + d).astype(np.float32), sysm.types, sysm.box, n)
    assert a.skin_rebuilds() == 1
    x1 = x0.copy()
    x1[7] += np.array([0.6, 0.0, 0.0], np.float32)   # one atom beyond skin / 2: rebuilt
    _compare_calls(dev, a, b, x1, sysm.types, sysm.box, n)
    assert a.skin_rebuilds() == 2
    # an atom that crosses the box face between rebuilds keeps its image shifts
    x2 = x1.copy()
    x2[11] = np.float32(sysm.box[0, 0] - 0.05) if x2[11, 0] > sysm.box[0, 0] / 2 else x2[11]
    x3 = x2.copy()
    x3[11, 0] += 0.2
    _compare_calls(dev, a, b, x2, sysm.types, sysm.box, n)
    _compare_calls(dev, a, b, x3, sysm.types, sysm.box, n)
    a.close()
    b.close()


def test_nve_with_skin_equals_rebuild_every_step(dev):
    """50 velocity-Verlet steps of 0.5 fs on the Mg-water slab with a 1 A skin and with lists rebuilt
    at every step: the same trajectory to FP32 rounding (the sums run in another order), and
    fewer rebuilds than steps."""
    from paper_2601_19034_gb300.qnep import QNEP, nve
    sysm, hp, params, elec = _small()
    masses = wl.species_masses(wl.MGWATER_SPECIES)
    v0 = wl.maxwell_boltzmann(masses[sysm.types], 300.0, seed=9).astype(np.float32)
    res = []
    for skin in (1.0, 0.0):
        model = QNEP(hp, params, elec)
        model.set_skin(skin)
        pos = torch.tensor(sysm.positions, device=dev)
        vel = torch.tensor(v0, device=dev)
        f, en = nve(model, pos, vel, torch.tensor(sysm.types, device=dev), masses, sysm.box, 0.5, 50)
        torch.cuda.synchronize()
        res.append((pos.cpu().numpy(), vel.cpu().numpy(), en.cpu().numpy(), model.skin_rebuilds() if skin else None))
        model.close()
    (p1, v1, e1, nreb), (p0, v0_, e0, _) = res
    n = sysm.n_atoms
    print(f"\nskin 1 A: {nreb} rebuilds in 51 force calls; max |dx| {np.abs(p1 - p0).max():.3g} A, "
          f"max |dE|/N {np.abs(e1 - e0).max() / n:.3g} eV")
    assert 1 <= nreb < 51
    assert np.abs(p1 - p0).max() <= 1e-3
    assert np.abs(v1 - v0_).max() <= 1e-3
    assert np.abs(e1 - e0).max() / n <= 1e-5


def test_skin_in_a_general_cell_and_with_the_per_atom_virial(dev):
    """The Verlet skin in a sheared cell (fractional cell grid, images t H) and with the per-atom
    virial requested: kept lists give the fresh search's force call after moves below skin / 2."""
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars
    sysm0 = wl.batio3_supercell(4, seed=81)
    box = sysm0.box.copy()
    box[1] = box[1] + 0.25 * box[0]
    box[2] = box[2] - 0.2 * box[1]
    frac = sysm0.positions.astype(np.float64) @ np.linalg.inv(sysm0.box)
    x0 = (frac @ box).astype(np.float32)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(82))[0]
    elec = wl.Elec(mode=1, kind="ewald")
    a = QNEP(hp, params, elec)
    a.set_skin(1.0)
    b = QNEP(hp, params, elec)
    rng = np.random.default_rng(83)
    typ = torch.tensor(sysm0.types, device=dev)
    n = len(x0)
    for step in range(3):
        d = rng.normal(size=x0.shape)
        d *= 0.3 * rng.uniform(size=(n, 1)) / np.linalg.norm(d, axis=1, keepdims=True)
        x = torch.tensor((x0 + (d if step else 0.0)).astype(np.float32), device=dev)
        oa = a.compute(x, typ, box, atom_virial=True)
        ob = b.compute(x, typ, box, atom_virial=True)
        torch.cuda.synchronize()
        sa, sb = parse_scalars(oa["scalars"]), parse_scalars(ob["scalars"])
        assert abs(sa["energy"] - sb["energy"]) / n <= 1e-6
        assert (oa["forces"] - ob["forces"]).abs().max().item() <= 1e-4
        assert (oa["bec"] - ob["bec"]).abs().max().item() <= 1e-4
        assert (oa["atom_virial"] - ob["atom_virial"]).abs().max().item() <= 1e-4
    assert a.skin_rebuilds() == 1
    a.close()
    b.close()


def test_nve_in_a_general_cell_with_pppm(dev):
    """NVE in a sheared water box (every off-diagonal element non-zero) with PPPM on the lattice-vector
    mesh and a 1 A skin: 10 steps of 0.5 fs equal the run that rebuilds its lists at every step to
    FP32 rounding, and the total energy is conserved (the FP64 oracle's velocity Verlet on this machine
    drifts by 8.4e-5 eV/atom over these steps; with random weights the box is not integrable much
    longer, as the potential has no short-range repulsion)."""
    from paper_2601_19034_gb300.qnep import QNEP, nve
    s0 = wl.water_box(5, seed=91)
    length = s0.box[0, 0]
    box = length * np.array([[1.0, 0.05, -0.04], [0.2, 1.0, 0.06], [-0.1, 0.15, 1.0]])
    pos0 = ((s0.positions.astype(np.float64) / length) @ box).astype(np.float32)
    hp = wl.HParams(n_species=2)
    params = wl.random_params(hp, np.random.default_rng(92))[0]
    elec = wl.Elec(mode=1, kind="pppm", mesh=(18, 18, 18), order=5)
    masses = wl.species_masses(s0.species)
    v0 = wl.maxwell_boltzmann(masses[s0.types], 300.0, seed=93).astype(np.float32)
    res = []
    for skin in (1.0, 0.0):
        model = QNEP(hp, params, elec)
        model.set_skin(skin)
        pos = torch.tensor(pos0, device=dev)
        vel = torch.tensor(v0, device=dev)
        _, en = nve(model, pos, vel, torch.tensor(s0.types, device=dev), masses, box, 0.5, 10)
        torch.cuda.synchronize()
        assert model.sync_status() == 0
        res.append((pos.cpu().numpy(), en.cpu().numpy()))
        model.close()
    (p1, e1), (p0, e0) = res
    n = len(pos0)
    etot = e0.sum(1)
    print(f"\nsheared water {n} atoms, PPPM, 10 x 0.5 fs: max |dx| skin vs rebuild {np.abs(p1 - p0).max():.3g} A, "
          f"max |dE_tot|/N {np.abs(etot - etot[0]).max() / n:.3g} eV")
    assert np.isfinite(etot).all()
    assert np.abs(p1 - p0).max() <= 1e-4
    assert np.abs(e1 - e0).max() / n <= 1e-5
    assert np.abs(etot - etot[0]).max() / n <= 1e-3
