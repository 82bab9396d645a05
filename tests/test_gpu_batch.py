"""GPU parity of the batched force call (many structures x many candidate parameter vectors).

Every (candidate, structure) pair of a small batch is compared with the FP64 oracle
(energy |dE|/N <= 1e-6 eV/atom, forces <= 1e-4 eV/A, charges <= 2e-6 e, the
tolerances of the single-structure path), and with the single-structure CUDA path.
The full 512 x 64 LLZO batch is checked on sampled (candidate, structure) pairs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = dict(e=1e-6, f=1e-4, q=2e-6)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _llzo(reps, seed, sigma=0.1):
    """Supercell reps of the random 192-atom LLZO cell with N(0, sigma) moves."""
    base = wl.llzo_base_cell()
    a = base.box[0, 0]
    rng = np.random.default_rng(seed)
    shifts = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    pos = (base.positions[None].astype(np.float64) + shifts[:, None, :] * a).reshape(-1, 3)
    pos += rng.normal(0.0, sigma, size=pos.shape)
    lengths = np.asarray(reps) * a
    pos %= lengths
    return wl.System(pos.astype(np.float32), np.tile(base.types, len(shifts)), np.diag(lengths.astype(np.float64)),
                     wl.LLZO_SPECIES)


def _run_batch(systems, hp, params, elec, dev, warps=8, order="largest_first", contract="fp32", virial=False):
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_config(warps, order)
    b.set_contraction(contract)
    out = b.compute(torch.tensor(pos, device=dev), torch.tensor(typ, device=dev), off, boxes, virial=virial)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    b.close()
    return res, off


def _check_pair(res, off, systems, s, c, hp, params, elec):
    sysm = systems[s]
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params[c], elec,
                               want_bec=False)
    n = sysm.n_atoms
    sl = slice(off[s], off[s + 1])
    assert abs(res["energy"][c, s] - ref["energy"]) / n <= TOL["e"], (s, c, res["energy"][c, s], ref["energy"])
    df = np.abs(res["forces"][c, sl] - ref["forces"]).max()
    assert df <= TOL["f"], (s, c, df)
    dq = np.abs(res["charges"][c, sl] - ref["charges"]).max()
    assert dq <= TOL["q"], (s, c, dq)


@pytest.mark.parametrize("warps,contract", [(8, "fp32"), (4, "fp32"), (8, "bf16x3")])
def test_small_batch_every_pair_against_oracle(dev, warps, contract):
    systems = [_llzo((1, 1, 1), 1), _llzo((2, 1, 1), 2), _llzo((1, 1, 2), 3)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(11), n_candidates=3)
    elec = wl.Elec(mode=1, kind="ewald")
    res, off = _run_batch(systems, hp, params, elec, dev, warps=warps, contract=contract)
    for s in range(len(systems)):
        for c in range(3):
            _check_pair(res, off, systems, s, c, hp, params, elec)


def test_two_groups_against_single_structure_path(dev):
    """40 candidates (a full and a partial lane group) x 4 structures vs qnep_compute per pair."""
    from paper_2601_19034_gb300.qnep import QNEP
    systems = [_llzo((1, 1, 1), 4), _llzo((1, 2, 1), 5), _llzo((2, 2, 1), 6), _llzo((1, 1, 1), 7)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(12), n_candidates=40)
    elec = wl.Elec(mode=1, kind="ewald")
    res, off = _run_batch(systems, hp, params, elec, dev)
    for c in range(40):
        model = QNEP(hp, params[c], elec)
        for s, sysm in enumerate(systems):
            out = model.compute(torch.tensor(sysm.positions, device=dev), torch.tensor(sysm.types, device=dev),
                                sysm.box, bec=False, virial=False)
            sl = slice(off[s], off[s + 1])
            e1 = out["scalars"][0].item()
            assert abs(res["energy"][c, s] - e1) / sysm.n_atoms <= 2 * TOL["e"], (s, c)
            assert np.abs(res["forces"][c, sl] - out["forces"].cpu().numpy()).max() <= 2 * TOL["f"], (s, c)
            assert np.abs(res["charges"][c, sl] - out["charges"].cpu().numpy()).max() <= 2 * TOL["q"], (s, c)
        model.close()
    # one pair of each group against the oracle as well
    for s, c in ((2, 5), (1, 37)):
        _check_pair(res, off, systems, s, c, hp, params, elec)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_mode2_total_charge_and_one_species_water(dev, contract):
    """k-space-only electrostatics, a charged target and 2-species water boxes of uneven size."""
    systems = [wl.water_box(4, seed=21), wl.water_box(5, seed=22)]
    hp = wl.HParams(n_species=2)
    params = wl.random_params(hp, np.random.default_rng(13), n_candidates=33)
    elec = wl.Elec(mode=2, kind="ewald", q_total=0.5)
    res, off = _run_batch(systems, hp, params, elec, dev, contract=contract)
    for s, c in ((0, 0), (1, 32), (1, 7)):
        _check_pair(res, off, systems, s, c, hp, params, elec)
    # total corrected charge is Q / sqrt(eps_inf) per pair
    for s in range(2):
        tot = res["charges"][:, off[s]:off[s + 1]].astype(np.float64).sum(1)
        np.testing.assert_allclose(tot, 0.5 / params[:, -1].astype(np.float64), atol=2e-4)


def test_graph_replay_and_autotuner_agree(dev):
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    systems = [_llzo((1, 1, 1), 8), _llzo((2, 1, 1), 9), _llzo((1, 2, 2), 10)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(14), n_candidates=64)
    elec = wl.Elec(mode=1, kind="ewald")
    pos, typ, off, boxes = stack_structures(systems)
    pos_d, typ_d = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
    b = QNEPBatch(hp, params, elec)
    ref = {k: v.clone() for k, v in b.compute(pos_d, typ_d, off, boxes).items()}
    ms = b.autotune(pos_d, typ_d, off, boxes, reps=2)
    assert ms > 0
    out = b.outputs(len(systems), pos.shape[0], dev)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        b.compute_into(pos_d, typ_d, off, boxes, out)   # description cached: launch only
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.compute_into(pos_d, typ_d, off, boxes, out)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    n = np.diff(off)
    de = (out["energy"] - ref["energy"]).abs().cpu().numpy() / n[None, :]
    assert de.max() <= 1e-6
    assert (out["forces"] - ref["forces"]).abs().max().item() <= 1e-4
    assert (out["charges"] - ref["charges"]).abs().max().item() <= 1e-6
    b.close()


def test_argument_errors_before_gpu_work(dev):
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEPBatch
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(15), n_candidates=2)
    b = QNEPBatch(hp, params, wl.Elec(mode=1, kind="ewald"))
    pos = torch.zeros(10, 3, device=dev)
    typ = torch.zeros(10, dtype=torch.int32, device=dev)
    with pytest.raises(_lib.QnepError) as e:   # box edge below the 6 A list cutoff
        b.compute(pos, typ, [0, 10], np.diag([5.0, 20.0, 20.0])[None])
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    with pytest.raises(_lib.QnepError) as e:   # box edge above the k-space tables' limit (~45 A)
        b.compute(pos, typ, [0, 10], np.diag([50.0, 50.0, 50.0])[None])
    assert e.value.status == _lib.QNEP_ERR_UNSUPPORTED
    with pytest.raises(_lib.QnepError) as e:   # offsets must not decrease
        b.compute(pos, typ, [0, 10, 5], np.stack([np.eye(3) * 20.0] * 2))
    assert e.value.status == _lib.QNEP_ERR_ARG
    # a species index outside [0, n_species) is reported by the status check (no out-of-range access)
    typ_bad = torch.tensor([0, 1, 2, 3, 7, 0, 1, 2, 3, 0], dtype=torch.int32, device=dev)
    pos_ok = torch.rand(10, 3, device=dev) * 20.0
    with pytest.raises(_lib.QnepError) as e:
        b.compute(pos_ok, typ_bad, [0, 10], (np.eye(3) * 20.0)[None])
    assert e.value.status == _lib.QNEP_ERR_ARG
    b.close()


def test_full_llzo_batch_sampled_pairs(dev):
    """512 LLZO cells (192-1536 atoms) x 64 candidates in one call; sampled pairs vs the oracle."""
    systems, hp, params, elec = wl.config_llzo_batch()
    res, off = _run_batch(systems, hp, params, elec, dev)
    assert np.isfinite(res["energy"]).all() and np.isfinite(res["forces"]).all()
    sizes = np.diff(off)
    big = int(np.argmax(sizes))
    small = int(np.argmin(sizes))
    for s, c in ((big, 63), (small, 0), (int(np.argsort(sizes)[len(sizes) // 2]), 33)):
        _check_pair(res, off, systems, s, c, hp, params, elec)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_edge_cases_empty_single_atom_and_one_candidate(dev, contract):
    """Empty and one-/two-atom structures next to a normal cell; one candidate (31 padded lanes)."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(16), n_candidates=1)
    elec = wl.Elec(mode=1, kind="ewald")
    one = wl.System(np.array([[1.0, 2.0, 3.0]], np.float32), np.array([2], np.int32), np.diag([9.0, 9.0, 9.0]),
                    wl.LLZO_SPECIES)
    two = wl.System(np.array([[1.0, 1.0, 1.0], [2.2, 1.1, 0.9]], np.float32), np.array([0, 3], np.int32),
                    np.diag([8.0, 10.0, 12.0]), wl.LLZO_SPECIES)
    empty = wl.System(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.diag([10.0, 10.0, 10.0]),
                      wl.LLZO_SPECIES)
    systems = [one, _llzo((1, 1, 1), 17), empty, two]
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction(contract)
    out = b.compute(torch.tensor(pos, device=dev), torch.tensor(typ, device=dev), off, boxes)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    b.close()
    for s in (0, 1, 3):
        _check_pair(res, off, systems, s, 0, hp, params, elec)
    assert res["energy"][0, 2] == 0.0     # an empty structure contributes nothing


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_batched_three_species_perovskite_mix(dev, contract):
    """BaTiO3 cells of several sizes (cubic 8 A to 12 A) in one batch, mode 1 with a charge target."""
    systems = [wl.batio3_supercell(2, seed=51), wl.batio3_supercell(3, seed=52), wl.batio3_supercell(2, seed=53)]
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(18), n_candidates=35)
    elec = wl.Elec(mode=1, kind="ewald", q_total=-0.4)
    res, off = _run_batch(systems, hp, params, elec, dev, contract=contract)
    for s, c in ((0, 0), (1, 34), (2, 17)):
        _check_pair(res, off, systems, s, c, hp, params, elec)


def test_full_llzo_batch_tensor_core_contraction(dev):
    """The full 512 x 64 batch with the BF16x3 tensor-core contraction: sampled pairs against the
    oracle at the FP32 tolerances, and every pair against the FP32 contraction (energy per atom
    1e-6 eV, forces 1e-4 eV/A, charges 2e-6 e)."""
    systems, hp, params, elec = wl.config_llzo_batch()
    res_tc, off = _run_batch(systems, hp, params, elec, dev, contract="bf16x3", virial=True)
    assert np.isfinite(res_tc["energy"]).all() and np.isfinite(res_tc["forces"]).all()
    assert np.isfinite(res_tc["virial"]).all()
    sizes = np.diff(off)
    big = int(np.argmax(sizes))
    small = int(np.argmin(sizes))
    for s, c in ((big, 62), (small, 1), (int(np.argsort(sizes)[len(sizes) // 2]), 31)):
        _check_pair(res_tc, off, systems, s, c, hp, params, elec)
        _check_virial(res_tc, off, systems, s, c, hp, params, elec)
    res_fp, _ = _run_batch(systems, hp, params, elec, dev, contract="fp32")
    de = np.abs(res_tc["energy"] - res_fp["energy"]) / sizes[None, :]
    assert de.max() <= TOL["e"], de.max()
    assert np.abs(res_tc["forces"] - res_fp["forces"]).max() <= TOL["f"]
    assert np.abs(res_tc["charges"] - res_fp["charges"]).max() <= TOL["q"]


def _check_virial(res, off, systems, s, c, hp, params, elec):
    sysm = systems[s]
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params[c], elec,
                               want_bec=False)
    dw = np.abs(res["virial"][c, s] - ref["virial"]).max() / sysm.n_atoms
    assert dw <= 1e-5, (s, c, dw)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_batched_virial_against_oracle(dev, contract):
    """The per-(candidate, structure) virial (entries, static real space, W^k) against the oracle's
    strain derivative, 1e-5 eV per atom; energies, forces and charges unchanged by asking for it."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    systems = [_llzo((1, 1, 1), 31), _llzo((2, 1, 1), 32), _llzo((1, 2, 2), 33)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(34), n_candidates=33)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.3)
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction(contract)
    pd, td = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
    out_v = b.compute(pd, td, off, boxes, virial=True)
    out = b.compute(pd, td, off, boxes)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out_v.items()}
    b.close()
    n = np.diff(off)
    assert np.abs(res["energy"] - out["energy"].cpu().numpy()).max() / n.min() <= 1e-9
    assert np.abs(res["forces"] - out["forces"].cpu().numpy()).max() <= 1e-5
    for s_, c in ((0, 0), (1, 32), (2, 7)):
        _check_virial(res, off, systems, s_, c, hp, params, elec)
        _check_pair(res, off, systems, s_, c, hp, params, elec)
    # the virial of every pair is symmetric to the FP32 rounding of its parts
    w = res["virial"]
    assert np.abs(w - np.swapaxes(w, 2, 3)).max() / n.min() <= 1e-5


def test_batched_virial_mode2_water_and_perovskite(dev):
    """k-space-only electrostatics (2-species water) and mode 1 on 3-species BaTiO3 cells."""
    for systems, hp, elec, seed in (
            ([wl.water_box(4, seed=41), wl.water_box(5, seed=42)], wl.HParams(n_species=2),
             wl.Elec(mode=2, kind="ewald", q_total=0.5), 43),
            ([wl.batio3_supercell(2, seed=44), wl.batio3_supercell(3, seed=45)], wl.HParams(n_species=3),
             wl.Elec(mode=1, kind="ewald", q_total=-0.4), 46)):
        params = wl.random_params(hp, np.random.default_rng(seed), n_candidates=3)
        from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
        pos, typ, off, boxes = stack_structures(systems)
        b = QNEPBatch(hp, params, elec)
        out = b.compute(torch.tensor(pos, device=dev), torch.tensor(typ, device=dev), off, boxes, virial=True)
        torch.cuda.synchronize()
        res = {k: v.cpu().numpy() for k, v in out.items()}
        b.close()
        for s_ in range(len(systems)):
            _check_virial(res, off, systems, s_, s_ % 3, hp, params, elec)


def test_host_buffer_call_equals_device_call(dev):
    """qnep_batch_compute_host: host inputs in, every output back (pinned and pageable host memory),
    equal to the device-buffer call of the same batch; then a new batch shape on the same object."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    systems = [_llzo((1, 1, 1), 51), _llzo((2, 1, 1), 52)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(53), n_candidates=5)
    elec = wl.Elec(mode=1, kind="ewald")
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction("bf16x3")
    ref = b.compute(torch.tensor(pos, device=dev), torch.tensor(typ, device=dev), off, boxes, virial=True)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    c, s_, n = 5, len(systems), int(off[-1])
    for pinned in (True, False):
        def h(shape, dtype):
            t = torch.full(shape, float("nan") if dtype.is_floating_point else 0, dtype=dtype)
            return t.pin_memory() if pinned else t.numpy()
        out = {"energy": h((c, s_), torch.float64), "forces": h((c, n, 3), torch.float32),
               "charges": h((c, n), torch.float32), "virial": h((c, s_, 3, 3), torch.float64)}
        ph = torch.tensor(pos).pin_memory() if pinned else np.ascontiguousarray(pos)
        th = torch.tensor(typ).pin_memory() if pinned else np.ascontiguousarray(typ)
        b.compute_host(ph, th, off, boxes, out)
        for k in out:
            got = out[k].numpy() if isinstance(out[k], torch.Tensor) else out[k]
            assert np.array_equal(got, ref[k]) or np.abs(got - ref[k]).max() <= (1e-9 if k == "energy" else 1e-5), k
    # a larger batch on the same object: the host-buffer workspaces grow
    systems2 = systems + [_llzo((1, 2, 2), 54)]
    pos2, typ2, off2, boxes2 = stack_structures(systems2)
    out2 = {"energy": np.zeros((c, 3)), "forces": np.zeros((c, int(off2[-1]), 3), np.float32)}
    b.compute_host(pos2, typ2, off2, boxes2, out2)
    _check_pair({"energy": out2["energy"], "forces": out2["forces"],
                 "charges": b.compute(torch.tensor(pos2, device=dev), torch.tensor(typ2, device=dev), off2,
                                      boxes2)["charges"].cpu().numpy()}, off2, systems2, 2, 4, hp, params, elec)
    b.close()


def test_reduced_precision_contraction_meets_the_mixed_bounds(dev):
    """The single-product BF16 contraction (the batched call's reduced-precision form) on small LLZO
    and perovskite batches: every pair against the FP64 oracle at the mixed-path bounds (force RMSE
    5e-3 eV/A, max 3e-2 eV/A, |dE|/N 2e-3 eV, charges 5e-3 e), and measurably different from the
    FP32 contraction (the products really are reduced)."""
    cases = [([_llzo((1, 1, 1), 71), _llzo((2, 1, 1), 72)], wl.HParams(n_species=4), wl.Elec(mode=1, kind="ewald")),
             ([wl.batio3_supercell(2, seed=73), wl.batio3_supercell(3, seed=74)], wl.HParams(n_species=3),
              wl.Elec(mode=2, kind="ewald", q_total=0.3))]
    worst = dict(rmse=0.0, fmax=0.0, de=0.0, dq=0.0)
    for k, (systems, hp, elec) in enumerate(cases):
        params = wl.random_params(hp, np.random.default_rng(75 + k), n_candidates=3)
        res, off = _run_batch(systems, hp, params, elec, dev, contract="bf16")
        res32, _ = _run_batch(systems, hp, params, elec, dev, contract="fp32")
        assert np.abs(res["forces"] - res32["forces"]).max() > 0.0
        for s in range(len(systems)):
            for c in range(3):
                sysm = systems[s]
                ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params[c],
                                           elec, want_bec=False)
                sl = slice(off[s], off[s + 1])
                df = res["forces"][c, sl] - ref["forces"]
                worst["rmse"] = max(worst["rmse"], float(np.sqrt((df ** 2).mean())))
                worst["fmax"] = max(worst["fmax"], float(np.abs(df).max()))
                worst["de"] = max(worst["de"], abs(res["energy"][c, s] - ref["energy"]) / sysm.n_atoms)
                worst["dq"] = max(worst["dq"], float(np.abs(res["charges"][c, sl] - ref["charges"]).max()))
    print(f"\nBF16 contraction against the oracle: {worst}")
    assert worst["rmse"] <= 5e-3 and worst["fmax"] <= 3e-2 and worst["de"] <= 2e-3 and worst["dq"] <= 5e-3, worst


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_few_or_no_wave_vectors(dev, contract):
    """k_max 0.3 1/A: the 12.97 A cells have no wave vector inside the sphere (U^k = 0, no k-space
    field), the 25.9 A cells a single partly filled chunk; every pair against the oracle, so the
    tensor-core passes' empty and ragged k-sets meet the FP32-path tolerances."""
    systems = [_llzo((1, 1, 1), 91), _llzo((2, 2, 1), 92), _llzo((2, 2, 2), 93)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(94), n_candidates=3)
    elec = wl.Elec(mode=1, kind="ewald", kmax=0.3, q_total=0.2)
    res, off = _run_batch(systems, hp, params, elec, dev, contract=contract)
    for s in range(len(systems)):
        for c in range(3):
            _check_pair(res, off, systems, s, c, hp, params, elec)
