"""GPU parity of the batched call's Born effective charges and uncorrected total charges, and of
the full training loss of Sec. II.E built on them.

* BEC (Eq. bec_2, periodic form) of sampled (candidate, structure) pairs element by element
  against the FP64 oracle at the single-structure BEC tolerance (1e-4 e), for both descriptor
  contractions, Ewald modes 1 and 2 and charged targets; the acoustic sum rule
  sum_i Z_i = Q I (every entry term is added to one atom and subtracted from another) on every
  pair; energies, forces and charges of the call unchanged by asking for BEC.
* polarization P = sum q~^c_i r_i per pair against the oracle (1e-5 e A per atom).
* total charge before the correction (the D_Q input) against the oracle's sum of q~ per pair:
  FP32 network charges summed in FP64, within N x 2e-6 e x sqrt(eps_inf) (the per-atom charge
  tolerance summed over the structure's atoms).
* qnep_batch_loss_full on the outputs of a small batch against oracle.training.loss_terms_full
  (a structure mask that leaves one structure without reference BEC, an empty structure).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall  # noqa: E402
from oracle import training as tr  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402
from tests.test_gpu_batch import TOL, _check_pair, _llzo  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_Z = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _run(systems, hp, params, elec, dev, contract="fp32", **kw):
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction(contract)
    pd, td = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
    out = b.compute(pd, td, off, boxes, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    b.close()
    return res, off


def _check_bec(res, off, systems, s, c, hp, params, elec):
    sysm = systems[s]
    ref = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params[c], elec)
    sl = slice(off[s], off[s + 1])
    dz = np.abs(res["bec"][c, sl] - ref["bec"]).max()
    assert dz <= TOL_Z, (s, c, dz)
    seps = float(params[c, -1])
    dq = abs(res["total_charge"][c, s] - ref["total_charge_raw"])
    assert dq <= 2e-6 * sysm.n_atoms * seps, (s, c, dq, ref["total_charge_raw"])
    if "polarization" in res:   # P = sum q~^c r over the positions as given, 1e-5 e A per atom
        dp = np.abs(res["polarization"][c, s] - ref["polarization"]).max() / sysm.n_atoms
        assert dp <= 1e-5, (s, c, dp)
    return ref


def _sum_rule(res, off, q_total):
    """sum_i Z_i = Q I on every pair (FP32 terms: 1e-4 e per atom of the structure at most)."""
    for s in range(len(off) - 1):
        n = off[s + 1] - off[s]
        if n == 0:
            continue
        tot = res["bec"][:, off[s]:off[s + 1]].astype(np.float64).sum(1)   # [C, 3, 3]
        err = np.abs(tot - q_total * np.eye(3)[None]).max()
        assert err <= 1e-5 * n, (s, err)


@pytest.mark.parametrize("contract", ["fp32", "bf16x3"])
def test_batched_bec_and_total_charge_against_oracle(dev, contract):
    systems = [_llzo((1, 1, 1), 61), _llzo((2, 1, 1), 62), _llzo((1, 1, 1), 63)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(64), n_candidates=33)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.3)
    res, off = _run(systems, hp, params, elec, dev, contract, bec=True, total_charge=True, polarization=True)
    plain, _ = _run(systems, hp, params, elec, dev, contract)
    n = np.diff(off)
    assert np.abs(res["energy"] - plain["energy"]).max() / n.min() <= 1e-9
    assert np.abs(res["forces"] - plain["forces"]).max() <= 1e-5
    assert np.abs(res["charges"] - plain["charges"]).max() <= 1e-6
    for s, c in ((0, 0), (1, 32), (2, 17), (1, 5)):
        _check_bec(res, off, systems, s, c, hp, params, elec)
        _check_pair(res, off, systems, s, c, hp, params, elec)
    _sum_rule(res, off, 0.3)


def test_batched_bec_mode2_water_perovskite_and_edge_cases(dev):
    """k-space-only water (2 species), a 3-species perovskite with Q != 0, and a batch with an empty
    structure and a one-atom structure next to a cell (one candidate, 31 padded lanes)."""
    for systems, hp, elec, seed, c_n in (
            ([wl.water_box(4, seed=65), wl.water_box(5, seed=66)], wl.HParams(n_species=2),
             wl.Elec(mode=2, kind="ewald", q_total=0.5), 67, 3),
            ([wl.batio3_supercell(2, seed=68), wl.batio3_supercell(3, seed=69)], wl.HParams(n_species=3),
             wl.Elec(mode=1, kind="ewald", q_total=-0.4), 70, 2)):
        params = wl.random_params(hp, np.random.default_rng(seed), n_candidates=c_n)
        res, off = _run(systems, hp, params, elec, dev, "bf16x3", bec=True, total_charge=True, polarization=True)
        for s in range(len(systems)):
            _check_bec(res, off, systems, s, s % c_n, hp, params, elec)
        _sum_rule(res, off, elec.q_total)
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(71), n_candidates=1)
    elec = wl.Elec(mode=1, kind="ewald")
    one = wl.System(np.array([[1.0, 2.0, 3.0]], np.float32), np.array([2], np.int32), np.diag([9.0, 9.0, 9.0]),
                    wl.LLZO_SPECIES)
    empty = wl.System(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.diag([10.0, 10.0, 10.0]),
                      wl.LLZO_SPECIES)
    systems = [one, _llzo((1, 1, 1), 72), empty]
    res, off = _run(systems, hp, params, elec, dev, "fp32", bec=True, total_charge=True, polarization=True)
    for s in (0, 1):
        _check_bec(res, off, systems, s, 0, hp, params, elec)
    assert res["total_charge"][0, 2] == 0.0


def test_full_llzo_batch_bec_sum_rule_and_sampled_pairs(dev):
    """The 512 x 64 batch with BEC and total charges (tensor-core contraction): the sum rule on every
    pair, the largest and smallest cells' pairs against the oracle."""
    systems, hp, params, elec = wl.config_llzo_batch()
    res, off = _run(systems, hp, params, elec, dev, "bf16x3", bec=True, total_charge=True, polarization=True)
    assert np.isfinite(res["bec"]).all() and np.isfinite(res["total_charge"]).all()
    _sum_rule(res, off, elec.q_total)
    sizes = np.diff(off)
    for s, c in ((int(np.argmax(sizes)), 63), (int(np.argmin(sizes)), 2)):
        _check_bec(res, off, systems, s, c, hp, params, elec)


def test_full_loss_matches_oracle(dev):
    """qnep_batch_loss_full on a small batch's outputs (with BEC and total charges) against the
    oracle's loss_terms_full: D_e, D_v, the norms and D_Q in FP64 (relative 1e-12), D_f and D_Z
    from FP32 squares (relative 2e-6); one structure without reference BEC, one empty structure."""
    from paper_2601_19034_gb300.qnep import batch_loss_full
    empty = wl.System(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.diag([10.0, 10.0, 10.0]),
                      wl.LLZO_SPECIES)
    systems = [_llzo((1, 1, 1), 81), empty, _llzo((2, 1, 1), 82), _llzo((1, 1, 1), 83)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(84), n_candidates=5)
    elec = wl.Elec(mode=1, kind="ewald")
    res, off = _run(systems, hp, params, elec, dev, "bf16x3", virial=True, bec=True, total_charge=True,
                    polarization=True)
    rng = np.random.default_rng(85)
    n, s = int(off[-1]), len(systems)
    refs = {"energy": res["energy"][0] + rng.normal(size=s) * 3.0,
            "forces": (res["forces"][1] + rng.normal(size=(n, 3)) * 0.1).astype(np.float32),
            "virial": res["virial"][2] + rng.normal(size=(s, 3, 3)),
            "bec": (res["bec"][3] + rng.normal(size=(n, 3, 3)) * 0.05).astype(np.float32),
            "total_charge": rng.normal(size=s) * 0.1}
    has = np.array([1, 1, 0, 1], np.int32)
    weights = (1.0, 0.5, 0.2, 0.3, 0.7, 1e-3, 1e-4)
    outs = {k: torch.tensor(res[k], device=dev) for k in ("energy", "forces", "virial", "bec", "total_charge")}
    rd = {k: torch.tensor(np.ascontiguousarray(v), device=dev) for k, v in refs.items()}
    pd = torch.tensor(params, device=dev)
    offd = torch.tensor(off.astype(np.int32), device=dev)
    loss, terms = batch_loss_full(outs, rd, offd, torch.tensor(has, device=dev), pd, weights)
    ref = tr.loss_terms_full(res["energy"], res["forces"], res["virial"], res["bec"], res["total_charge"],
                             refs["energy"], refs["forces"], refs["virial"], refs["bec"], has.astype(bool),
                             refs["total_charge"], off, params)
    terms = terms.cpu().numpy()
    for k, rt in zip(range(7), (1e-12, 2e-6, 1e-12, 2e-6, 1e-12, 1e-12, 1e-12)):
        np.testing.assert_allclose(terms[:, k], ref[k], rtol=rt, err_msg=str(k))
    np.testing.assert_allclose(loss.cpu().numpy(), tr.loss_full(ref, *weights), rtol=2e-6)
    assert (terms[:, 3] > 0).all() and (terms[:, 4] > 0).all()
    # without BEC or total charges their terms are 0 and the rest unchanged
    loss0, terms0 = batch_loss_full({k: outs[k] for k in ("energy", "forces", "virial")},
                                    {k: rd[k] for k in ("energy", "forces", "virial")}, offd, None, pd, weights)
    t0 = terms0.cpu().numpy()
    assert (t0[:, 3] == 0).all() and (t0[:, 4] == 0).all()
    np.testing.assert_allclose(t0[:, [0, 1, 2, 5, 6]], terms[:, [0, 1, 2, 5, 6]], rtol=1e-12)


def test_host_buffer_call_with_every_output(dev):
    """qnep_batch_compute_host with BEC, total charges, polarization and virial requested: every
    output copied back to (pinned) host memory equals the device-buffer call's."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    systems = [_llzo((1, 1, 1), 91), _llzo((2, 1, 1), 92)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(93), n_candidates=3)
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.1)
    pos, typ, off, boxes = stack_structures(systems)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction("bf16x3")
    ref = b.compute(torch.tensor(pos, device=dev), torch.tensor(typ, device=dev), off, boxes, virial=True, bec=True,
                    total_charge=True, polarization=True)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    c, s_, n = 3, len(systems), int(off[-1])
    out = {"energy": torch.zeros(c, s_, dtype=torch.float64).pin_memory(),
           "forces": torch.zeros(c, n, 3).pin_memory(), "charges": torch.zeros(c, n).pin_memory(),
           "virial": torch.zeros(c, s_, 3, 3, dtype=torch.float64).pin_memory(),
           "bec": torch.zeros(c, n, 3, 3).pin_memory(),
           "total_charge": torch.zeros(c, s_, dtype=torch.float64).pin_memory(),
           "polarization": torch.zeros(c, s_, 3, dtype=torch.float64).pin_memory()}
    b.compute_host(torch.tensor(pos).pin_memory(), torch.tensor(typ).pin_memory(), off, boxes, out)
    b.close()
    for k, v in out.items():
        tol = 1e-9 if v.dtype == torch.float64 else 1e-5
        assert np.abs(v.numpy() - ref[k]).max() <= tol * max(1.0, float(np.abs(ref[k]).max())), k
