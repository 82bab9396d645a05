"""GPU parity of the training loop around the batched call (Sec. II.E; SNES of Schaul et al. 2011).

qnep_snes_sample, qnep_batch_set_params, qnep_batch_loss and qnep_snes_update against
the oracle (oracle/training.py) on the same inputs:
  * sampling: one FP32 fused multiply-add per element, within 1 ulp of the FP64 value;
  * loss: seeded energies, forces and parameters (an empty structure, ragged force
    chunks), D_e / |z|_1 / |z|_2^2 in FP64 (relative 1e-12), D_f from FP32 squares of
    FP32 differences (relative 2e-6);
  * update: 64 candidates x the 4-species blob, losses with a tie and a NaN: identical
    ranks, so mu and sigma agree to the float32 rounding of the FP64 step (1e-6 relative);
  * set_params: a batch whose candidates are replaced on the device gives the outputs of a
    batch created with those candidates (up to the order of FP32 / FP64 atomics);
  * the chain on a small LLZO batch (targets from a teacher candidate): the device loss of
    the batched outputs equals the oracle loss of the same outputs, and one SNES step
    equals the oracle's step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import training as tr  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _t(a, dev, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device=dev, dtype=dtype)


def test_sample_matches_oracle(dev):
    from paper_2601_19034_gb300.qnep import snes_sample
    rng = np.random.default_rng(1)
    c, p = 37, 1001
    mu = rng.normal(size=p).astype(np.float32)
    sigma = (np.abs(rng.normal(size=p)) * 0.1).astype(np.float32)
    s = rng.normal(size=(c, p)).astype(np.float32)
    z = snes_sample(_t(mu, dev), _t(sigma, dev), _t(s, dev)).cpu().numpy()
    ref = tr.sample(mu, sigma, s)
    assert np.all(np.abs(z - ref) <= np.spacing(np.abs(ref).astype(np.float32)))


@pytest.mark.parametrize("sizes", [(192, 0, 384, 7, 1536), (1,), (300, 300)])
def test_loss_matches_oracle(dev, sizes):
    from paper_2601_19034_gb300.qnep import batch_loss
    rng = np.random.default_rng(len(sizes))
    c, p = 9, 613
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    n, s = int(off[-1]), len(sizes)
    e = rng.normal(size=(c, s)) * 50
    e_ref = rng.normal(size=s) * 50
    f = rng.normal(size=(c, n, 3)).astype(np.float32)
    f_ref = rng.normal(size=(n, 3)).astype(np.float32)
    z = rng.normal(size=(c, p)).astype(np.float32)
    weights = (1.0, 2.5, 0.01, 0.003)
    loss, terms = batch_loss(_t(e, dev), _t(f, dev), _t(e_ref, dev), _t(f_ref, dev), _t(off, dev), _t(z, dev),
                             weights)
    loss, terms = loss.cpu().numpy(), terms.cpu().numpy()
    d_e, d_f, l1, l2 = tr.loss_terms(e, f, e_ref, f_ref, off, z)
    np.testing.assert_allclose(terms[:, 0], d_e, rtol=1e-12)
    np.testing.assert_allclose(terms[:, 1], d_f, rtol=2e-6)
    np.testing.assert_allclose(terms[:, 2], l1, rtol=1e-12)
    np.testing.assert_allclose(terms[:, 3], l2, rtol=1e-12)
    np.testing.assert_allclose(loss, tr.loss((d_e, d_f, l1, l2), *weights), rtol=2e-6)
    # no forces, no parameters: D_f and the norms are zero
    loss0, terms0 = batch_loss(_t(e, dev), None, _t(e_ref, dev), None, _t(off, dev), None, weights)
    np.testing.assert_allclose(terms0.cpu().numpy()[:, 0], d_e, rtol=1e-12)
    assert np.all(terms0.cpu().numpy()[:, 1:] == 0.0)


def test_update_matches_oracle(dev):
    from paper_2601_19034_gb300.qnep import snes_update
    hp = wl.HParams(n_species=4)
    p, c = hp.n_params, 64
    rng = np.random.default_rng(3)
    mu = rng.normal(size=p).astype(np.float32) * 0.1
    sigma = (np.abs(rng.normal(size=p)) * 0.1 + 0.01).astype(np.float32)
    s = rng.normal(size=(c, p)).astype(np.float32)
    f = rng.normal(size=c)
    f[5] = f[17]           # a tie (broken by index)
    f[40] = np.nan         # ranks last
    mu_d, sg_d = _t(mu, dev), _t(sigma, dev)
    snes_update(_t(f, dev), _t(s, dev), mu_d, sg_d)
    mu_r, sg_r = tr.update(mu, sigma, s, f)
    np.testing.assert_allclose(mu_d.cpu().numpy(), mu_r, rtol=1e-6, atol=1e-6 * np.abs(sigma).max())
    np.testing.assert_allclose(sg_d.cpu().numpy(), sg_r, rtol=1e-6)
    # explicit rates
    mu_d, sg_d = _t(mu, dev), _t(sigma, dev)
    snes_update(_t(f, dev), _t(s, dev), mu_d, sg_d, eta_mu=0.5, eta_sigma=0.02)
    mu_r, sg_r = tr.update(mu, sigma, s, f, 0.5, 0.02)
    np.testing.assert_allclose(mu_d.cpu().numpy(), mu_r, rtol=1e-6, atol=1e-6 * np.abs(sigma).max())
    np.testing.assert_allclose(sg_d.cpu().numpy(), sg_r, rtol=1e-6)


def _small_batch():
    from tests.test_gpu_batch import _llzo
    systems = [_llzo((1, 1, 1), 61), _llzo((2, 1, 1), 62), _llzo((1, 1, 1), 63)]
    return systems


def test_set_params_equals_fresh_batch(dev):
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    systems = _small_batch()
    hp = wl.HParams(n_species=4)
    a = wl.random_params(hp, np.random.default_rng(71), n_candidates=35)
    b = wl.random_params(hp, np.random.default_rng(72), n_candidates=35)
    pos, typ, off, boxes = stack_structures(systems)
    pos_d, typ_d = _t(pos, dev), _t(typ, dev)
    elec = wl.Elec(mode=1, kind="ewald")
    ba = QNEPBatch(hp, a, elec)
    ba.compute(pos_d, typ_d, off, boxes)
    ba.set_params(_t(b.astype(np.float32), dev))
    out_a = ba.compute(pos_d, typ_d, off, boxes)
    bb = QNEPBatch(hp, b, elec)
    out_b = bb.compute(pos_d, typ_d, off, boxes)
    torch.cuda.synchronize()
    # the same arithmetic; only the order of the force and charge-sum atomics may differ
    assert torch.allclose(out_a["energy"], out_b["energy"], rtol=1e-12, atol=1e-9)
    assert (out_a["forces"] - out_b["forces"]).abs().max().item() <= 1e-5
    assert (out_a["charges"] - out_b["charges"]).abs().max().item() <= 1e-7
    ba.close()
    bb.close()


def test_one_training_iteration_chain(dev):
    """sample -> set_params -> batched call -> loss -> update, against the oracle on the same outputs."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, batch_loss, snes_sample, snes_update, stack_structures
    systems = _small_batch()
    hp = wl.HParams(n_species=4)
    p, c = hp.n_params, 32
    rng = np.random.default_rng(81)
    teacher = wl.random_params(hp, rng, n_candidates=1)[0].astype(np.float32)
    mu = (teacher + rng.normal(size=p) * 0.02).astype(np.float32)
    sigma = np.full(p, 0.01, np.float32)
    s = rng.normal(size=(c, p)).astype(np.float32)
    pos, typ, off, boxes = stack_structures(systems)
    pos_d, typ_d = _t(pos, dev), _t(typ, dev)
    elec = wl.Elec(mode=1, kind="ewald")
    tb = QNEPBatch(hp, teacher[None], elec)
    ref = tb.compute(pos_d, typ_d, off, boxes)
    e_ref, f_ref = ref["energy"][0].contiguous(), ref["forces"][0].contiguous()
    b = QNEPBatch(hp, np.repeat(mu[None], c, 0), elec)
    mu_d, sg_d, s_d = _t(mu, dev), _t(sigma, dev), _t(s, dev)
    z_d = snes_sample(mu_d, sg_d, s_d)
    b.set_params(z_d)
    out = b.compute(pos_d, typ_d, off, boxes, charges=False)
    weights = (1.0, 1.0, 1e-4, 1e-4)
    loss, terms = batch_loss(out["energy"], out["forces"], e_ref, f_ref, _t(off.astype(np.int32), dev), z_d, weights)
    loss_h = loss.cpu().numpy()
    snes_update(loss, s_d, mu_d, sg_d)
    torch.cuda.synchronize()
    terms_o = tr.loss_terms(out["energy"].cpu().numpy(), out["forces"].cpu().numpy(), e_ref.cpu().numpy(),
                            f_ref.cpu().numpy(), off, z_d.cpu().numpy())
    np.testing.assert_allclose(loss_h, tr.loss(terms_o, *weights), rtol=2e-6)
    assert np.isfinite(loss_h).all() and loss_h.min() > 0
    mu_r, sg_r = tr.update(mu, sigma, s, loss_h)
    np.testing.assert_allclose(mu_d.cpu().numpy(), mu_r, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(sg_d.cpu().numpy(), sg_r, rtol=1e-6)
    tb.close()
    b.close()


def test_argument_errors(dev):
    from paper_2601_19034_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(64, device=dev)
    d = torch.zeros(64, dtype=torch.float64, device=dev)
    w = _lib.LossWeightsC(1.0, 1.0, 0.0, 0.0)
    bad = _lib.LossWeightsC(float("inf"), 1.0, 0.0, 0.0)
    st = torch.cuda.current_stream().cuda_stream
    assert lib.qnep_snes_sample(0, 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), st) == _lib.QNEP_ERR_ARG
    assert lib.qnep_snes_update(1025, 4, d.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), -1.0, -1.0,
                                st) == _lib.QNEP_ERR_ARG
    off = torch.zeros(2, dtype=torch.int32, device=dev)
    # forces without references
    assert lib.qnep_batch_loss(1, 1, off.data_ptr(), 0, d.data_ptr(), x.data_ptr(), d.data_ptr(), None, None, 0,
                               w, d.data_ptr(), d.data_ptr(), st) == _lib.QNEP_ERR_ARG
    assert lib.qnep_batch_loss(1, 1, off.data_ptr(), 0, d.data_ptr(), None, d.data_ptr(), None, None, 0,
                               bad, d.data_ptr(), d.data_ptr(), st) == _lib.QNEP_ERR_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("sizes", [(192, 0, 384, 7, 1536), (300, 300)])
def test_loss_with_virial_matches_oracle(dev, sizes):
    """D_v (virial RMSE per atom over the six independent components) and the weighted sum."""
    from paper_2601_19034_gb300.qnep import batch_loss_v
    rng = np.random.default_rng(10 + len(sizes))
    c, p = 7, 301
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    n, s = int(off[-1]), len(sizes)
    e = rng.normal(size=(c, s)) * 50
    e_ref = rng.normal(size=s) * 50
    f = rng.normal(size=(c, n, 3)).astype(np.float32)
    f_ref = rng.normal(size=(n, 3)).astype(np.float32)
    w = rng.normal(size=(c, s, 3, 3)) * 30
    w_ref = rng.normal(size=(s, 3, 3)) * 30
    z = rng.normal(size=(c, p)).astype(np.float32)
    weights = (1.0, 0.5, 0.3, 0.01, 0.002)
    loss, terms = batch_loss_v(_t(e, dev), _t(f, dev), _t(w, dev), _t(e_ref, dev), _t(f_ref, dev), _t(w_ref, dev),
                               _t(off, dev), _t(z, dev), weights)
    terms = terms.cpu().numpy()
    ref = tr.loss_terms_v(e, f.astype(np.float64), w, e_ref, f_ref.astype(np.float64), w_ref, off,
                          z.astype(np.float64))
    np.testing.assert_allclose(terms[:, 0], ref[0], rtol=1e-12)
    np.testing.assert_allclose(terms[:, 1], ref[1], rtol=2e-6)
    np.testing.assert_allclose(terms[:, 2], ref[2], rtol=1e-12)
    np.testing.assert_allclose(terms[:, 3], ref[3], rtol=1e-12)
    np.testing.assert_allclose(terms[:, 4], ref[4], rtol=1e-12)
    np.testing.assert_allclose(loss.cpu().numpy(), tr.loss_v(ref, *weights), rtol=2e-6)
    # no virial given: D_v = 0 and the rest unchanged
    loss0, terms0 = batch_loss_v(_t(e, dev), _t(f, dev), None, _t(e_ref, dev), _t(f_ref, dev), None, _t(off, dev),
                                 _t(z, dev), weights)
    assert np.all(terms0.cpu().numpy()[:, 2] == 0.0)
    np.testing.assert_allclose(terms0.cpu().numpy()[:, [0, 1, 3, 4]], terms[:, [0, 1, 3, 4]], rtol=1e-12)


def test_static_geometry_keeps_the_prepass_and_follows_changes(dev):
    """qnep_batch_set_static_geometry: calls after the first reuse its pre-pass and give the outputs
    of full calls, new candidates included (the training loop's case); a captured call replays
    without the pre-pass; after an in-place move of the positions and qnep_batch_geometry_changed
    the next call equals a full call on the moved structures; a contraction change rebuilds."""
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    from tests.test_gpu_batch import _llzo
    systems = [_llzo((1, 1, 1), 141), _llzo((2, 1, 1), 142)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(143), n_candidates=5)
    params2 = wl.random_params(hp, np.random.default_rng(144), n_candidates=5)
    elec = wl.Elec(mode=1, kind="ewald")
    pos, typ, off, boxes = stack_structures(systems)
    pd, td = _t(pos, dev), _t(typ, dev)

    def full(prm, positions, contract="bf16x3"):
        f = QNEPBatch(hp, prm, elec)
        f.set_contraction(contract)
        o = {k: v.clone() for k, v in f.compute(positions, td, off, boxes).items()}
        f.close()
        return o

    def same(a, b_):
        n = np.diff(off)
        assert ((a["energy"] - b_["energy"]).abs().cpu().numpy() / n[None]).max() <= 1e-9
        assert (a["forces"] - b_["forces"]).abs().max().item() <= 1e-5
        assert (a["charges"] - b_["charges"]).abs().max().item() <= 1e-6

    b = QNEPBatch(hp, params, elec)
    b.set_contraction("bf16x3")
    b.set_static_geometry(True)
    same(b.compute(pd, td, off, boxes), full(params, pd))          # builds the geometry
    b.set_params(_t(params2, dev))
    same(b.compute(pd, td, off, boxes), full(params2, pd))         # reuses it, new candidates
    out = b.outputs(len(off) - 1, pos.shape[0], dev)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.compute_into(pd, td, off, boxes, out, stream=stream.cuda_stream)
    for v in out.values():
        v.zero_()
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    same(out, full(params2, pd))
    del g
    pd.add_(0.05)                                                   # the structures move in place
    b.geometry_changed()
    same(b.compute(pd, td, off, boxes), full(params2, pd))
    b.set_contraction("fp32")                                       # FP32 B^A sums are built anew
    same(b.compute(pd, td, off, boxes), full(params2, pd, "fp32"))
    b.close()


def test_static_geometry_reports_the_kept_prepass_status(dev):
    """A list overflow recorded by the pre-pass whose geometry is kept is reported by the calls
    that reuse it, not only by the call that built it; the report ends the reuse (the next call
    runs the pre-pass again), and with capacities from the density again the outputs are those of
    a fresh batch."""
    from paper_2601_19034_gb300 import _lib
    from paper_2601_19034_gb300.qnep import QNEPBatch, stack_structures
    from tests.test_gpu_batch import _llzo
    systems = [_llzo((1, 1, 1), 151)]
    hp = wl.HParams(n_species=4)
    params = wl.random_params(hp, np.random.default_rng(152), n_candidates=2)
    elec = wl.Elec(mode=1, kind="ewald")
    pos, typ, off, boxes = stack_structures(systems)
    pd, td = _t(pos, dev), _t(typ, dev)
    b = QNEPBatch(hp, params, elec)
    b.set_static_geometry(True)
    b.set_capacity(32, 16)             # ~80 neighbours within 6 A and ~24 within 4 A in LLZO: both overflow
    out = b.outputs(1, pos.shape[0], dev)
    b.compute_into(pd, td, off, boxes, out)                         # builds the kept geometry, unchecked
    b.compute_into(pd, td, off, boxes, out)                         # reuses it
    assert b.sync_status() == _lib.QNEP_ERR_NBR_OVERFLOW
    b.compute_into(pd, td, off, boxes, out)                         # the pre-pass runs again
    assert b.sync_status() == _lib.QNEP_ERR_NBR_OVERFLOW
    b.set_capacity(0, 0)                                            # capacities from the density
    got = b.compute(pd, td, off, boxes)
    fresh = QNEPBatch(hp, params, elec)
    ref = fresh.compute(pd, td, off, boxes)
    assert (got["energy"] - ref["energy"]).abs().max().item() / pos.shape[0] <= 1e-9
    assert (got["forces"] - ref["forces"]).abs().max().item() <= 1e-5
    assert (got["charges"] - ref["charges"]).abs().max().item() <= 1e-6
    fresh.close()
    b.close()
