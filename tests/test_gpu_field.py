"""GPU parity of the field response (Sec. II.D, Eqs. electric_force and polarization_derivative).

qnep_field_response against the oracle's contractions, on the same inputs:
  * the chain force call -> Z -> F^ext, Pdot on a 320-atom BaTiO3 cell (two
    256-atom tiles, the second ragged) against the oracle's own Z;
  * seeded random Z, v and force arrays at sizes around the tile (0, 1, 255, 256,
    257, 1000, 65,537 atoms), with 16-byte-aligned and 4-byte-offset arrays, in
    every output combination, overwrite and accumulate;
  * the 4,194,304-atom launch the benchmark times: sampled atoms and the full Pdot;
  * NVE in a field (qnep_nve_run_field): one velocity-Verlet step under F + E.Z and the current
    of both states against the oracle; E = 0 against qnep_nve_run; momentum kept when Q = 0.
Tolerances: the kernel forms each component with three FP32 fused multiply-adds
(relative error <= 2^-22 of sum_a |E_a Z_i,ab|, bound here by 1e-6 of it); Pdot is a
compensated FP32 sum per thread, FP32 warp sums (5 roundings) and FP64 beyond, so its
error is <= 7 x 2^-24 < 1e-6 of sum_i sum_b |Z_i,ab v_i,b|.  Through the force call the BEC bound (1e-4 e) carries
over: |dF^ext| <= 1e-4 sum_a |E_a|, |dPdot_a| <= 1e-4 sum_i sum_b |v_i,b| (+ the FP32 term).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import field, forcecall, md  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19034_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _bounds(z, e, v):
    fb = np.einsum("a,iab->ib", np.abs(e), np.abs(z)) if e is not None else None
    pb = np.einsum("iab,ib->a", np.abs(z), np.abs(v)) if v is not None else None
    return fb, pb


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(n, 3, 3)).astype(np.float32)
    v = (rng.normal(size=(n, 3)) * 0.02).astype(np.float32)
    f0 = rng.normal(size=(n, 3)).astype(np.float32)
    return z, v, f0


def _on_device(a, dev, offset):
    """Copy a float32 array to the device, starting `offset` floats into a larger buffer."""
    flat = torch.zeros(a.size + offset + 4, dtype=torch.float32, device=dev)
    view = flat[offset:offset + a.size]
    view.copy_(torch.from_numpy(a.reshape(-1)))
    return view.view(a.shape)


def test_chain_from_force_call_batio3_320(dev):
    from paper_2601_19034_gb300.qnep import QNEP, field_response
    s = wl.batio3_supercell(4, seed=51)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(52))[0]
    elec = wl.Elec(mode=1, kind="ewald", q_total=0.3)
    model = QNEP(hp, params, elec)
    out = model.compute(torch.tensor(s.positions, device=dev), torch.tensor(s.types, device=dev), s.box)
    e = np.array([0.25, -0.4, 0.15])
    v = (np.random.default_rng(53).normal(size=(s.n_atoms, 3)) * 0.02).astype(np.float32)
    f, pdot = field_response(out["bec"], efield=e, velocities=torch.tensor(v, device=dev))
    torch.cuda.synchronize()
    ref = forcecall.force_call(s.positions.astype(np.float64), s.box, s.types, hp, params, elec)
    f_ref = field.electric_force(ref["bec"], e)
    p_ref = field.polarization_current(ref["bec"], v)
    assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-4 * np.abs(e).sum()
    fb, pb = _bounds(ref["bec"], None, v)
    assert np.all(np.abs(pdot.cpu().numpy() - p_ref) <= 1e-4 * np.abs(v).sum() + 1e-6 * pb)
    # sum rule of Eq. bec_2 carried through: sum_i F^ext_i = Q E
    np.testing.assert_allclose(f.cpu().double().numpy().sum(0), 0.3 * e, atol=1e-3)
    model.close()


@pytest.mark.parametrize("n", [0, 1, 255, 256, 257, 1000, 65537])
@pytest.mark.parametrize("offset", [0, 1])
def test_random_inputs_every_combination(dev, n, offset):
    from paper_2601_19034_gb300.qnep import field_response
    z, v, f0 = _inputs(n, seed=100 + n + offset)
    e = np.array([0.31, -0.17, 0.52])
    zd, vd = _on_device(z, dev, offset), _on_device(v, dev, offset)
    f_ref = field.electric_force(z, e)
    p_ref = field.polarization_current(z, v)
    fb, pb = _bounds(z, e, v)
    for want_f, want_p, acc in ((1, 1, 0), (1, 1, 1), (1, 0, 0), (1, 0, 1), (0, 1, 0)):
        fd = _on_device(f0, dev, offset) if want_f else None
        f, pdot = field_response(zd, efield=e if want_f else None, velocities=vd if want_p else None,
                                 forces=fd, accumulate=bool(acc))
        torch.cuda.synchronize()
        if want_f:
            expect = f_ref + (f0 if acc else 0.0)
            got = f.cpu().numpy()
            assert np.all(np.abs(got - expect) <= 1e-6 * fb + 2e-7 * np.abs(expect) + 1e-30), (want_p, acc)
        else:
            assert f is None
        if want_p:
            got_p = pdot.cpu().numpy()
            assert np.all(np.abs(got_p - p_ref) <= 1e-6 * pb + 1e-30), (got_p, p_ref)
        else:
            assert pdot is None


def test_full_size_launch_sampled(dev):
    """The benchmark's 4,194,304-atom launch: sampled forces, the whole Pdot."""
    from paper_2601_19034_gb300.qnep import field_response
    n = wl.FIELD_RESPONSE_ATOMS
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    zd = torch.randn(n, 3, 3, device=dev, generator=g)
    vd = torch.randn(n, 3, device=dev, generator=g) * 0.02
    e = np.array([0.12, 0.05, -0.33])
    f, pdot = field_response(zd, efield=e, velocities=vd)
    torch.cuda.synchronize()
    z = zd.cpu().numpy()
    v = vd.cpu().numpy()
    idx = np.random.default_rng(8).choice(n, 4096, replace=False)
    idx = np.concatenate([idx, [0, 255, 256, n - 1]])
    f_ref = field.electric_force(z[idx], e)
    fb, _ = _bounds(z[idx], e, None)
    assert np.all(np.abs(f.cpu().numpy()[idx] - f_ref) <= 1e-6 * fb + 1e-30)
    p_ref = field.polarization_current(z, v)
    _, pb = _bounds(z, None, v)
    assert np.all(np.abs(pdot.cpu().numpy() - p_ref) <= 1e-6 * pb)


def test_argument_errors(dev):
    from paper_2601_19034_gb300 import _lib
    lib = _lib.load()
    z = torch.zeros(10, 3, 3, device=dev)
    v = torch.zeros(10, 3, device=dev)
    f = torch.zeros(10, 3, device=dev)
    pd = torch.zeros(3, dtype=torch.float64, device=dev)
    e = (ctypes.c_double * 3)(0.1, 0.2, 0.3)
    bad = (ctypes.c_double * 3)(0.1, float("nan"), 0.3)
    s = torch.cuda.current_stream().cuda_stream
    call = lib.qnep_field_response
    assert call(-1, z.data_ptr(), e, v.data_ptr(), f.data_ptr(), 0, pd.data_ptr(), s) == _lib.QNEP_ERR_ARG
    assert call(10, z.data_ptr(), None, None, f.data_ptr(), 0, None, s) == _lib.QNEP_ERR_ARG       # no field
    assert call(10, z.data_ptr(), e, None, None, 0, pd.data_ptr(), s) == _lib.QNEP_ERR_ARG         # no velocities
    assert call(10, None, e, None, f.data_ptr(), 0, None, s) == _lib.QNEP_ERR_ARG                  # no Z
    assert call(10, z.data_ptr(), bad, None, f.data_ptr(), 0, None, s) == _lib.QNEP_ERR_ARG        # NaN field
    assert call(10, z.data_ptr() + 2, e, None, f.data_ptr(), 0, None, s) == _lib.QNEP_ERR_ARG      # misaligned
    assert call(10, z.data_ptr(), e, None, f.data_ptr(), 2, None, s) == _lib.QNEP_ERR_ARG          # accumulate flag
    assert call(10, z.data_ptr(), None, None, None, 0, None, s) == _lib.QNEP_OK                    # nothing asked
    torch.cuda.synchronize()


def _batio3_md():
    s = wl.batio3_supercell(4, seed=91)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(92))[0]
    # k-space-only electrostatics: the truncated real-space sum jumps at r_c, and this lattice has
    # many Ti-O pairs within 1e-4 A of 6 A, where FP32 and FP64 may classify a pair differently
    elec = wl.Elec(mode=2, kind="ewald")
    masses = wl.species_masses(wl.BATIO3_SPECIES)
    v0 = wl.maxwell_boltzmann(masses[s.types], 300.0, seed=93).astype(np.float32)
    return s, hp, params, elec, masses, v0


def test_nve_in_field_step_against_oracle(dev):
    """One velocity-Verlet step under F + E.Z, and Pdot of both states, against the oracle."""
    from paper_2601_19034_gb300.qnep import QNEP, nve_field
    s, hp, params, elec, masses, v0 = _batio3_md()
    m_atom = masses[s.types]
    e = np.array([0.05, -0.02, 0.08])
    dt = 0.5
    model = QNEP(hp, params, elec)
    pos = torch.tensor(s.positions, device=dev)
    vel = torch.tensor(v0, device=dev)
    f1, z1, en, pdot = nve_field(model, pos, vel, torch.tensor(s.types, device=dev), masses, s.box, dt, 1, e)
    torch.cuda.synchronize()
    assert model.sync_status() == 0
    x0 = s.positions.astype(np.float64)
    r0 = forcecall.force_call(x0, s.box, s.types, hp, params, elec)
    ft0 = r0["forces"] + field.electric_force(r0["bec"], e)
    x1 = md.positions_after_step(x0, v0, ft0, m_atom, dt)
    x1_gpu = pos.cpu().numpy()
    np.testing.assert_allclose(x1_gpu, x1, atol=2e-5)
    r1 = forcecall.force_call(x1_gpu.astype(np.float64), s.box, s.types, hp, params, elec)
    ft1 = r1["forces"] + field.electric_force(r1["bec"], e)
    np.testing.assert_allclose(f1.cpu().numpy(), ft1, atol=1e-4 + 1e-4 * np.abs(e).sum())
    np.testing.assert_allclose(z1.cpu().numpy(), r1["bec"], atol=1e-4)
    v1 = md.velocities_after_step(v0, ft0, ft1, m_atom, dt)
    v1_gpu = vel.cpu().numpy()
    np.testing.assert_allclose(v1_gpu, v1, atol=1e-6)
    p = pdot.cpu().numpy()
    for k, (z_ref, v) in enumerate(((r0["bec"], v0), (r1["bec"], v1_gpu))):
        p_ref = field.polarization_current(z_ref, v)
        assert np.all(np.abs(p[k] - p_ref) <= 1e-4 * np.abs(v).sum()), (k, p[k], p_ref)
    model.close()


def test_nve_in_zero_field_is_plain_nve_and_momentum_is_kept(dev):
    """E = 0 reproduces qnep_nve_run; in a field with Q = 0 the total momentum stays zero
    (sum_i F^ext_i = Q E by the sum rule of Eq. bec_2)."""
    from paper_2601_19034_gb300.qnep import QNEP, nve, nve_field
    s, hp, params, elec, masses, v0 = _batio3_md()
    m_atom = masses[s.types]
    typ = torch.tensor(s.types, device=dev)
    model = QNEP(hp, params, elec)
    pos_a, vel_a = torch.tensor(s.positions, device=dev), torch.tensor(v0, device=dev)
    nve(model, pos_a, vel_a, typ, masses, s.box, 0.5, 5)
    pos_b, vel_b = torch.tensor(s.positions, device=dev), torch.tensor(v0, device=dev)
    _, _, _, pdot = nve_field(model, pos_b, vel_b, typ, masses, s.box, 0.5, 5, (0.0, 0.0, 0.0))
    torch.cuda.synchronize()
    np.testing.assert_allclose(pos_b.cpu().numpy(), pos_a.cpu().numpy(), atol=1e-5)
    np.testing.assert_allclose(vel_b.cpu().numpy(), vel_a.cpu().numpy(), atol=1e-6)
    assert np.isfinite(pdot.cpu().numpy()).all()
    pos_c, vel_c = torch.tensor(s.positions, device=dev), torch.tensor(v0, device=dev)
    nve_field(model, pos_c, vel_c, typ, masses, s.box, 0.5, 10, (0.3, -0.2, 0.25))
    torch.cuda.synchronize()
    assert model.sync_status() == 0
    mom = (m_atom[:, None] * vel_c.cpu().numpy().astype(np.float64)).sum(0)
    scale = (m_atom[:, None] * np.abs(vel_c.cpu().numpy())).sum(0)
    assert np.all(np.abs(mom) <= 1e-4 * scale), (mom, scale)
    model.close()
