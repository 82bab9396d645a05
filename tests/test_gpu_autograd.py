"""Differentiation form: QNEPFunction (autograd) against the oracle gradient and finite differences.

loss = a U^tot + sum_i c_i q^c_i + d . P.  The oracle gradient is
-a F (autograd of the energy) + autograd of sum c q^c + d . Z (periodic BEC, Eq. bec_2),
and the GPU result comes from one qnep_compute_vjp backward.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import forcecall  # noqa: E402
from paper_2601_19034_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _oracle_grad(sysm, hp, params, elec, a, c, d):
    pos = sysm.positions.astype(np.float64)
    ref = forcecall.force_call(pos, sysm.box, sysm.types, hp, params, elec)
    qc, leaf = forcecall.charges_autograd(pos, sysm.box, sysm.types, hp, params, elec)
    (torch.as_tensor(c) * qc).sum().backward()
    grad = -a * ref["forces"] + leaf.grad.numpy() + np.einsum("a,iab->ib", d, ref["bec"])
    return grad, ref


@pytest.mark.parametrize("path", ["warp", "thread"])
def test_autograd_matches_oracle_gradient(dev, path):
    from paper_2601_19034_gb300.qnep import QNEP, qnep_energy
    s = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(32))[0]
    elec = wl.Elec(mode=1, kind="ewald")
    model = QNEP(hp, params, elec)
    model.set_path(path)
    rng = np.random.default_rng(9)
    a, c, d = 0.7, rng.normal(size=s.n_atoms), np.array([0.3, -0.5, 0.2])
    pos = torch.tensor(s.positions, device=dev, requires_grad=True)
    typ = torch.tensor(s.types, device=dev)
    e, q, p = qnep_energy(model, pos, typ, s.box)
    loss = a * e + (torch.as_tensor(c, device=dev) * q).sum() + (torch.as_tensor(d, device=dev) * p).sum()
    loss.backward()
    ref_grad, ref = _oracle_grad(s, hp, params, elec, a, c, d)
    assert abs(e.item() - ref["energy"]) / s.n_atoms < 1e-6
    np.testing.assert_allclose(q.detach().cpu().numpy(), ref["charges"], atol=2e-6)
    np.testing.assert_allclose(p.detach().cpu().numpy(), ref["polarization"], atol=1e-5 * s.n_atoms)
    err = np.abs(pos.grad.cpu().numpy() - ref_grad).max()
    assert err < 1e-4, err


def test_energy_gradient_is_minus_forces_and_finite_differences(dev):
    from paper_2601_19034_gb300.qnep import QNEP, qnep_energy
    sysm, hp, params, elec = wl.config_water_small()
    model = QNEP(hp, params, elec)
    typ = torch.tensor(sysm.types, device=dev)
    pos = torch.tensor(sysm.positions, device=dev, requires_grad=True)
    e, _, _ = qnep_energy(model, pos, typ, sysm.box)
    e.backward()
    forces = model.compute(pos.detach(), typ, sysm.box)["forces"]
    assert (pos.grad + forces).abs().max().item() < 2e-5
    # central differences of the GPU energy itself (h = 5e-3 A: FP32 noise ~1e-4 eV/A, O(h^2) truncation)
    h = 5e-3
    for i, dd in ((0, 0), (40, 1), (191, 2)):
        pp = pos.detach().clone()
        pm = pos.detach().clone()
        pp[i, dd] += h
        pm[i, dd] -= h
        ep = model.compute(pp, typ, sysm.box, forces=False, bec=False, virial=False)["scalars"][0].item()
        em = model.compute(pm, typ, sysm.box, forces=False, bec=False, virial=False)["scalars"][0].item()
        assert abs((ep - em) / (2 * h) - pos.grad[i, dd].item()) < 2e-3


def test_autograd_large_system_gradient_consistency(dev):
    """5000-atom BaTiO3: the VJP with only g_E equals minus the forces of qnep_compute."""
    from paper_2601_19034_gb300.qnep import QNEP
    sysm, hp, params, elec = wl.config_batio3()
    model = QNEP(hp, params, elec)
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    f = model.compute(pos, typ, sysm.box)["forces"]
    g = model.vjp(pos, typ, sysm.box, 1.0)
    assert (g + f).abs().max().item() < 2e-5


@pytest.mark.parametrize("kind", ["ewald", "pppm"])
def test_autograd_in_a_general_cell(dev, kind):
    """The differentiation form in a sheared perovskite cell (every off-diagonal element non-zero):
    the gradient of a U + sum c q^c + d . P against the oracle's, Ewald and PPPM."""
    from paper_2601_19034_gb300.qnep import QNEP, qnep_energy
    s0 = wl.batio3_supercell(3, seed=33)
    box = s0.box + np.array([[0.0, 0.4, -0.3], [0.9, 0.0, 0.5], [-0.7, 1.1, 0.0]])
    pos0 = (s0.positions.astype(np.float64) @ np.linalg.inv(s0.box)) @ box
    s = wl.System(pos0.astype(np.float32), s0.types, box, s0.species)
    hp = wl.HParams(n_species=3)
    params = wl.random_params(hp, np.random.default_rng(34))[0]
    elec = wl.Elec(mode=1, kind=kind, q_total=0.2, mesh=(16, 16, 16), order=5)
    model = QNEP(hp, params, elec)
    rng = np.random.default_rng(35)
    a, c, d = 0.7, rng.normal(size=s.n_atoms), np.array([0.3, -0.5, 0.2])
    pos = torch.tensor(s.positions, device=dev, requires_grad=True)
    typ = torch.tensor(s.types, device=dev)
    e, q, p = qnep_energy(model, pos, typ, s.box)
    loss = a * e + (torch.as_tensor(c, device=dev) * q).sum() + (torch.as_tensor(d, device=dev) * p).sum()
    loss.backward()
    ref_grad, ref = _oracle_grad(s, hp, params, elec, a, c, d)
    assert abs(e.item() - ref["energy"]) / s.n_atoms < 1e-6
    err = np.abs(pos.grad.cpu().numpy() - ref_grad).max()
    assert err < 1e-4, err
    model.close()
