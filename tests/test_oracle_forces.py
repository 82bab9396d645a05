"""Pins of the oracle's force call: finite differences, invariants, replication.

Forces and the virial are checked against central finite differences of the
total energy (h = 1e-4 A, strain +-1e-6), the periodic BEC per-entry
derivatives against finite differences of one neighbour-entry vector, the
cluster BEC (Eq. bec_1, relative-vector form with the charge correction
differentiated) against finite differences of P, plus the charge constraint,
zero net force, translation invariance and supercell replication.
"""
import numpy as np
import pytest
import torch

from oracle import descriptor as dm
from oracle import forcecall as fc
from oracle import geometry, network
from oracle.params import unpack
from paper_2601_19034_gb300 import workloads as wl


def _energy(pos, box, types, hp, blob, elec):
    with torch.no_grad():
        e, _, _ = fc.total_energy_autograd(pos, box, types, hp, blob, elec)
    return float(e)


@pytest.fixture(scope="module")
def batio3_subcell():
    """40-atom BaTiO3 2x2x2 cell (edge 8 A < 2 r_c: several images per pair)."""
    s = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(32))[0]
    elec = wl.Elec(mode=1, kind="ewald")
    return s.positions.astype(np.float64), s.box, s.types, hp, blob, elec


def test_forces_match_central_differences(batio3_subcell):
    pos, box, types, hp, blob, elec = batio3_subcell
    out = fc.force_call(pos, box, types, hp, blob, elec)
    h = 1e-4
    for i in (0, 7, 23, 39):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = -(_energy(pp, box, types, hp, blob, elec) - _energy(pm, box, types, hp, blob, elec)) / (2 * h)
            assert abs(fd - out["forces"][i, d]) < 2e-6 * max(1.0, abs(fd))
    assert np.abs(out["forces"].sum(0)).max() < 1e-9


def test_mode2_forces_match_central_differences(batio3_subcell):
    pos, box, types, hp, blob, _ = batio3_subcell
    elec = wl.Elec(mode=2, kind="ewald")
    out = fc.force_call(pos, box, types, hp, blob, elec)
    h = 1e-4
    for i, d in ((3, 0), (17, 2)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += h
        pm[i, d] -= h
        fd = -(_energy(pp, box, types, hp, blob, elec) - _energy(pm, box, types, hp, blob, elec)) / (2 * h)
        assert abs(fd - out["forces"][i, d]) < 2e-6 * max(1.0, abs(fd))


def test_virial_matches_strain_differences(batio3_subcell):
    pos, box, types, hp, blob, elec = batio3_subcell
    out = fc.force_call(pos, box, types, hp, blob, elec)
    h = 1e-6
    for a, b in ((0, 0), (1, 1), (0, 1), (2, 1)):
        eps = np.zeros((3, 3))
        eps[a, b] = h
        defp, defm = np.eye(3) + eps, np.eye(3) - eps
        ep = _energy(pos @ defp.T, box @ defp.T, types, hp, blob, elec)
        em = _energy(pos @ defm.T, box @ defm.T, types, hp, blob, elec)
        # W = -(dU/d eps)^T
        assert abs(-(ep - em) / (2 * h) - out["virial"][b, a]) < 1e-4 * max(1.0, abs(out["virial"][b, a]))
    np.testing.assert_allclose(out["virial"], out["virial"].T, atol=1e-8)


def test_charge_correction_and_bec_sum_rule(batio3_subcell):
    pos, box, types, hp, blob, elec = batio3_subcell
    for q_total in (0.0, 0.7):
        e = wl.Elec(mode=1, kind="ewald", q_total=q_total)
        out = fc.force_call(pos, box, types, hp, blob, e)
        assert abs(out["qtilde"].sum() - q_total) < 1e-12
        s = blob[-1]
        np.testing.assert_allclose(out["charges"] * s, out["qtilde"], rtol=1e-12)
        np.testing.assert_allclose(out["bec"].sum(0), q_total * np.eye(3), atol=1e-10)


def test_translation_invariance(batio3_subcell):
    pos, box, types, hp, blob, elec = batio3_subcell
    out = fc.force_call(pos, box, types, hp, blob, elec)
    shifted = (pos + np.array([1.37, -2.11, 0.53])) % 8.0
    out2 = fc.force_call(shifted, box, types, hp, blob, elec)
    assert abs(out["energy"] - out2["energy"]) < 1e-9
    np.testing.assert_allclose(out2["forces"], out["forces"], atol=1e-9)
    np.testing.assert_allclose(out2["charges"], out["charges"], atol=1e-12)
    np.testing.assert_allclose(out2["bec"], out["bec"], atol=1e-9)


def test_supercell_replication_with_electrostatics(batio3_subcell):
    pos, box, types, hp, blob, elec = batio3_subcell
    out1 = fc.force_call(pos, box, types, hp, blob, elec, want_bec=False)
    shifts = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    big = (pos[None] + shifts[:, None, :] * 8.0).reshape(-1, 3)
    out8 = fc.force_call(big, box * 2, np.tile(types, 8), hp, blob, elec, want_bec=False)
    assert abs(out8["energy"] - 8 * out1["energy"]) < 1e-8 * abs(out8["energy"])
    np.testing.assert_allclose(out8["forces"], np.tile(out1["forces"], (8, 1)), atol=1e-8)
    np.testing.assert_allclose(out8["virial"], 8 * out1["virial"], rtol=1e-8, atol=1e-7)


def test_bec_entry_derivative_matches_finite_difference(batio3_subcell):
    """a_ij = d q~_i / d r_ij: perturb one neighbour-entry vector, not an atom."""
    pos, box, types, hp, blob, elec = batio3_subcell
    model = unpack(blob, hp)
    ent = geometry.neighbor_entries(pos, box, hp.rc_radial)
    i = 5
    sel = np.nonzero(ent.i == i)[0]
    vec = ent.vec[sel].copy()
    angular = np.linalg.norm(vec, axis=1) < hp.rc_angular

    def qtilde(v):
        vt = torch.as_tensor(v)
        d = dm.descriptor(vt, ent.i[sel], ent.j[sel], vt[angular], ent.i[sel][angular],
                          ent.j[sel][angular], types, np.array([i]), model)
        return model.sqrt_eps_inf * float(network.site_energy_and_charge(d, types[[i]], model)[1][0])

    vt = torch.tensor(vec, requires_grad=True)
    d = dm.descriptor(vt, ent.i[sel], ent.j[sel], vt[angular], ent.i[sel][angular], ent.j[sel][angular],
                      types, np.array([i]), model)
    q = model.sqrt_eps_inf * network.site_energy_and_charge(d, types[[i]], model)[1][0]
    a = torch.autograd.grad(q, vt)[0].numpy()
    h = 1e-5
    for e in (0, 3, len(sel) - 1):
        for dd in range(3):
            vp, vm = vec.copy(), vec.copy()
            vp[e, dd] += h
            vm[e, dd] -= h
            assert abs((qtilde(vp) - qtilde(vm)) / (2 * h) - a[e, dd]) < 1e-8
    # the oracle's periodic BEC (Eq. bec_2) is built from these a_ij: its row sums over the
    # entries of atom i reproduce 1/2 sum_j r_ij (x) a_ij once the reverse entries are removed
    out = fc.force_call(pos, box, types, hp, blob, elec)
    own = 0.5 * np.einsum("ea,eb->ab", vec, a)
    assert np.abs(own).max() > 0


def test_cluster_bec_relative_form_matches_dp_dr():
    """Cluster: Z_i = dP/dr_i (FD) equals Eq. bec_1 in relative vectors.

    With the total-charge correction differentiated, the relative form is
    Z_i = q~^c_i I + sum_{(j->i)} (r_j - rbar) (x) a_ji - sum_{(i->k)} (r_i - rbar) (x) a_ik.
    """
    rng = np.random.default_rng(14)
    pos = rng.uniform(-2.2, 2.2, size=(8, 3)) + 30.0
    types = rng.integers(0, 2, size=8)
    box = np.diag([60.0] * 3)
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(15))[0]
    elec = wl.Elec(mode=2, kind="ewald")
    out = fc.force_call(pos, box, types, hp, blob, elec)
    ent_r = geometry.neighbor_entries(pos, box, hp.rc_radial)
    # per-entry a from the oracle's own staged chain rule (radial list contains the angular pairs)
    model = unpack(blob, hp)
    vt = torch.tensor(ent_r.vec, requires_grad=True)
    ang = np.linalg.norm(ent_r.vec, axis=1) < hp.rc_angular
    d = dm.descriptor(vt, ent_r.i, ent_r.j, vt[ang], ent_r.i[ang], ent_r.j[ang], types,
                      np.arange(len(pos)), model)
    q = network.site_energy_and_charge(d, types, model)[1]
    a = torch.autograd.grad(model.sqrt_eps_inf * q.sum(), vt)[0].numpy()
    rbar = pos.mean(0)
    z = out["qtilde"][:, None, None] * np.eye(3)[None]
    for e in range(len(ent_r.i)):
        i, j = ent_r.i[e], ent_r.j[e]
        z[j] += np.outer(pos[i] - rbar, a[e])
        z[i] -= np.outer(pos[i] - rbar, a[e])
    h = 1e-5
    for i in (0, 4):
        for b in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, b] += h
            pm[i, b] -= h
            with torch.no_grad():
                p_plus = fc.polarization_autograd(pp, box, types, hp, blob, elec)[0].numpy()
                p_minus = fc.polarization_autograd(pm, box, types, hp, blob, elec)[0].numpy()
            np.testing.assert_allclose((p_plus - p_minus) / (2 * h), z[i][:, b], atol=1e-8)


def test_charge_gradient_matches_finite_differences(batio3_subcell):
    """d(sum_i c_i q^c_i)/dr by autograd against central differences (charge correction included)."""
    pos, box, types, hp, blob, elec = batio3_subcell
    c = np.random.default_rng(3).normal(size=len(pos))
    qc, leaf = fc.charges_autograd(pos, box, types, hp, blob, elec)
    (torch.as_tensor(c) * qc).sum().backward()
    grad = leaf.grad.numpy()
    h = 1e-5
    for i, d in ((1, 0), (22, 2), (35, 1)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += h
        pm[i, d] -= h
        with torch.no_grad():
            fp = float((torch.as_tensor(c) * fc.charges_autograd(pp, box, types, hp, blob, elec)[0]).sum())
            fm = float((torch.as_tensor(c) * fc.charges_autograd(pm, box, types, hp, blob, elec)[0]).sum())
        assert abs((fp - fm) / (2 * h) - grad[i, d]) < 1e-7
    # and it agrees with the staged force call's charges
    out = fc.force_call(pos, box, types, hp, blob, elec, want_bec=False)
    np.testing.assert_allclose(qc.detach().numpy(), out["charges"], atol=1e-12)


def test_periodic_bec_is_dp_dr_for_an_isolated_dimer():
    """For two atoms alone in a large box, Eq. bec_2 (raw per-entry charge derivatives, corrected
    charge on the diagonal) must equal the exact dP/dr_i: with q~^c_A = (q~_A - q~_B) / 2 and
    P = -q~^c_A r_AB, both give Z_A = q~^c_A I + 1/2 (q~_A' - q~_B') r_AB (x) r_AB / r.
    This fixes the factor 1/2 of Eq. bec_2, which the sum rule and translation do not."""
    pos = np.array([[30.0, 30.0, 30.0], [31.1, 30.9, 30.7]])       # 1.59 A: radial and angular terms
    types = np.array([0, 1])
    box = np.diag([60.0] * 3)
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(23))[0]
    elec = wl.Elec(mode=2, kind="ewald")
    z = fc.force_call(pos, box, types, hp, blob, elec)["bec"]
    h = 1e-5
    for i in range(2):
        for b in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, b] += h
            pm[i, b] -= h
            with torch.no_grad():
                dp = (fc.polarization_autograd(pp, box, types, hp, blob, elec)[0].numpy()
                      - fc.polarization_autograd(pm, box, types, hp, blob, elec)[0].numpy()) / (2 * h)
            np.testing.assert_allclose(z[i][:, b], dp, atol=1e-8)
    assert np.abs(z[0] - z[0][0, 0] * np.eye(3)).max() > 1e-3      # the off-diagonal part is exercised


@pytest.mark.parametrize("q_total", [0.0, 0.7])
def test_polarization_moves_by_q_total_under_translation(q_total):
    """P = sum_i q~^c_i r_i (Eq. polarization, positions as given): a uniform shift d of all atoms
    leaves the charges unchanged and moves P by (sum_i q~^c_i) d = Q d exactly (the corrected
    charges meet the target Q; the uncorrected ones would not)."""
    rng = np.random.default_rng(29)
    pos = rng.uniform(-2.5, 2.5, size=(9, 3)) + 30.0
    types = rng.integers(0, 3, size=9)
    box = np.diag([60.0] * 3)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(30))[0]
    elec = wl.Elec(mode=2, kind="ewald", q_total=q_total)
    d = np.array([0.37, -1.21, 0.58])
    p0 = fc.force_call(pos, box, types, hp, blob, elec, want_bec=False)["polarization"]
    p1 = fc.force_call(pos + d, box, types, hp, blob, elec, want_bec=False)["polarization"]
    np.testing.assert_allclose(p1 - p0, q_total * d, atol=1e-11)


def test_network_with_zero_input_weights_is_a_closed_form(batio3_subcell):
    """Every first-layer weight W0 = 0: the hidden layer is tanh(-b0) of the central atom's species
    (Eq. U_i with the bias subtracted), so U_i = sum_mu w1E tanh(-b0) - b1E and q_i likewise are
    constants per species, whatever the descriptor.  Then the charges do not move with the atoms:
    the forces are the static electrostatic forces of those fixed charges, the BEC are q~^c times
    the identity, and the NEP energy is the sum of the per-species constants (numpy's tanh)."""
    from oracle import ewald
    pos, box, types, hp, blob, elec = batio3_subcell
    blob = np.array(blob, dtype=np.float32)
    s, nn, nd = hp.n_species, hp.n_neurons, hp.n_des
    o = s * s * (hp.n_radial * hp.basis_radial + hp.n_angular * hp.basis_angular) + nd
    u_t, q_t = [], []
    for _ in range(s):
        blob[o:o + nn * nd] = 0.0                      # W0
        o += nn * nd
        b0 = blob[o:o + nn].astype(np.float64)
        w1e = blob[o + nn:o + 2 * nn].astype(np.float64)
        w1q = blob[o + 2 * nn:o + 3 * nn].astype(np.float64)
        b1e, b1q = float(blob[o + 3 * nn]), float(blob[o + 3 * nn + 1])
        u_t.append(float((w1e * np.tanh(-b0)).sum()) - b1e)
        q_t.append(float((w1q * np.tanh(-b0)).sum()) - b1q)
        o += 3 * nn + 2
    out = fc.force_call(pos, box, types, hp, blob, elec)
    np.testing.assert_allclose(out["site_energy"], np.asarray(u_t)[types], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["q_raw"], np.asarray(q_t)[types], rtol=0, atol=1e-12)
    assert abs(out["e_nep"] - float(np.asarray(u_t)[types].sum())) < 1e-10
    ent_real = geometry.neighbor_entries(pos, box, elec.rc_real)
    static = ewald.ewald_static(pos, box, out["charges"], ent_real, elec)
    np.testing.assert_allclose(out["forces"], static["force"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["bec"], out["qtilde"][:, None, None] * np.eye(3)[None], rtol=0, atol=1e-12)
