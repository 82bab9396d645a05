"""Pins of the oracle's field response (Sec. II.D, Eqs. electric_force and polarization_derivative).

The contractions are checked against what fixes them independently of the
einsum strings: for a cluster, where P = sum_i q~^c_i r_i is a function of the
positions, the external-field force is the gradient of E . P (central
differences) and the polarization current is dP/dt along r + t v (central
differences); for a periodic cell with total charge Q, the acoustic sum rule of
Eq. bec_2 (sum_i Z_i = Q I) fixes sum_i F^ext_i = Q E and, for a uniform
velocity, Pdot = Q v.  A transposed Z in either contraction fails the cluster
pins (the cluster Z is not symmetric), which the tests also show.
"""
import numpy as np
import pytest
import torch

from oracle import field
from oracle import forcecall as fc
from paper_2601_19034_gb300 import workloads as wl


@pytest.fixture(scope="module")
def cluster():
    rng = np.random.default_rng(41)
    pos = rng.uniform(-2.2, 2.2, size=(8, 3)) + 30.0
    types = rng.integers(0, 2, size=8)
    box = np.diag([60.0] * 3)
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(42))[0]
    elec = wl.Elec(mode=2, kind="ewald")
    p, leaf = fc.polarization_autograd(pos, box, types, hp, blob, elec)
    z = np.zeros((len(pos), 3, 3))
    for a in range(3):
        g = torch.autograd.grad(p[a], leaf, retain_graph=True)[0].numpy()
        z[:, a, :] = g          # Z_i,ab = dP_a / dr_ib
    return pos, box, types, hp, blob, elec, z


def _p(pos, box, types, hp, blob, elec):
    with torch.no_grad():
        return fc.polarization_autograd(pos, box, types, hp, blob, elec)[0].numpy()


def test_cluster_bec_is_not_symmetric(cluster):
    z = cluster[-1]
    assert np.abs(z - z.transpose(0, 2, 1)).max() > 1e-3


def test_cluster_electric_force_is_gradient_of_field_energy(cluster):
    pos, box, types, hp, blob, elec, z = cluster
    e = np.array([0.31, -0.17, 0.52])
    f = field.electric_force(z, e)
    h = 1e-5
    for i in (0, 3, 7):
        for b in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, b] += h
            pm[i, b] -= h
            fd = (e @ _p(pp, box, types, hp, blob, elec) - e @ _p(pm, box, types, hp, blob, elec)) / (2 * h)
            assert abs(fd - f[i, b]) < 1e-8
    # the transposed contraction is a different, wrong force
    wrong = np.einsum("b,iab->ia", e, z)
    assert np.abs(wrong - f).max() > 1e-4


def test_cluster_polarization_current_is_time_derivative(cluster):
    pos, box, types, hp, blob, elec, z = cluster
    v = np.random.default_rng(43).normal(size=pos.shape) * 0.01
    pdot = field.polarization_current(z, v)
    h = 1e-3
    fd = (_p(pos + h * v, box, types, hp, blob, elec) - _p(pos - h * v, box, types, hp, blob, elec)) / (2 * h)
    np.testing.assert_allclose(pdot, fd, atol=1e-10)
    wrong = np.einsum("iba,ib->a", z, v)
    assert np.abs(wrong - pdot).max() > 1e-6


def test_periodic_sum_rules():
    """Periodic Z (Eq. bec_2) with sum q~^c = Q: sum_i F^ext_i = Q E and Pdot(v uniform) = Q v."""
    s = wl.batio3_supercell(2, seed=31)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(32))[0]
    q_total = 0.7
    elec = wl.Elec(mode=1, kind="ewald", q_total=q_total)
    out = fc.force_call(s.positions.astype(np.float64), s.box, s.types, hp, blob, elec)
    z = out["bec"]
    e = np.array([-0.2, 0.45, 0.1])
    np.testing.assert_allclose(field.electric_force(z, e).sum(0), q_total * e, atol=1e-10)
    v = np.array([0.013, -0.004, 0.021])
    np.testing.assert_allclose(field.polarization_current(z, np.tile(v, (len(z), 1))), q_total * v, atol=1e-10)
    # and the field does work on the ions at the rate E . Pdot
    vr = np.random.default_rng(44).normal(size=(len(z), 3))
    power = (field.electric_force(z, e) * vr).sum()
    assert abs(power - e @ field.polarization_current(z, vr)) < 1e-10 * max(1.0, abs(power))
