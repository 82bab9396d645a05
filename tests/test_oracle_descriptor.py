"""Pins of the oracle's descriptor and network (CPU only).

Each test checks the oracle against something other than itself: library
polynomials, the spherical-harmonic addition theorem (scipy), a brute-force
triple sum, symmetry invariances and supercell replication.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
import torch

from oracle import descriptor as dm
from oracle import geometry, network
from oracle.forcecall import descriptors
from oracle.params import unpack
from paper_2601_19034_gb300 import workloads as wl


def test_chebyshev_matches_numpy():
    x = torch.linspace(-1, 1, 101, dtype=torch.float64)
    t = dm.chebyshev_t(x, 9).numpy()
    for k in range(9):
        c = np.zeros(k + 1)
        c[k] = 1
        np.testing.assert_allclose(t[:, k], np.polynomial.chebyshev.chebval(x.numpy(), c), atol=1e-13)


def test_legendre_matches_scipy():
    c = torch.linspace(-1, 1, 77, dtype=torch.float64)
    p = dm.legendre(c, 4).numpy()
    for l in range(1, 5):
        np.testing.assert_allclose(p[:, l - 1], sp.eval_legendre(l, c.numpy()), atol=1e-13)


def test_cutoff_and_basis_edges():
    rc = 6.0
    r = torch.tensor([1e-9, rc * (1 - 1e-12)], dtype=torch.float64)
    fc = dm.cutoff_function(r, rc).numpy()
    assert abs(fc[0] - 1) < 1e-12 and abs(fc[1]) < 1e-12
    f = dm.basis_functions(r, rc, 9).numpy()
    # at r -> 0, x = 1 and T_k(1) = 1, so every f_k -> f_c = 1
    np.testing.assert_allclose(f[0], 1.0, atol=1e-9)
    np.testing.assert_allclose(f[1], 0.0, atol=1e-12)


def _cluster(n=7, seed=3):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.8, 1.8, size=(n, 3)) + 20.0
    types = rng.integers(0, 2, size=n)
    box = np.diag([40.0, 40.0, 40.0])
    return pos, types, box


def _sph_y(l, m, polar, azim):
    if hasattr(sp, "sph_harm_y"):
        return sp.sph_harm_y(l, m, polar, azim)
    return sp.sph_harm(m, l, azim, polar)  # older scipy argument order


def test_angular_descriptor_addition_theorem():
    """D^A_{nl} = 4 pi / (2l+1) sum_m |sum_j g_n(r_ij) Y_lm(u_ij)|^2 (complex Y, scipy)."""
    hp = wl.HParams(n_species=2, rc_radial=6.0, rc_angular=4.0)
    blob = wl.random_params(hp, np.random.default_rng(5))[0]
    model = unpack(blob, hp)
    pos, types, box = _cluster()
    d = descriptors(pos, box, types, hp, blob)
    ent = geometry.neighbor_entries(pos, box, hp.rc_angular)
    r = np.linalg.norm(ent.vec, axis=1)
    g = dm.radial_functions(torch.as_tensor(r), types[ent.i], types[ent.j], model.c_angular,
                            hp.rc_angular).numpy()
    polar = np.arccos(np.clip(ent.vec[:, 2] / r, -1, 1))
    azim = np.arctan2(ent.vec[:, 1], ent.vec[:, 0])
    nr = hp.n_radial
    for i in range(len(pos)):
        sel = ent.i == i
        for l in range(1, 5):
            ylm = np.stack([_sph_y(l, m, polar[sel], azim[sel]) for m in range(-l, l + 1)], 1)
            a = g[sel].T @ ylm                                       # [n, 2l+1]
            ref = 4 * math.pi / (2 * l + 1) * (np.abs(a) ** 2).sum(1)
            got = d[i, nr + (l - 1) * hp.n_angular: nr + l * hp.n_angular]
            np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_four_body_brute_force_triple_sum():
    """tr(T^3) equals the explicit triple sum over neighbours j, k, m."""
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(6))[0]
    model = unpack(blob, hp)
    pos, types, box = _cluster(6, seed=11)
    d = descriptors(pos, box, types, hp, blob)
    ent = geometry.neighbor_entries(pos, box, hp.rc_angular)
    r = np.linalg.norm(ent.vec, axis=1)
    u = ent.vec / r[:, None]
    g = dm.radial_functions(torch.as_tensor(r), types[ent.i], types[ent.j], model.c_angular,
                            hp.rc_angular).numpy()
    off = hp.n_radial + 4 * hp.n_angular
    for i in range(len(pos)):
        sel = np.nonzero(ent.i == i)[0]
        ref = np.zeros(hp.n_angular)
        for a in sel:
            for b in sel:
                for c in sel:
                    ab, bc, ca = u[a] @ u[b], u[b] @ u[c], u[c] @ u[a]
                    ker = ab * bc * ca - (ab * ab + bc * bc + ca * ca) / 3.0 + 2.0 / 9.0
                    ref += g[a] * g[b] * g[c] * ker
        np.testing.assert_allclose(d[i, off:off + hp.n_angular], ref, rtol=1e-10, atol=1e-13)


def test_radial_descriptor_direct_sum():
    """D^R_n = sum_j sum_k c[ti][tj][n][k] f_k(r_ij), evaluated pair by pair."""
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(7))[0]
    model = unpack(blob, hp)
    pos, types, box = _cluster(6, seed=12)
    d = descriptors(pos, box, types, hp, blob)
    c = model.c_radial.numpy()
    rc = hp.rc_radial
    for i in range(len(pos)):
        ref = np.zeros(hp.n_radial)
        for j in range(len(pos)):
            if j == i:
                continue
            r = np.linalg.norm(pos[j] - pos[i])
            if r >= rc:
                continue
            x = 2 * (r / rc - 1) ** 2 - 1
            fc = 0.5 * (1 + math.cos(math.pi * r / rc))
            fk = np.array([0.5 * (math.cos(k * math.acos(x)) + 1) * fc for k in range(9)])
            ref += c[types[i], types[j]] @ fk
        np.testing.assert_allclose(d[i, :hp.n_radial], ref, rtol=1e-11, atol=1e-13)


def test_descriptor_rotation_permutation_translation_invariance():
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(8))[0]
    pos, types, box = _cluster(9, seed=13)
    d0 = descriptors(pos, box, types, hp, blob)
    rng = np.random.default_rng(1)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    centre = pos.mean(0)
    d_rot = descriptors((pos - centre) @ q.T + centre, box, types, hp, blob)
    np.testing.assert_allclose(d_rot, d0, rtol=1e-10, atol=1e-12)
    perm = rng.permutation(len(pos))
    d_perm = descriptors(pos[perm], box, types[perm], hp, blob)
    np.testing.assert_allclose(d_perm, d0[perm], rtol=1e-10, atol=1e-12)
    # periodic translation with wrapping (water box)
    s, hpw, pw, _ = wl.config_water_small()
    dw = descriptors(s.positions.astype(np.float64), s.box, s.types, hpw, pw)
    shifted = (s.positions.astype(np.float64) + np.array([3.1, -7.7, 5.3])) % 12.42
    np.testing.assert_allclose(descriptors(shifted, s.box, s.types, hpw, pw), dw, rtol=1e-9, atol=1e-11)


def test_descriptor_supercell_replication_small_box():
    """A 40-atom BaTiO3 cell (edge 8 A < 2 r_c) and its 2x2x2 replica give equal D per atom."""
    s = wl.batio3_supercell(2, seed=21)
    hp = wl.HParams(n_species=3)
    blob = wl.random_params(hp, np.random.default_rng(9))[0]
    d1 = descriptors(s.positions.astype(np.float64), s.box, s.types, hp, blob)
    shifts = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    big = (s.positions[None].astype(np.float64) + shifts[:, None, :] * 8.0).reshape(-1, 3)
    d2 = descriptors(big, s.box * 2, np.tile(s.types, 8), hp, blob)
    np.testing.assert_allclose(d2, np.tile(d1, (8, 1)), rtol=1e-10, atol=1e-12)


def test_image_enumeration_counts_and_kdtree():
    # one atom in a cube of edge 4 with r_c = 6: images with 0 < |T| 4 < 6 are |T|^2 in {1, 2}
    ent = geometry.neighbor_entries(np.zeros((1, 3)), np.diag([4.0] * 3), 6.0)
    assert len(ent.i) == 6 + 12
    s = wl.water_box(5, seed=4)
    ref = geometry.neighbor_entries(s.positions.astype(np.float64), s.box, 6.0)
    kd = geometry.neighbor_entries_kdtree(s.positions.astype(np.float64), s.box, 6.0)
    for a, b in ((ref.i, kd.i), (ref.j, kd.j), (ref.shift, kd.shift)):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(ref.vec, kd.vec, atol=1e-12)


def test_network_matches_explicit_loop():
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(10))[0]
    model = unpack(blob, hp)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(4, hp.n_des))
    types = np.array([0, 1, 1, 0])
    u, q = network.site_energy_and_charge(torch.as_tensor(d), types, model)
    for i in range(4):
        t = types[i]
        w0, b0 = model.w0[t].numpy(), model.b0[t].numpy()
        h = [math.tanh(sum(w0[mu, nu] * d[i, nu] for nu in range(hp.n_des)) - b0[mu])
             for mu in range(hp.n_neurons)]
        ue = sum(model.w1e[t, mu].item() * h[mu] for mu in range(hp.n_neurons)) - model.b1e[t].item()
        qe = sum(model.w1q[t, mu].item() * h[mu] for mu in range(hp.n_neurons)) - model.b1q[t].item()
        assert abs(u[i].item() - ue) < 1e-12 and abs(q[i].item() - qe) < 1e-12
