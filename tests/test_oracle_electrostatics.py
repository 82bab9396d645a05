"""Pins of the oracle's Ewald and PPPM electrostatics (CPU only).

Fixed references: the NaCl Madelung constant (golden file), Ewald against a
direct Coulomb sum on small neutral clusters (with the tin-foil dipole term),
the paper's own partial-force / virial formulas evaluated term by term, the
closed-form aliasing sum against brute force, B-spline identities, the PPPM
potential against finite differences in q, and PPPM converging to Ewald.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import ewald, geometry, pppm
from paper_2601_19034_gb300 import workloads as wl

KE = 14.3996454784
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_values(name):
    rows = [ln for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    return [np.array([float(x) for x in r.split()]) for r in rows]


def _ewald_energy(pos, box, q, alpha, rc, kmax):
    elec = wl.Elec(mode=1, alpha=alpha, rc_real=rc, kmax=kmax)
    ent = geometry.neighbor_entries(pos, box, rc)
    out = ewald.ewald_static(pos, box, q, ent, elec)
    return out


def test_nacl_madelung_constant():
    m_ref = _golden_values("madelung_nacl.txt")[0][0]
    a = 5.64
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos = np.concatenate([fcc, fcc + [.5, 0, 0]]) * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    box = np.diag([a] * 3)
    out = _ewald_energy(pos, box, q, alpha=0.8, rc=6.0, kmax=2 * 0.8 * math.sqrt(math.log(1e18)))
    e = out["e_real"] + out["e_kspace"] + out["e_self"]
    madelung = -e / 4 / (KE / (a / 2))
    assert abs(madelung - m_ref) < 2e-6
    # the same constant from a second (alpha, r_c) split: Ewald is alpha independent
    out2 = _ewald_energy(pos, box, q, alpha=0.6, rc=8.0, kmax=2 * 0.6 * math.sqrt(math.log(1e18)))
    e2 = out2["e_real"] + out2["e_kspace"] + out2["e_self"]
    assert abs(e2 - e) < 1e-9 * abs(e)
    assert np.abs(out["force"]).max() < 1e-9     # every ion at an inversion centre


def _direct_coulomb(pos, q):
    e = 0.0
    for i in range(len(pos)):
        for j in range(i + 1, len(pos)):
            e += KE * q[i] * q[j] / np.linalg.norm(pos[i] - pos[j])
    return e


@pytest.mark.parametrize("zero_dipole", [True, False])
def test_ewald_matches_direct_sum_on_cluster(zero_dipole):
    rng = np.random.default_rng(4)
    if zero_dipole:
        # two antiparallel dipoles: zero total charge and zero dipole
        pos = np.array([[0, 0, 0], [1.1, 0, 0], [0, 1.5, 0.3], [1.1, 1.5, 0.3]], float)
        q = np.array([0.7, -0.7, -0.7, 0.7])
    else:
        pos = rng.uniform(-1.5, 1.5, size=(5, 3))
        q = rng.normal(size=5)
        q -= q.mean()
    alpha = 0.35
    resid = []
    for length in (48.0, 96.0):
        p = pos + length / 2
        box = np.diag([length] * 3)
        out = _ewald_energy(p, box, q, alpha=alpha, rc=23.0, kmax=2 * alpha * math.sqrt(math.log(1e16)))
        e_ewald = out["e_real"] + out["e_kspace"] + out["e_self"]
        dipole = (q[:, None] * p).sum(0)
        # tin-foil (k = 0 excluded) versus spherical-shell vacuum summation: +2 pi/(3 V) k_e |M|^2
        e_shell = e_ewald + 2 * math.pi / (3 * length ** 3) * KE * dipole @ dipole
        resid.append(abs(e_shell - _direct_coulomb(p, q)))
    # what remains is the multipole interaction with the images, decaying as L^-5
    assert resid[1] < 2e-6
    assert resid[0] < 1e-6 or resid[0] / resid[1] > 20


def _paper_formulas(pos, box, q, alpha, rc, kmax):
    """Static forces, potential and virial from the paper's Sec. II.C formulas."""
    n = len(pos)
    lengths = np.diag(box)
    ent = geometry.neighbor_entries(pos, box, rc)
    f = np.zeros((n, 3))
    phi = np.zeros(n)
    vir = np.zeros((3, 3))
    for i, j, v in zip(ent.i, ent.j, ent.vec):
        r = np.linalg.norm(v)
        # F^{r,static}_ij = 1/2 (-q_i q_j k_e) r_ij / r^3 [2 alpha r / sqrt(pi) e^{-a^2 r^2} + erfc(a r)]
        fij = -0.5 * KE * q[i] * q[j] * v / r ** 3 * (
            2 * alpha * r / math.sqrt(math.pi) * math.exp(-alpha * alpha * r * r) + math.erfc(alpha * r))
        f[i] += fij      # F_i = sum_j (F_ij - F_ji) and F_ji = -F_ij for this pair term
        f[j] -= fij
        vir -= np.outer(v, fij)   # W_i = sum_j r_ij (x) F_ji
        phi[i] += KE * q[j] * math.erfc(alpha * r) / r
    phi += -2 * KE * alpha / math.sqrt(math.pi) * q
    nvec = ewald.kspace_integers(box, kmax)
    kv = 2 * math.pi * nvec / lengths
    k2 = (kv ** 2).sum(1)
    g = 2 * math.pi / np.prod(lengths) * np.exp(-k2 / (4 * alpha ** 2)) / k2
    s = (q[:, None] * np.exp(-1j * pos @ kv.T)).sum(0)
    e_ikr = np.exp(1j * pos @ kv.T)
    f += 2 * KE * q[:, None] * ((g * (s[None, :] * e_ikr).imag) @ kv)
    phi += 2 * KE * ((g * (s[None, :] * e_ikr).real).sum(1))
    bfac = 2 / (4 * alpha ** 2) + 2 / k2
    for a in range(3):
        for b in range(3):
            bab = (a == b) - bfac * kv[:, a] * kv[:, b]
            vir[a, b] += KE * (g * np.abs(s) ** 2 * bab).sum()
    return f, phi, vir


def test_ewald_autograd_matches_paper_formulas():
    s = wl.water_box(2, length=6.5, seed=7)
    pos = s.positions.astype(np.float64)
    rng = np.random.default_rng(3)
    q = rng.normal(0, 0.4, size=len(pos))
    q -= q.mean()
    alpha, rc, kmax = 0.45, 5.0, 2.5
    out = _ewald_energy(pos, s.box, q, alpha, rc, kmax)
    f, phi, vir = _paper_formulas(pos, s.box, q, alpha, rc, kmax)
    np.testing.assert_allclose(out["force"], f, atol=1e-10)
    np.testing.assert_allclose(out["phi"], phi, atol=1e-10)
    np.testing.assert_allclose(out["virial"], vir, atol=1e-9)
    assert np.abs(out["force"].sum(0)).max() < 1e-10


def test_ewald_kmax_relative_error_budget():
    """k_max = 2 alpha sqrt(ln 1e6) truncates U^k at about 1e-6 relative."""
    sysm, hp, blob, elec = wl.config_water_small()
    pos = sysm.positions.astype(np.float64)
    q = np.random.default_rng(0).normal(0, 0.4, size=len(pos))
    q -= q.mean()
    ent = geometry.neighbor_entries(pos, sysm.box, 6.0)
    e1 = ewald.ewald_static(pos, sysm.box, q, ent, elec)["e_kspace"]
    big = wl.Elec(mode=1, kmax=1.5 * elec.kmax)
    e2 = ewald.ewald_static(pos, sysm.box, q, ent, big)["e_kspace"]
    assert abs(e1 - e2) <= 1e-6 * abs(e2)


def test_alias_sum_closed_form_and_sign():
    coef, at_half = _golden_values("alias_sum_p5.txt")
    x = np.linspace(-0.5, 0.5, 41)
    z2 = np.sin(np.pi * x) ** 2
    closed = sum(c * z2 ** k for k, c in enumerate(coef))
    brute = pppm.alias_sum(x * 64, 64, 5, terms=400)
    np.testing.assert_allclose(closed, brute, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(pppm.alias_sum(x * 64, 64, 5), brute, rtol=1e-9, atol=1e-12)
    assert abs(pppm.alias_sum(np.array([32.0]), 64, 5)[0] - at_half[0]) < 1e-5
    printed = 1 - 5 / 3 + 7 / 9 + 17 / 189 + 2 / 2835
    assert abs(printed - at_half[0]) > 0.1


def test_bspline_identities():
    u = np.random.default_rng(0).uniform(-20, 20, size=500)
    for order in range(1, 8):
        _, w = pppm.stencil(u, order)
        np.testing.assert_allclose(w.sum(-1), 1.0, atol=1e-13)          # partition of unity
        if order == 1:
            continue      # the box has jumps; the trapezoid rule is only first order there
        xs = np.linspace(-order / 2, order / 2, 20001)
        for kk in (0.3, 1.1, 2.5):
            ft = np.trapezoid(pppm.bspline(order, xs) * np.cos(kk * xs), xs)
            assert abs(ft - np.sinc(kk / (2 * np.pi)) ** order) < 1e-6   # FT = sinc^P(k/2)
    # M_2 is the hat function
    xs = np.linspace(-1.5, 1.5, 31)
    np.testing.assert_allclose(pppm.bspline(2, xs), np.clip(1 - np.abs(xs), 0, None), atol=1e-14)


def _water_q(n_side=3, seed=9):
    s = wl.water_box(n_side, seed=seed)
    rng = np.random.default_rng(seed)
    q = np.tile([0.8, -0.4, -0.4], len(s.positions) // 3) + rng.normal(0, 0.05, len(s.positions))
    q -= q.mean()
    return s, q


def test_pppm_energy_identity_and_potential_is_gradient():
    s, q = _water_q()
    pos = s.positions.astype(np.float64)
    out = pppm.pppm(pos, s.box, q, (24, 24, 24), 5, 0.3)
    assert abs(out["e_kspace"] - 0.5 * (q * out["phi"]).sum()) < 1e-10 * abs(out["e_kspace"])
    h = 1e-5
    for i in (0, 5, 17):
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (pppm.pppm(pos, s.box, qp, (24,) * 3, 5, 0.3)["e_kspace"]
              - pppm.pppm(pos, s.box, qm, (24,) * 3, 5, 0.3)["e_kspace"]) / (2 * h)
        assert abs(fd - out["phi"][i]) < 1e-6


def test_pppm_converges_to_ewald():
    """Mesh spacing < 1 A with P = 5 gives ~1e-4 relative accuracy (Sec. II.F)."""
    s, q = _water_q(4, seed=2)
    pos = s.positions.astype(np.float64)
    alpha = 0.3
    ent = geometry.neighbor_entries(pos, s.box, 6.0)
    ref = ewald.ewald_static(pos, s.box, q, ent,
                             wl.Elec(mode=1, alpha=alpha, kmax=2 * alpha * math.sqrt(math.log(1e14))))
    length = s.box[0, 0]
    mesh = int(math.ceil(length / 0.9))
    mesh += mesh % 2
    out = pppm.pppm(pos, s.box, q, (mesh,) * 3, 5, alpha)
    fnorm = np.sqrt((ref["force"] ** 2).sum(1).mean())
    k_force_ref = ref["force"] - ewald.ewald_static(pos, s.box, q, ent, wl.Elec(mode=1, alpha=alpha),
                                                    with_kspace=False)["force"]
    err = np.sqrt(((out["force"] - k_force_ref) ** 2).sum(1).mean())
    assert err / fnorm < 3e-4
    assert abs(out["e_kspace"] - ref["e_kspace"]) < 1e-4 * abs(ref["e_real"] + ref["e_kspace"])
    printed = pppm.pppm(pos, s.box, q, (mesh,) * 3, 5, alpha, printed_form=True)
    err_printed = np.sqrt(((printed["force"] - k_force_ref) ** 2).sum(1).mean())
    assert err_printed > 2 * err      # the squared alias denominator is the accurate reading
    np.testing.assert_allclose(out["virial"], ref["virial"] - ewald.ewald_static(
        pos, s.box, q, ent, wl.Elec(mode=1, alpha=alpha), with_kspace=False)["virial"],
        atol=2e-3 * np.abs(ref["virial"]).max())


def test_coulomb_constant_from_the_si_definitions():
    """k_e = e^2 / (4 pi eps_0) in eV A per e^2 follows from e = 1.602176634e-19 C (exact) and
    eps_0 = 8.8541878128e-12 F/m (CODATA 2018): k_e [eV A] = e / (4 pi eps_0) [V m] x 1e10.  The
    oracle's constant, and the CUDA path's own literals (written separately: FP64 to 1e-11, FP32 to
    its rounding), are that value.  The Madelung pin above divides by k_e and cannot see it."""
    import re
    ke = 1.602176634e-19 / (4.0 * math.pi * 8.8541878128e-12) * 1e10
    assert ewald.KE == pytest.approx(ke, rel=1e-11)
    assert pppm.KE == pytest.approx(ke, rel=1e-11)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2601_19034_gb300", "csrc")
    internal = open(os.path.join(csrc, "qnep_internal.cuh")).read()
    assert float(re.search(r"constexpr double KE_D = ([0-9.]+);", internal).group(1)) == pytest.approx(ke, rel=1e-11)
    assert float(re.search(r"constexpr float KE = ([0-9.]+)f;", internal).group(1)) == pytest.approx(ke, rel=6e-8)
    batch = open(os.path.join(csrc, "api_batch.cu")).read()
    assert float(re.search(r"\bke = ([0-9.]+);", batch).group(1)) == pytest.approx(ke, rel=1e-11)
