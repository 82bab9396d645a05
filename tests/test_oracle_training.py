"""Pins of the oracle's population loss and SNES update (Sec. II.E; SNES of Schaul et al. 2011).

D_e and D_f against brute-force loops over structures and atoms and against
closed forms; the utilities' zero sum and ordering; rank invariance of the
update; and SNES converging on a separable quadratic (a sign error in either
gradient, or in the utilities, stops it converging).
"""
import math

import numpy as np

from oracle import training as tr


def _case(seed=0, c=5, sizes=(3, 0, 7, 1)):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)])
    n, s = off[-1], len(sizes)
    e = rng.normal(size=(c, s)) * 10
    e_ref = rng.normal(size=s) * 10
    f = rng.normal(size=(c, n, 3))
    f_ref = rng.normal(size=(n, 3))
    z = rng.normal(size=(c, 11))
    return e, f, e_ref, f_ref, off, z


def test_loss_terms_match_brute_force():
    e, f, e_ref, f_ref, off, z = _case()
    d_e, d_f, l1, l2 = tr.loss_terms(e, f, e_ref, f_ref, off, z)
    for c in range(e.shape[0]):
        acc, cnt = 0.0, 0
        for s in range(len(off) - 1):
            n_s = off[s + 1] - off[s]
            if n_s == 0:
                continue
            acc += ((e[c, s] - e_ref[s]) / n_s) ** 2
            cnt += 1
        assert abs(d_e[c] - math.sqrt(acc / cnt)) < 1e-12
        acc = 0.0
        for i in range(off[-1]):
            for b in range(3):
                acc += (f[c, i, b] - f_ref[i, b]) ** 2
        assert abs(d_f[c] - math.sqrt(acc / (3 * off[-1]))) < 1e-12
        assert abs(l1[c] - sum(abs(x) for x in z[c])) < 1e-12
        assert abs(l2[c] - sum(x * x for x in z[c])) < 1e-12


def test_loss_closed_forms():
    e, f, e_ref, f_ref, off, z = _case(seed=1)
    n_s = np.diff(off)
    delta = np.array([0.3, -0.02, 0.0, 1.5, -0.7])
    e_shift = e_ref[None, :] + delta[:, None] * n_s[None, :]
    c_f = np.array([0.1, -0.25, 0.0, 2.0, 0.04])
    f_shift = f_ref[None] + c_f[:, None, None]
    d_e, d_f, _, _ = tr.loss_terms(e_shift, f_shift, e_ref, f_ref, off, z)
    np.testing.assert_allclose(d_e, np.abs(delta), atol=1e-12)
    np.testing.assert_allclose(d_f, np.abs(c_f), atol=1e-12)
    terms = tr.loss_terms(e_ref[None].repeat(5, 0), f_ref[None].repeat(5, 0), e_ref, f_ref, off, z)
    np.testing.assert_allclose(tr.loss(terms, 1.0, 1.0, 0.05, 0.01),
                               0.05 * np.abs(z).sum(1) + 0.01 * (z ** 2).sum(1), atol=1e-12)


def test_utilities_and_ranks():
    for n in (2, 3, 4, 7, 64, 100):
        u = tr.utilities(n)
        assert abs(u.sum()) < 1e-12
        assert np.all(np.diff(u) <= 1e-15)
        top = (n + 1) // 2                    # ranks k < n/2 + 1 have a positive raw weight
        assert np.all(u[:top] > -1.0 / n) and np.allclose(u[top:], -1.0 / n)
    f = np.array([3.0, np.nan, 1.0, 1.0, -2.0])
    np.testing.assert_array_equal(tr.ranks(f), [3, 4, 1, 2, 0])


def test_update_is_rank_invariant():
    rng = np.random.default_rng(5)
    mu, sigma = rng.normal(size=9), np.abs(rng.normal(size=9)) + 0.1
    s = rng.normal(size=(12, 9))
    f = rng.normal(size=12)
    a = tr.update(mu, sigma, s, f)
    b = tr.update(mu, sigma, s, np.exp(3 * f) + 7.0)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=0)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=0)


def test_snes_minimises_separable_quadratic():
    rng = np.random.default_rng(6)
    d, lam = 10, 10
    a = rng.uniform(0.5, 3.0, size=d)
    target = rng.normal(size=d) * 2
    mu, sigma = np.zeros(d) + 5.0, np.ones(d)
    for _ in range(400):
        s = rng.normal(size=(lam, d))
        z = tr.sample(mu, sigma, s)
        f = ((z - target) ** 2 * a).sum(1)
        mu, sigma = tr.update(mu, sigma, s, f)
    assert np.abs(mu - target).max() < 1e-3
    assert sigma.max() < 1e-3


def _virial_case(seed=3, c=4, sizes=(5, 0, 2, 9)):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)])
    w = rng.normal(size=(c, len(sizes), 3, 3)) * 20
    w_ref = rng.normal(size=(len(sizes), 3, 3)) * 20
    return w, w_ref, off


def test_virial_rmse_matches_brute_force():
    w, w_ref, off = _virial_case()
    d_v = tr.virial_rmse(w, w_ref, off)
    for c in range(w.shape[0]):
        acc, cnt = 0.0, 0
        for s in range(len(off) - 1):
            n_s = off[s + 1] - off[s]
            if n_s == 0:
                continue
            for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)):
                acc += ((w[c, s, a, b] - w_ref[s, a, b]) / n_s) ** 2
                cnt += 1
        assert abs(d_v[c] - math.sqrt(acc / cnt)) < 1e-12


def test_virial_rmse_closed_forms():
    """Per-atom offsets: all components -> |v|; the three off-diagonal (upper) ones -> |v|/sqrt(2);
    the lower triangle only (not one of the six read) -> 0."""
    _, w_ref, off = _virial_case(seed=4)
    n_s = np.diff(off).astype(np.float64)
    v = np.array([0.2, -1.3, 0.0, 0.05])
    all_c = w_ref[None] + v[:, None, None, None] * n_s[None, :, None, None]
    np.testing.assert_allclose(tr.virial_rmse(all_c, w_ref, off), np.abs(v), atol=1e-12)
    upper = np.zeros((3, 3))
    upper[0, 1] = upper[1, 2] = upper[0, 2] = 1.0
    off_c = w_ref[None] + v[:, None, None, None] * n_s[None, :, None, None] * upper
    np.testing.assert_allclose(tr.virial_rmse(off_c, w_ref, off), np.abs(v) / math.sqrt(2.0), atol=1e-12)
    low_c = w_ref[None] + v[:, None, None, None] * n_s[None, :, None, None] * upper.T
    np.testing.assert_allclose(tr.virial_rmse(low_c, w_ref, off), 0.0, atol=1e-12)
    e, f, e_ref, f_ref, off2, z = _case(seed=2, c=4)
    terms = tr.loss_terms_v(e_ref[None].repeat(4, 0), f_ref[None].repeat(4, 0), None, e_ref, f_ref, None, off2, z)
    np.testing.assert_allclose(terms[2], 0.0)
    np.testing.assert_allclose(tr.loss_v(terms, 1.0, 1.0, 0.3, 0.05, 0.01),
                               0.05 * np.abs(z).sum(1) + 0.01 * (z ** 2).sum(1), atol=1e-12)


def _bec_case(seed=7, c=3, sizes=(4, 0, 6, 2), has=(True, True, False, True)):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)])
    z = rng.normal(size=(c, off[-1], 3, 3))
    z_ref = rng.normal(size=(off[-1], 3, 3))
    return z, z_ref, off, np.asarray(has)


def test_bec_rmse_matches_brute_force():
    z, z_ref, off, has = _bec_case()
    d_z = tr.bec_rmse(z, z_ref, off, has)
    for c in range(z.shape[0]):
        acc, cnt = 0.0, 0
        for s in range(len(off) - 1):
            if not has[s]:
                continue
            for i in range(off[s], off[s + 1]):
                for a in range(3):
                    for b in range(3):
                        acc += (z[c, i, a, b] - z_ref[i, a, b]) ** 2
                        cnt += 1
        assert abs(d_z[c] - math.sqrt(acc / cnt)) < 1e-12
    np.testing.assert_allclose(tr.bec_rmse(z, z_ref, off, np.zeros(4, bool)), 0.0)


def test_bec_rmse_closed_forms():
    """A uniform offset on every component of the referenced structures gives its size; on the
    diagonal only, its size / sqrt(3); on the structures without reference, 0."""
    _, z_ref, off, has = _bec_case(seed=8)
    d = np.array([0.4, -0.03, 1.7])
    mask = np.zeros(off[-1], bool)
    for s in range(len(has)):
        mask[off[s]:off[s + 1]] = has[s]
    every = z_ref[None] + d[:, None, None, None] * mask[None, :, None, None]
    np.testing.assert_allclose(tr.bec_rmse(every, z_ref, off, has), np.abs(d), atol=1e-12)
    diag = z_ref[None] + d[:, None, None, None] * mask[None, :, None, None] * np.eye(3)
    np.testing.assert_allclose(tr.bec_rmse(diag, z_ref, off, has), np.abs(d) / math.sqrt(3.0), atol=1e-12)
    other = z_ref[None] + d[:, None, None, None] * (~mask)[None, :, None, None]
    np.testing.assert_allclose(tr.bec_rmse(other, z_ref, off, has), 0.0, atol=1e-12)


def test_total_charge_rmse_brute_force_and_offset():
    rng = np.random.default_rng(9)
    off = np.array([0, 3, 3, 8, 9])
    q = rng.normal(size=(4, 4))
    q_ref = rng.normal(size=4)
    d_q = tr.total_charge_rmse(q, q_ref, off)
    for c in range(4):
        acc = [(q[c, s] - q_ref[s]) ** 2 for s in range(4) if off[s + 1] > off[s]]
        assert abs(d_q[c] - math.sqrt(sum(acc) / len(acc))) < 1e-12
    d = np.array([0.25, -0.5, 0.0, 3.0])
    np.testing.assert_allclose(tr.total_charge_rmse(q_ref[None] + d[:, None], q_ref, off), np.abs(d), atol=1e-12)
    # the full loss: every term zero at the reference leaves the norms, each weight on its own term
    e, f, e_ref, f_ref, off2, z = _case(seed=10, c=4)
    n = off2[-1]
    terms = tr.loss_terms_full(e_ref[None].repeat(4, 0), f_ref[None].repeat(4, 0), None,
                               np.zeros((4, n, 3, 3)) + d[:, None, None, None], np.zeros((4, 4)) + d[:, None],
                               e_ref, f_ref, None, np.zeros((n, 3, 3)), np.ones(4, bool), np.zeros(4), off2, z)
    np.testing.assert_allclose(terms[3], np.abs(d), atol=1e-12)
    np.testing.assert_allclose(terms[4], np.abs(d), atol=1e-12)
    np.testing.assert_allclose(tr.loss_full(terms, 1.0, 1.0, 1.0, 0.7, 0.2, 0.05, 0.01),
                               0.9 * np.abs(d) + 0.05 * np.abs(z).sum(1) + 0.01 * (z ** 2).sum(1), atol=1e-12)


def test_force_call_total_charge_before_the_correction():
    """With the charge output weights zero every raw charge is -b1q of its species (the bias is
    subtracted, Eq. U_i's convention for the charge node), so the predicted total charge is
    -sqrt(eps_inf) sum_i b1q[t_i], whatever the positions and the target Q; the corrected
    charges still sum to Q / sqrt(eps_inf)."""
    from oracle import forcecall
    from paper_2601_19034_gb300 import workloads as wl
    sysm = wl.water_box(2, seed=3)
    hp = wl.HParams(n_species=2)
    blob = wl.random_params(hp, np.random.default_rng(4))[0].astype(np.float32)
    s, nn, nd = hp.n_species, hp.n_neurons, hp.n_des
    o = s * s * (hp.n_radial * hp.basis_radial + hp.n_angular * hp.basis_angular) + nd
    b1q = []
    for _ in range(s):
        o += nn * nd + nn + nn          # W0, b0, w1E
        blob[o:o + nn] = 0.0            # w1q
        o += nn
        b1q.append(float(blob[o + 1]))  # b1E, b1q
        o += 2
    seps = float(blob[-1])
    expect = -seps * sum(b1q[t] for t in sysm.types)
    for q_total in (0.0, 0.6):
        out = forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, blob,
                                   wl.Elec(mode=1, kind="ewald", q_total=q_total), want_bec=False)
        assert abs(out["total_charge_raw"] - expect) < 1e-9 * max(1.0, abs(expect))
        assert abs(out["charges"].sum() - q_total / seps) < 1e-9
