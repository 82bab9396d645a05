"""Fitness of a candidate population and the separable NES update (oracle, float64).

Test infrastructure only (see the package docstring).

Sec. II.E trains every parameter z (descriptor coefficients, network, sqrt(eps_inf))
with the separable natural evolution strategy (SNES, Schaul et al. 2011, cited
there) on the loss
    L(z) = l_e D_e + l_f D_f + l_v D_v + l_Z D_Z + l_Q D_Q + l_1 |z|_1 + l_2 |z|_2^2,
the D being root-mean-square errors against reference data.  The batched force
call returns energies, forces, corrected charges, virials, the total charge before the
correction and (on request) BEC per (candidate, structure); every term is fed, read as
    D_e = sqrt( 1/S sum_s ((E_s - E_s^ref) / N_s)^2 )        energy RMSE per atom
    D_f = sqrt( 1/(3 N) sum_i sum_b (F_ib - F_ib^ref)^2 )     force RMSE per component
    D_v = sqrt( 1/(6 S) sum_s sum_ab ((W_s,ab - W_s,ab^ref) / N_s)^2 ),  ab in xx, yy, zz, xy, yz, zx
                                                               virial RMSE per atom
    D_Z = sqrt( 1/(9 N_Z) sum_{s in Z} sum_{i in s} sum_ab (Z_i,ab - Z_i,ab^ref)^2 )
                                                               BEC RMSE per component
    D_Q = sqrt( 1/S sum_s (Q_s - Q_s^ref)^2 )                  total-charge RMSE per structure
over the S structures with atoms (N_s > 0) and their N atoms in all; Z is the subset of
structures that carry reference BEC (the paper makes them optional, for a subset of the
training structures) and N_Z their atoms; Q_s = sum_i q~_i = sqrt(eps_inf) sum_i q_i is the
predicted total charge BEFORE the correction of Eq. charge-scaling (after it, the sum is the
target by construction; the penalty is what keeps the uncorrected sum near the target).  The
paper names the RMSEs only; the normalisations are the NEP convention (per atom; the six
independent components of the virial, read from its upper triangle), per component for Z and
per structure for the total charge.

SNES, as published: a population of lambda candidates z_k = mu + sigma * s_k with
s_k ~ N(0, I) (drawn by the caller and passed in); candidates ranked by loss
(lowest first, ties by index, NaN last); rank-based utilities
    u_k = max(0, ln(lambda/2 + 1) - ln k) / sum_j max(0, ln(lambda/2 + 1) - ln j) - 1/lambda
for rank k = 1..lambda; gradients g_mu = sum_k u_k s_k, g_sigma = sum_k u_k (s_k^2 - 1);
updates mu <- mu + eta_mu sigma g_mu, sigma <- sigma exp(eta_sigma / 2 g_sigma), with the
published rates eta_mu = 1, eta_sigma = (3 + ln d) / (5 sqrt d) for d parameters.

Pins (tests/test_oracle_training.py): D_e, D_f, D_v, D_Z and D_Q against brute-force
loops and closed forms (a uniform per-atom energy offset d gives D_e = |d|, a uniform force
offset c gives D_f = |c|, a uniform per-atom virial offset v on every component gives
D_v = |v|, on the three off-diagonal ones D_v = |v| / sqrt(2), on the lower triangle only
0; a uniform BEC offset z on every component of the referenced structures gives D_Z = |z|,
on the diagonal only |z| / sqrt(3), on unreferenced structures 0; a total-charge offset d
gives D_Q = |d|); the utilities sum to zero and decrease with rank; the update is invariant under a
monotone transform of the losses; SNES minimises a separable quadratic from a distant start.
"""
from __future__ import annotations

import math

import numpy as np


def loss_terms(energy, forces, energy_ref, forces_ref, atom_offsets, params):
    """Per candidate: (D_e, D_f, |z|_1, |z|_2^2), arrays of shape [C].

    energy [C, S], forces [C, N, 3] (or None), energy_ref [S], forces_ref [N, 3],
    atom_offsets [S + 1], params [C, P].
    """
    off = np.asarray(atom_offsets, dtype=np.int64)
    n_s = np.diff(off)
    has = n_s > 0
    e = np.asarray(energy, dtype=np.float64)
    de = (e[:, has] - np.asarray(energy_ref, dtype=np.float64)[None, has]) / n_s[None, has]
    d_e = np.sqrt((de ** 2).mean(axis=1)) if has.any() else np.zeros(e.shape[0])
    if forces is None or off[-1] == 0:
        d_f = np.zeros(e.shape[0])
    else:
        df = np.asarray(forces, dtype=np.float64) - np.asarray(forces_ref, dtype=np.float64)[None]
        d_f = np.sqrt((df ** 2).reshape(df.shape[0], -1).mean(axis=1))
    z = np.asarray(params, dtype=np.float64)
    return d_e, d_f, np.abs(z).sum(axis=1), (z ** 2).sum(axis=1)


VIRIAL_COMPONENTS = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))


def virial_rmse(virial, virial_ref, atom_offsets):
    """D_v per candidate: virial [C, S, 3, 3], virial_ref [S, 3, 3] (eV), atom_offsets [S + 1]."""
    off = np.asarray(atom_offsets, dtype=np.int64)
    n_s = np.diff(off)
    has = n_s > 0
    w = np.asarray(virial, dtype=np.float64).reshape(-1, len(n_s), 3, 3)
    wr = np.asarray(virial_ref, dtype=np.float64).reshape(len(n_s), 3, 3)
    if not has.any():
        return np.zeros(w.shape[0])
    dv = np.stack([(w[:, has, a, b] - wr[None, has, a, b]) / n_s[None, has] for a, b in VIRIAL_COMPONENTS], -1)
    return np.sqrt((dv ** 2).reshape(w.shape[0], -1).mean(axis=1))


def loss_terms_v(energy, forces, virial, energy_ref, forces_ref, virial_ref, atom_offsets, params):
    """Per candidate: (D_e, D_f, D_v, |z|_1, |z|_2^2); virial None gives D_v = 0."""
    d_e, d_f, l1, l2 = loss_terms(energy, forces, energy_ref, forces_ref, atom_offsets, params)
    d_v = np.zeros_like(d_e) if virial is None else virial_rmse(virial, virial_ref, atom_offsets)
    return d_e, d_f, d_v, l1, l2


def loss_v(terms, lambda_e, lambda_f, lambda_v, lambda_1, lambda_2):
    """L(z) of Sec. II.E with the virial term."""
    d_e, d_f, d_v, l1, l2 = terms
    return lambda_e * d_e + lambda_f * d_f + lambda_v * d_v + lambda_1 * l1 + lambda_2 * l2


def bec_rmse(bec, bec_ref, atom_offsets, has_ref):
    """D_Z per candidate: bec [C, N, 3, 3], bec_ref [N, 3, 3] (e), has_ref [S] (structures with
    reference BEC); 0 when no referenced structure has atoms."""
    off = np.asarray(atom_offsets, dtype=np.int64)
    z = np.asarray(bec, dtype=np.float64).reshape(-1, off[-1], 9)
    zr = np.asarray(bec_ref, dtype=np.float64).reshape(off[-1], 9)
    mask = np.zeros(off[-1], dtype=bool)
    for s, h in enumerate(np.asarray(has_ref, dtype=bool)):
        if h:
            mask[off[s]:off[s + 1]] = True
    if not mask.any():
        return np.zeros(z.shape[0])
    d = z[:, mask] - zr[None, mask]
    return np.sqrt((d ** 2).reshape(z.shape[0], -1).mean(axis=1))


def total_charge_rmse(total_charge, charge_ref, atom_offsets):
    """D_Q per candidate: total_charge [C, S] (sum of q~ before the correction), charge_ref [S]."""
    off = np.asarray(atom_offsets, dtype=np.int64)
    has = np.diff(off) > 0
    q = np.asarray(total_charge, dtype=np.float64)
    if not has.any():
        return np.zeros(q.shape[0])
    d = q[:, has] - np.asarray(charge_ref, dtype=np.float64)[None, has]
    return np.sqrt((d ** 2).mean(axis=1))


def loss_terms_full(energy, forces, virial, bec, total_charge, energy_ref, forces_ref, virial_ref, bec_ref,
                    has_bec_ref, charge_ref, atom_offsets, params):
    """Per candidate: (D_e, D_f, D_v, D_Z, D_Q, |z|_1, |z|_2^2); a None output gives its term 0."""
    d_e, d_f, d_v, l1, l2 = loss_terms_v(energy, forces, virial, energy_ref, forces_ref, virial_ref, atom_offsets,
                                         params)
    d_z = np.zeros_like(d_e) if bec is None else bec_rmse(bec, bec_ref, atom_offsets, has_bec_ref)
    d_q = np.zeros_like(d_e) if total_charge is None else total_charge_rmse(total_charge, charge_ref, atom_offsets)
    return d_e, d_f, d_v, d_z, d_q, l1, l2


def loss_full(terms, lambda_e, lambda_f, lambda_v, lambda_z, lambda_q, lambda_1, lambda_2):
    """L(z) of Sec. II.E with every term."""
    d_e, d_f, d_v, d_z, d_q, l1, l2 = terms
    return (lambda_e * d_e + lambda_f * d_f + lambda_v * d_v + lambda_z * d_z + lambda_q * d_q + lambda_1 * l1
            + lambda_2 * l2)


def loss(terms, lambda_e, lambda_f, lambda_1, lambda_2):
    """L(z) of Sec. II.E restricted to the terms the batched call feeds."""
    d_e, d_f, l1, l2 = terms
    return lambda_e * d_e + lambda_f * d_f + lambda_1 * l1 + lambda_2 * l2


def ranks(fitness):
    """0-based rank of each candidate: lowest loss first, ties by index, NaN last."""
    f = np.asarray(fitness, dtype=np.float64)
    key = np.where(np.isnan(f), np.inf, f)
    nan = np.isnan(f)
    order = sorted(range(len(f)), key=lambda c: (nan[c], key[c], c))
    r = np.empty(len(f), dtype=np.int64)
    for k, c in enumerate(order):
        r[c] = k
    return r


def utilities(n):
    """u_k for ranks k = 1..n (index k - 1)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    w = np.maximum(0.0, math.log(n / 2.0 + 1.0) - np.log(k))
    return w / w.sum() - 1.0 / n


def default_rates(d):
    return 1.0, (3.0 + math.log(d)) / (5.0 * math.sqrt(d))


def update(mu, sigma, s, fitness, eta_mu=None, eta_sigma=None):
    """One SNES step: returns the new (mu, sigma) from the samples s [C, P] and their losses."""
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    c, d = s.shape
    em, es = default_rates(d)
    eta_mu = em if eta_mu is None else eta_mu
    eta_sigma = es if eta_sigma is None else eta_sigma
    u = utilities(c)[ranks(fitness)]
    g_mu = u @ s
    g_sigma = u @ (s * s - 1.0)
    return mu + eta_mu * sigma * g_mu, sigma * np.exp(0.5 * eta_sigma * g_sigma)


def sample(mu, sigma, s):
    """Candidates z_k = mu + sigma * s_k, [C, P]."""
    return np.asarray(mu, dtype=np.float64)[None] + np.asarray(sigma, dtype=np.float64)[None] * np.asarray(s)
