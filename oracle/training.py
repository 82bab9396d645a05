"""Fitness of a candidate population and the separable NES update (oracle, float64).

Test infrastructure only (see the package docstring).

Sec. II.E trains every parameter z (descriptor coefficients, network, sqrt(eps_inf))
with the separable natural evolution strategy (SNES, Schaul et al. 2011, cited
there) on the loss
    L(z) = l_e D_e + l_f D_f + l_v D_v + l_Z D_Z + l_Q D_Q + l_1 |z|_1 + l_2 |z|_2^2,
the D being root-mean-square errors against reference data.  The batched force
call returns energies, forces, corrected charges and virials per (candidate, structure);
the terms it can feed are D_e, D_f and D_v (its corrected charges sum to the target
exactly, and it computes no BEC), read as
    D_e = sqrt( 1/S sum_s ((E_s - E_s^ref) / N_s)^2 )        energy RMSE per atom
    D_f = sqrt( 1/(3 N) sum_i sum_b (F_ib - F_ib^ref)^2 )     force RMSE per component
    D_v = sqrt( 1/(6 S) sum_s sum_ab ((W_s,ab - W_s,ab^ref) / N_s)^2 ),  ab in xx, yy, zz, xy, yz, zx
                                                               virial RMSE per atom
over the S structures with atoms (N_s > 0) and their N atoms in all; the paper names the
RMSEs only, the normalisations are the NEP convention (per atom; the six independent
components of the virial, read from its upper triangle).

SNES, as published: a population of lambda candidates z_k = mu + sigma * s_k with
s_k ~ N(0, I) (drawn by the caller and passed in); candidates ranked by loss
(lowest first, ties by index, NaN last); rank-based utilities
    u_k = max(0, ln(lambda/2 + 1) - ln k) / sum_j max(0, ln(lambda/2 + 1) - ln j) - 1/lambda
for rank k = 1..lambda; gradients g_mu = sum_k u_k s_k, g_sigma = sum_k u_k (s_k^2 - 1);
updates mu <- mu + eta_mu sigma g_mu, sigma <- sigma exp(eta_sigma / 2 g_sigma), with the
published rates eta_mu = 1, eta_sigma = (3 + ln d) / (5 sqrt d) for d parameters.

Pins (tests/test_oracle_training.py): D_e, D_f and D_v against brute-force loops and
closed forms (a uniform per-atom energy offset d gives D_e = |d|, a uniform force
offset c gives D_f = |c|, a uniform per-atom virial offset v on every component gives
D_v = |v|, on the three off-diagonal ones D_v = |v| / sqrt(2), on the lower triangle only
0); the utilities sum to zero and decrease with rank; the update is invariant under a
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
