"""Unpacking of the documented qNEP parameter blob (oracle side, float64).

Layout of one candidate (all float32 in the blob), S species, n_des descriptor
components, N_neu hidden units:
  c_R[ti][tj][n][k]   S*S*n_radial*basis_radial   radial expansion coefficients
  c_A[ti][tj][n][k]   S*S*n_angular*basis_angular angular expansion coefficients
  scaler[nu]          n_des                       descriptor scaling
  per species t:      W0[mu][nu] (N_neu*n_des), b0[mu], w1E[mu], w1q[mu], b1E, b1q
  sqrt_eps_inf        1                           sqrt of the high-frequency permittivity
The trainable parameters are those of Sec. II.A (Eq. U_i), the charge node of
Sec. II.B and eps_inf of Sec. II.D; the per-species network (NEP4, Sec. II.A)
is indexed by the species of the central atom.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch


@dataclasses.dataclass
class Model:
    c_radial: torch.Tensor   # [S, S, n_radial, basis_radial]
    c_angular: torch.Tensor  # [S, S, n_angular, basis_angular]
    scaler: torch.Tensor     # [n_des]
    w0: torch.Tensor         # [S, N_neu, n_des]
    b0: torch.Tensor         # [S, N_neu]
    w1e: torch.Tensor        # [S, N_neu]
    w1q: torch.Tensor        # [S, N_neu]
    b1e: torch.Tensor        # [S]
    b1q: torch.Tensor        # [S]
    sqrt_eps_inf: float
    rc_radial: float
    rc_angular: float
    l_max: int
    use_4body: bool


def unpack(blob: np.ndarray, hp) -> Model:
    p = torch.as_tensor(np.asarray(blob, dtype=np.float32).astype(np.float64))
    s, nr, kr, na, ka = hp.n_species, hp.n_radial, hp.basis_radial, hp.n_angular, hp.basis_angular
    nd, nn = hp.n_des, hp.n_neurons
    o = 0

    def take(count):
        nonlocal o
        out = p[o:o + count]
        o += count
        return out

    c_r = take(s * s * nr * kr).reshape(s, s, nr, kr)
    c_a = take(s * s * na * ka).reshape(s, s, na, ka)
    scaler = take(nd)
    w0, b0, w1e, w1q, b1e, b1q = [], [], [], [], [], []
    for _ in range(s):
        w0.append(take(nn * nd).reshape(nn, nd))
        b0.append(take(nn))
        w1e.append(take(nn))
        w1q.append(take(nn))
        b1e.append(take(1))
        b1q.append(take(1))
    sqrt_eps = float(take(1)[0])
    assert o == p.numel(), (o, p.numel())
    return Model(c_r, c_a, scaler, torch.stack(w0), torch.stack(b0), torch.stack(w1e),
                 torch.stack(w1q), torch.cat(b1e), torch.cat(b1q), sqrt_eps,
                 float(hp.rc_radial), float(hp.rc_angular), int(hp.l_max), bool(hp.use_4body))
