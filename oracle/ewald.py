"""Ewald electrostatics of the partial charges (oracle, float64 torch).

Energies as written in Sec. II.B:
  U^r = 1/2 k_e sum_i sum_{j != i} q_i q_j erfc(alpha r_ij) / r_ij     (r_ij < r_c, every image)
  U^k = k_e sum_{k != 0, |k| < k_max} G(k) |S(k)|^2                     Eq. (U_k), full k sphere
  S(k) = sum_i q_i exp(-i k.r_i)                                        Eq. (S_k)
  G(k) = (2 pi / Omega) exp(-k^2 / 4 alpha^2) / k^2
  U^s = -k_e alpha / sqrt(pi) sum_i q_i^2
Mode 1 uses U^r + U^k + U^s (Eq. U_ES), mode 2 uses U^k only (Eq. mode2).
k_e = 1/(4 pi eps_0) = 14.3996454784 eV A / e^2.

Derivatives (the potential phi_i = dU/dq_i, the static forces and the static
virial) are autograd gradients of these energies.  The virial is
W = -(dU/d eps)^T for the homogeneous deformation r -> (I + eps) r applied to
positions and cell together, the convention of the per-atom virial of Sec. II.C.
"""
from __future__ import annotations

import math

import numpy as np
import torch

KE = 14.3996454784


def kspace_integers(box: np.ndarray, kmax: float) -> np.ndarray:
    """Integer triples n with 0 < |k| < kmax, k = 2 pi n . inv(box)^T (full sphere).

    |n_d| <= kmax |a_d| / (2 pi) because k . a_d = 2 pi n_d.
    """
    box = np.asarray(box, dtype=np.float64)
    if box.ndim == 1:
        box = np.diag(box)
    nmax = [int(math.floor(kmax * np.linalg.norm(box[d]) / (2.0 * math.pi))) for d in range(3)]
    grids = np.meshgrid(*[np.arange(-m, m + 1) for m in nmax], indexing="ij")
    n = np.stack([g.ravel() for g in grids], 1)
    k = 2.0 * math.pi * n @ np.linalg.inv(box).T
    k2 = np.einsum("kd,kd->k", k, k)
    keep = (k2 > 0) & (k2 < kmax * kmax)
    return n[keep]


def real_space_energy(vec: torch.Tensor, i, j, q: torch.Tensor, alpha: float) -> torch.Tensor:
    r = torch.linalg.norm(vec, dim=1)
    ii = torch.as_tensor(i)
    jj = torch.as_tensor(j)
    return 0.5 * KE * (q[ii] * q[jj] * torch.special.erfc(alpha * r) / r).sum()


def reciprocal_energy(pos: torch.Tensor, box: torch.Tensor, q: torch.Tensor, alpha: float,
                      nvec: np.ndarray) -> torch.Tensor:
    inv = torch.linalg.inv(box)
    kv = 2.0 * math.pi * torch.as_tensor(nvec, dtype=torch.float64) @ inv.T
    k2 = (kv * kv).sum(1)
    omega = torch.abs(torch.linalg.det(box))
    g = (2.0 * math.pi / omega) * torch.exp(-k2 / (4.0 * alpha * alpha)) / k2
    phase = pos @ kv.T
    s_re = (q[:, None] * torch.cos(phase)).sum(0)
    s_im = -(q[:, None] * torch.sin(phase)).sum(0)
    return KE * (g * (s_re * s_re + s_im * s_im)).sum()


def self_energy(q: torch.Tensor, alpha: float) -> torch.Tensor:
    return -KE * alpha / math.sqrt(math.pi) * (q * q).sum()


def ewald_static(pos_np: np.ndarray, box_np: np.ndarray, q_np: np.ndarray, ent_real, elec,
                 k_chunk: int = 1024, with_kspace: bool = True) -> dict:
    """Ewald energy parts with phi = dU/dq, static forces and static virial.

    ``with_kspace=False`` leaves out U^k (the PPPM path adds its own).
    """
    pos = torch.tensor(np.asarray(pos_np, np.float64), requires_grad=True)
    eps = torch.zeros(3, 3, dtype=torch.float64, requires_grad=True)
    q = torch.tensor(np.asarray(q_np, np.float64), requires_grad=True)
    box = torch.as_tensor(np.asarray(box_np, np.float64))

    def strained():
        defm = torch.eye(3, dtype=torch.float64) + eps
        return pos @ defm.T, box @ defm.T

    out = {"e_real": 0.0, "e_self": 0.0, "e_kspace": 0.0}
    if elec.mode == 1:
        pos_s, box_s = strained()
        shift = torch.as_tensor(ent_real.shift, dtype=torch.float64)
        vec = pos_s[ent_real.j] + shift @ box_s - pos_s[ent_real.i]
        u_r = real_space_energy(vec, ent_real.i, ent_real.j, q, elec.alpha)
        u_s = self_energy(q, elec.alpha)
        (u_r + u_s).backward()
        out["e_real"] = float(u_r.detach())
        out["e_self"] = float(u_s.detach())
    nvec = kspace_integers(box_np, elec.kmax) if with_kspace else np.zeros((0, 3), np.int64)
    for c0 in range(0, len(nvec), k_chunk):
        pos_s, box_s = strained()
        u_k = reciprocal_energy(pos_s, box_s, q, elec.alpha, nvec[c0:c0 + k_chunk])
        u_k.backward()
        out["e_kspace"] += float(u_k.detach())
    out["phi"] = q.grad.numpy().copy() if q.grad is not None else np.zeros(len(q_np))
    out["force"] = -pos.grad.numpy().copy() if pos.grad is not None else np.zeros_like(pos_np)
    out["virial"] = -eps.grad.numpy().T.copy() if eps.grad is not None else np.zeros((3, 3))
    out["n_kvec_full"] = len(nvec)
    return out
