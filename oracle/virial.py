"""Per-atom virial of the force call (oracle, float64).

Test infrastructure only (see the package docstring).

Sec. II.C writes the forces of the many-body potential with partial forces,
F_i = sum_j (F_ij - F_ji), and the per-atom virial as Eq. (per-atom_virial),
    W_i = sum_{j != i} r_ij (x) F_ji,      r_ij = r_j - r_i,
for the NEP term and every dynamic-charge term (real space, reciprocal space and
self energy all reach the positions through q_i(D^i), so their partial forces are
dE/dr_ij through the adjoint of the charge).  The static real-space term is a pair
term whose partial force is the gradient of half the pair energy.  The static
reciprocal-space term has no partial force; Sec. II.C gives it per atom (Heyes),
    W_i^k = k_e sum_{k != 0} G(k) Re[q_i e^{i k.r_i} S(k)] B(k),
    B(k) = I - (2/(4 alpha^2) + 2/k^2) k k^T,
read with the real part (the printed form has no Re; summed over i the imaginary
parts cancel and the sum is Eq. virial-kspace-total).
For PPPM (Sec. II.F) the same per-atom form is taken on the mesh: six more inverse
FFTs give F^-1[G_opt B_ab S] and W_i,ab = k_e q_i sum_s W(r_i - r_s) F^-1[G_opt B_ab S](r_s),
which sums over i to the mesh virial k_e sum_k G_opt |S|^2 B.

Here the many-body partial forces are the per-entry gradients of the staged
force call (``forcecall.force_call``), the static real-space partial forces the
autograd gradients of the per-entry half pair energies, and the reciprocal terms
the formulas above.  Convention: an entry (i -> j) with vector r_ij and partial
force F_ij adds r_ji (x) F_ij = -r_ij (x) F_ij to W_j.

Pins (tests/test_oracle_virial.py): sum_i W_i equals the force call's total virial
(itself pinned by finite differences of the energy under strain) for Ewald in
modes 1 and 2 and for PPPM; W_i is unchanged by a uniform translation; the per-atom
virials of a 2 x 2 x 2 replica equal those of the cell; and, for a cluster with the
NEP term alone, the time derivative of the energy moment sum_i r_i U_i along any
velocities equals sum_i v_i U_i - sum_i r_i (F_i . v_i) + sum_i W_i v_i, an identity
that fixes the assignment of the many-body terms (giving them to the central atom
instead fails it).  The split of the static reciprocal-space term among the atoms
(the Heyes form) is pinned only by its sum and the invariances.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import ewald, forcecall, geometry, pppm

KE = ewald.KE


def _entry_term(w, ent, g):
    """Add -r_ij (x) F_ij of every entry (i -> j) to W_j."""
    if len(ent.i):
        np.add.at(w, ent.j, -np.einsum("ea,eb->eab", ent.vec, g))


def real_space_static(pos, box, q, alpha, rc):
    """Per-atom static real-space virial [N, 3, 3] from the per-entry half pair energies."""
    n = len(pos)
    w = np.zeros((n, 3, 3))
    ent = geometry.find_entries(np.asarray(pos, np.float64), box, rc)
    if not len(ent.i):
        return w
    vec = torch.tensor(ent.vec, requires_grad=True)
    u = ewald.real_space_energy(vec, ent.i, ent.j, torch.as_tensor(np.asarray(q, np.float64)), alpha)
    g = torch.autograd.grad(u, vec)[0].numpy()
    _entry_term(w, ent, g)
    return w


def kspace_static_ewald(pos, box, q, alpha, kmax, chunk: int = 2048):
    """Per-atom static reciprocal-space virial (Heyes form, full k sphere) [N, 3, 3]."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    box = np.asarray(box, np.float64)
    nvec = ewald.kspace_integers(box, kmax)
    omega = abs(np.linalg.det(box))
    w = np.zeros((len(pos), 3, 3))
    for c0 in range(0, len(nvec), chunk):
        kv = 2.0 * math.pi * nvec[c0:c0 + chunk] @ np.linalg.inv(box).T
        k2 = np.einsum("kd,kd->k", kv, kv)
        g = (2.0 * math.pi / omega) * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
        th = pos @ kv.T                                            # [N, K]
        s_re = (q[:, None] * np.cos(th)).sum(0)                    # S(k) = sum_j q_j e^{-i k.r_j}
        s_im = -(q[:, None] * np.sin(th)).sum(0)
        re = q[:, None] * (np.cos(th) * s_re[None] - np.sin(th) * s_im[None])   # Re[q_i e^{i k.r_i} S]
        fac = 2.0 / (4.0 * alpha * alpha) + 2.0 / k2
        bmat = np.eye(3)[None] - fac[:, None, None] * np.einsum("ka,kb->kab", kv, kv)
        w += KE * np.einsum("ik,k,kab->iab", re, g, bmat)
    return w


def kspace_static_pppm(pos, box, q, mesh, order, alpha, chunk: int = 65536):
    """Per-atom static mesh virial [N, 3, 3] from the six inverse FFTs of G_opt B_ab S (a general
    cell: the fractional mesh and k = 2 pi H^-1 n of the PPPM module)."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    box = np.asarray(box, np.float64)
    general = bool(np.count_nonzero(box - np.diag(np.diag(box))))
    hinv = np.linalg.inv(box) if general else None
    lengths = np.linalg.norm(box, axis=1) if general else np.diag(box).copy()
    mesh = tuple(int(m) for m in mesh)
    ntot = int(np.prod(mesh))
    rho = np.zeros(ntot)
    for a0 in range(0, len(pos), chunk):
        pts, wt_ = pppm._gather_weights(pos[a0:a0 + chunk], lengths, mesh, order, hinv)
        flat, wt = pppm._flat_stencil(pts, wt_, mesh)
        np.add.at(rho, flat.ravel(), (wt * q[a0:a0 + chunk, None]).ravel())
    s = np.fft.fftn(rho.reshape(mesh))
    gopt, k, k2 = pppm.influence(lengths, mesh, order, alpha, box=box if general else None)[:3]
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(k2 > 0, 2.0 / (4 * alpha * alpha) + 2.0 / k2, 0.0)
    w = np.zeros((len(pos), 3, 3))
    for a in range(3):
        for b in range(a, 3):
            bab = (1.0 if a == b else 0.0) - fac * k[a] * k[b]
            field = (np.fft.ifftn(gopt * bab * s) * ntot).real.ravel()
            for a0 in range(0, len(pos), chunk):
                pts, wt_ = pppm._gather_weights(pos[a0:a0 + chunk], lengths, mesh, order, hinv)
                flat, wt = pppm._flat_stencil(pts, wt_, mesh)
                val = KE * q[a0:a0 + chunk] * (wt * field[flat]).sum(1)
                w[a0:a0 + chunk, a, b] = val
                w[a0:a0 + chunk, b, a] = val
    return w


def per_atom_virial(positions, box, types, hp, blob, elec) -> tuple[np.ndarray, dict]:
    """W_i [N, 3, 3] of Eq. (per-atom_virial) and the force call's outputs.

    Sum over the atoms = the force call's total virial.
    """
    pos = np.asarray(positions, np.float64)
    out = forcecall.force_call(pos, box, types, hp, blob, elec, want_bec=False)
    w = np.zeros((len(pos), 3, 3))
    for ent, g in out["partials"]:
        _entry_term(w, ent, g)
    q = out["charges"]                         # the corrected screened charges the energy uses
    if elec.mode == 1:
        w += real_space_static(pos, box, q, elec.alpha, elec.rc_real)
    if elec.kind == "ewald":
        w += kspace_static_ewald(pos, box, q, elec.alpha, elec.kmax)
    else:
        w += kspace_static_pppm(pos, box, q, elec.mesh, elec.order, elec.alpha)
    return w, out
