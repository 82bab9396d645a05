"""The full qNEP force call (oracle, float64).

Stages, in the paper's order:
  1. descriptor D^i of every atom (Sec. II.A, reading in ``descriptor``)
  2. network: site energies U_i (Eq. U_i) and charges q_i (Sec. II.B)
  3. charge scaling q~ = sqrt(eps_inf) q (Sec. II.D) and total-charge correction
     (Eq. charge-scaling, read as q~_i <- q~_i + (Q - sum_j q~_j) / N: the printed
     form does not give sum q~ = Q); the energy uses the screened corrected
     charges q^c = q~^c / sqrt(eps_inf) (Sec. II.D, Coulomb identity)
  4. electrostatics U^ES of q^c: Ewald (Sec. II.B) or PPPM (Sec. II.F), giving
     phi_i = dU^ES/dq^c_i, the static forces and the static virial
  5. chain rule through the charges and the descriptor (Sec. II.C): the
     adjoint lambda_i = dU_i/dD + (phi_i - mean(phi)) dq_i/dD (the correction
     of stage 3 differentiated), then per neighbour entry the gradient
     g_ij = dE/dr_ij of lambda . D^i, taken with autograd; forces
     F_i = sum_j (g_ij - g_ji) + static, virial W = -sum r_ij (x) g_ij + static
  6. polarization P = sum_i q~^c_i r_i (Eq. polarization, positions as given)
     and periodic Born effective charges, Eq. (bec_2), with per-entry
     a_ij = dq~_i/dr_ij (uncorrected network charges) and q~^c_i on the diagonal

Autograd is the differentiation primitive throughout; the paper's explicit
partial-force formulas are not used here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import descriptor as desc_mod
from . import ewald, geometry, network, pppm
from .params import unpack


def correct_charges(qt, q_total):
    """Total-charge correction of the naked charges, read as q~_i + (Q - sum_j q~_j) / N
    (Eq. charge-scaling as printed does not give sum q~ = Q); numpy or torch."""
    return qt + (q_total - qt.sum()) / len(qt)


def _entry_sets(pos, box, hp, elec):
    rc_all = max(hp.rc_radial, hp.rc_angular, elec.rc_real if elec.mode == 1 else 0.0)
    ent = geometry.find_entries(pos, box, rc_all)
    dist = ent.dist
    return (ent.select(dist < hp.rc_radial), ent.select(dist < hp.rc_angular),
            ent.select(dist < elec.rc_real) if elec.mode == 1 else ent.select(dist < 0))


def _chunks(n, size):
    for a0 in range(0, n, size):
        yield np.arange(a0, min(n, a0 + size))


def _slice(ent, atoms, off):
    lo, hi = off[atoms[0]], off[atoms[-1] + 1]
    return ent.i[lo:hi], ent.j[lo:hi], ent.vec[lo:hi], slice(lo, hi)


def descriptors(pos, box, types, hp, blob, chunk=512, entries=None):
    """D for every atom [N, n_des] (no derivatives)."""
    model = unpack(blob, hp)
    if entries is None:
        ent_r, ent_a, _ = _entry_sets(pos, box, hp, _NoReal())
    else:
        ent_r, ent_a = entries
    n = len(pos)
    off_r = geometry.offsets(ent_r.i, n)
    off_a = geometry.offsets(ent_a.i, n)
    out = []
    with torch.no_grad():
        for atoms in _chunks(n, chunk):
            ir, jr, vr, _ = _slice(ent_r, atoms, off_r)
            ia, ja, va, _ = _slice(ent_a, atoms, off_a)
            out.append(desc_mod.descriptor(torch.as_tensor(vr), ir, jr, torch.as_tensor(va), ia, ja,
                                           types, atoms, model))
    return torch.cat(out).numpy()


class _NoReal:
    mode = 2
    rc_real = 0.0


def force_call(positions, box, types, hp, blob, elec, want_bec: bool = True,
               sample=None, chunk: int = 512, printed_pppm: bool = False) -> dict:
    """Energy, forces, virial, charges, BEC and polarization of one structure.

    ``sample``: optional atom ids; forces / BEC are then exact only for those
    atoms (used for large systems), every other output stays exact.
    """
    pos = np.asarray(positions, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    types = np.asarray(types, dtype=np.int64)
    n = len(pos)
    model = unpack(blob, hp)
    ent_r, ent_a, ent_real = _entry_sets(pos, box, hp, elec)
    off_r = geometry.offsets(ent_r.i, n)
    off_a = geometry.offsets(ent_a.i, n)

    # 1. descriptor
    d_all = descriptors(pos, box, types, hp, blob, chunk, (ent_r, ent_a))

    # 2. network and its input gradients (U_i and q_i depend on D^i only)
    d_leaf = torch.tensor(d_all, requires_grad=True)
    u, q = network.site_energy_and_charge(d_leaf, types, model)
    du = torch.autograd.grad(u.sum(), d_leaf, retain_graph=True)[0].numpy()
    dq = torch.autograd.grad(q.sum(), d_leaf)[0].numpy()
    u = u.detach().numpy()
    q = q.detach().numpy()

    # 3. charges
    s = model.sqrt_eps_inf
    qt = s * q
    qt_c = correct_charges(qt, elec.q_total)
    q_c = qt_c / s

    # 4. electrostatics
    if elec.kind == "ewald":
        es = ewald.ewald_static(pos, box, q_c, ent_real, elec)
    else:
        es = ewald.ewald_static(pos, box, q_c, ent_real, elec, with_kspace=False)
        pm = pppm.pppm(pos, box, q_c, elec.mesh, elec.order, elec.alpha, printed_form=printed_pppm)
        es["e_kspace"] = pm["e_kspace"]
        es["phi"] = es["phi"] + pm["phi"]
        es["force"] = es["force"] + pm["force"]
        es["virial"] = es["virial"] + pm["virial"]
    phi = es["phi"]

    # 5. chain rule through charges and descriptor
    lam = du + (phi - phi.mean())[:, None] * dq
    kap = s * dq
    if sample is None:
        central = np.arange(n)
    else:
        sample = np.asarray(sample, dtype=np.int64)
        nbrs = ent_r.i[np.isin(ent_r.j, sample)]
        central = np.unique(np.concatenate([sample, nbrs, ent_a.i[np.isin(ent_a.j, sample)]]))
    g_r = np.zeros_like(ent_r.vec)
    g_a = np.zeros_like(ent_a.vec)
    a_r = np.zeros_like(ent_r.vec)
    a_a = np.zeros_like(ent_a.vec)
    done = np.zeros(n, bool)
    done[central if sample is None else sample] = True
    # contiguous runs of central atoms
    runs = np.split(central, np.nonzero(np.diff(central) != 1)[0] + 1) if len(central) else []
    for run in runs:
        for atoms in _chunks(len(run), chunk):
            atoms = run[atoms]
            ir, jr, vr, sl_r = _slice(ent_r, atoms, off_r)
            ia, ja, va, sl_a = _slice(ent_a, atoms, off_a)
            vr_t = torch.tensor(vr, requires_grad=True)
            va_t = torch.tensor(va, requires_grad=True)
            dc = desc_mod.descriptor(vr_t, ir, jr, va_t, ia, ja, types, atoms, model)
            lam_c = torch.as_tensor(lam[atoms])
            gr, ga = torch.autograd.grad((lam_c * dc).sum(), (vr_t, va_t), retain_graph=want_bec,
                                         allow_unused=True)
            g_r[sl_r] = gr.numpy() if gr is not None else 0.0
            g_a[sl_a] = ga.numpy() if ga is not None else 0.0
            if want_bec:
                kap_c = torch.as_tensor(kap[atoms])
                ar, aa = torch.autograd.grad((kap_c * dc).sum(), (vr_t, va_t), allow_unused=True)
                a_r[sl_r] = ar.numpy() if ar is not None else 0.0
                a_a[sl_a] = aa.numpy() if aa is not None else 0.0

    force = es["force"].copy()
    virial = es["virial"].copy()
    for ent, g in ((ent_r, g_r), (ent_a, g_a)):
        np.add.at(force, ent.i, g)
        np.subtract.at(force, ent.j, g)
        virial -= np.einsum("ea,eb->ab", ent.vec, g)
    out = {
        "energy": float(u.sum() + es["e_real"] + es["e_kspace"] + es["e_self"]),
        "e_nep": float(u.sum()), "e_real": es["e_real"], "e_kspace": es["e_kspace"],
        "e_self": es["e_self"], "site_energy": u, "descriptor": d_all,
        "q_raw": q, "charges": q_c, "qtilde": qt_c, "phi": phi,
        # predicted total charge before the correction, sum_i q~_i (the D_Q term of Sec. II.E)
        "total_charge_raw": float(qt.sum()),
        "forces": force, "virial": virial,
        "polarization": (qt_c[:, None] * pos).sum(0),
        "n_radial_entries": len(ent_r.i), "n_angular_entries": len(ent_a.i),
        "adjoint": lam, "charge_adjoint": kap, "sample_valid": done,
        # per-entry partial forces F_ij = dE/dr_ij of the radial and angular entry sets (the
        # gradients behind the forces and the virial above), with their entries
        "partials": ((ent_r, g_r), (ent_a, g_a)),
    }
    if want_bec:
        out["bec"] = periodic_bec(qt_c, ((ent_r, a_r), (ent_a, a_a)))
    return out


def periodic_bec(qt_c, entry_derivs):
    """Eq. (bec_2) from per-entry charge derivatives a_ij = dq~_i/dr_ij.

    Z_i = q~^c_i I + 1/2 sum over i's entries r_ij (x) a_ij - 1/2 sum over the entries
    (j -> i) of r_ji (x) a_ji (the second term of Eq. bec_2, -r_ji (x) dq~_j/dr_ji).
    """
    bec = qt_c[:, None, None] * np.eye(3)[None]
    for ent, a in entry_derivs:
        half = 0.5 * np.einsum("ea,eb->eab", ent.vec, a)
        np.add.at(bec, ent.i, half)
        np.subtract.at(bec, ent.j, half)
    return bec


def total_energy_autograd(positions, box, types, hp, blob, elec, strain=None):
    """Whole energy as one differentiable function of positions and strain (small systems).

    Returns (energy tensor, positions leaf, strain leaf).  Ewald only.  Used to
    pin the staged chain rule of ``force_call`` (they must agree to rounding).
    """
    pos0 = np.asarray(positions, dtype=np.float64)
    box0 = np.asarray(box, dtype=np.float64)
    types = np.asarray(types, dtype=np.int64)
    n = len(pos0)
    model = unpack(blob, hp)
    ent_r, ent_a, ent_real = _entry_sets(pos0, box0, hp, elec)
    pos = torch.tensor(pos0, requires_grad=True)
    eps = torch.zeros(3, 3, dtype=torch.float64, requires_grad=True) if strain is None else strain
    defm = torch.eye(3, dtype=torch.float64) + eps
    pos_s = pos @ defm.T
    box_s = torch.as_tensor(box0) @ defm.T

    def vecs(ent):
        return pos_s[ent.j] + torch.as_tensor(ent.shift, dtype=torch.float64) @ box_s - pos_s[ent.i]

    d = desc_mod.descriptor(vecs(ent_r), ent_r.i, ent_r.j, vecs(ent_a), ent_a.i, ent_a.j, types,
                            np.arange(n), model)
    u, q = network.site_energy_and_charge(d, types, model)
    s = model.sqrt_eps_inf
    qt = s * q
    q_c = correct_charges(qt, elec.q_total) / s
    e = u.sum()
    if elec.mode == 1:
        e = e + ewald.real_space_energy(vecs(ent_real), ent_real.i, ent_real.j, q_c, elec.alpha)
        e = e + ewald.self_energy(q_c, elec.alpha)
    e = e + ewald.reciprocal_energy(pos_s, box_s, q_c, elec.alpha,
                                    ewald.kspace_integers(box0, elec.kmax))
    return e, pos, eps


def polarization_autograd(positions, box, types, hp, blob, elec):
    """P = sum_i q~^c_i r_i as a differentiable function of the positions (cluster BEC pin)."""
    pos0 = np.asarray(positions, dtype=np.float64)
    box0 = np.asarray(box, dtype=np.float64)
    types = np.asarray(types, dtype=np.int64)
    n = len(pos0)
    model = unpack(blob, hp)
    ent_r, ent_a, _ = _entry_sets(pos0, box0, hp, elec)
    pos = torch.tensor(pos0, requires_grad=True)

    def vecs(ent):
        return pos[ent.j] + torch.as_tensor(ent.shift @ box0) - pos[ent.i]

    d = desc_mod.descriptor(vecs(ent_r), ent_r.i, ent_r.j, vecs(ent_a), ent_a.i, ent_a.j, types,
                            np.arange(n), model)
    _, q = network.site_energy_and_charge(d, types, model)
    s = model.sqrt_eps_inf
    qt = s * q
    qt_c = correct_charges(qt, elec.q_total)
    return (qt_c[:, None] * pos).sum(0), pos


def charges_autograd(positions, box, types, hp, blob, elec):
    """Corrected screened charges q^c(r) as a differentiable function of the positions.

    q~ = sqrt(eps_inf) q, q~^c = q~ + (Q - sum q~)/N (Eq. charge-scaling, reading of
    the stage-3 docstring), q^c = q~^c / sqrt(eps_inf).  Returns (q^c, positions leaf).
    """
    pos0 = np.asarray(positions, dtype=np.float64)
    box0 = np.asarray(box, dtype=np.float64)
    types = np.asarray(types, dtype=np.int64)
    n = len(pos0)
    model = unpack(blob, hp)
    ent_r, ent_a, _ = _entry_sets(pos0, box0, hp, elec)
    pos = torch.tensor(pos0, requires_grad=True)

    def vecs(ent):
        return pos[ent.j] + torch.as_tensor(ent.shift @ box0) - pos[ent.i]

    d = desc_mod.descriptor(vecs(ent_r), ent_r.i, ent_r.j, vecs(ent_a), ent_a.i, ent_a.j, types,
                            np.arange(n), model)
    _, q = network.site_energy_and_charge(d, types, model)
    s = model.sqrt_eps_inf
    qt = s * q
    return correct_charges(qt, elec.q_total) / s, pos
