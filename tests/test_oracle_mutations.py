"""Planted mistakes: each pin of the oracle must fail when a plausible error is put into the oracle.

Every test here replaces one oracle function, on the CPU and for the duration of the
test only (pytest's monkeypatch), by a variant with a typical slip -- a dropped term,
a wrong sign, an index off by one, a transposed operand, a term given to the wrong
atom -- and checks that the pin written for that function then fails.  The pins are
the ordinary tests of tests/test_oracle_*.py, called directly.
"""
import math

import numpy as np
import pytest
import torch

from oracle import descriptor as dm
from oracle import ewald, field, forcecall, md, pppm, training, virial
from tests import test_oracle_descriptor as t_desc
from tests import test_oracle_electrostatics as t_es
from tests import test_oracle_forces as t_forces
from tests import test_oracle_md as t_md
from tests import test_oracle_training as t_tr
from tests import test_oracle_virial as t_vir
from tests.test_oracle_field import cluster  # noqa: F401  (fixture for the field pins)
from tests.test_oracle_forces import batio3_subcell  # noqa: F401  (fixture for the force pins)
from tests import test_oracle_field as t_field
from paper_2601_19034_gb300 import workloads as wl


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_control_pins_pass_unmodified(cluster):  # noqa: F811
    t_desc.test_cutoff_and_basis_edges()
    t_desc.test_chebyshev_matches_numpy()
    t_es.test_nacl_madelung_constant()
    t_field.test_cluster_electric_force_is_gradient_of_field_energy(cluster)
    t_tr.test_utilities_and_ranks()


def test_cutoff_with_the_wrong_sign(monkeypatch):
    monkeypatch.setattr(dm, "cutoff_function", lambda r, rc: 0.5 * (1.0 - torch.cos(math.pi * r / rc)))
    _fails(t_desc.test_cutoff_and_basis_edges)


def test_chebyshev_index_off_by_one(monkeypatch):
    orig = dm.chebyshev_t
    monkeypatch.setattr(dm, "chebyshev_t", lambda x, count: orig(x, count + 1)[..., 1:])
    _fails(t_desc.test_chebyshev_matches_numpy)


def test_legendre_recurrence_slip(monkeypatch):
    def wrong(c, l_max):
        p = [torch.ones_like(c), c]
        for l in range(1, l_max):
            p.append(((2 * l - 1) * c * p[l] - l * p[l - 1]) / (l + 1))
        return torch.stack(p[1:l_max + 1], dim=-1)
    monkeypatch.setattr(dm, "legendre", wrong)
    _fails(t_desc.test_legendre_matches_scipy)
    _fails(t_desc.test_angular_descriptor_addition_theorem)


def test_angular_sum_without_the_diagonal(monkeypatch):
    orig = dm._pair_indices

    def off_diagonal(counts, starts):
        owner, e1, e2 = orig(counts, starts)
        keep = e1 != e2
        return owner[keep], e1[keep], e2[keep]
    monkeypatch.setattr(dm, "_pair_indices", off_diagonal)
    _fails(t_desc.test_angular_descriptor_addition_theorem)


def test_self_energy_dropped(monkeypatch):
    monkeypatch.setattr(ewald, "self_energy", lambda q, alpha: 0.0 * q.sum())
    _fails(t_es.test_nacl_madelung_constant)


def test_real_space_with_erf_for_erfc(monkeypatch):
    def wrong(vec, i, j, q, alpha):
        r = torch.linalg.norm(vec, dim=1)
        ii, jj = torch.as_tensor(i), torch.as_tensor(j)
        return 0.5 * ewald.KE * (q[ii] * q[jj] * torch.special.erf(alpha * r) / r).sum()
    monkeypatch.setattr(ewald, "real_space_energy", wrong)
    _fails(t_es.test_nacl_madelung_constant)


def test_reciprocal_green_function_without_1_over_k2(monkeypatch):
    def wrong(pos, box, q, alpha, nvec):
        inv = torch.linalg.inv(box)
        kv = 2.0 * math.pi * torch.as_tensor(nvec, dtype=torch.float64) @ inv.T
        k2 = (kv * kv).sum(1)
        omega = torch.abs(torch.linalg.det(box))
        g = (2.0 * math.pi / omega) * torch.exp(-k2 / (4.0 * alpha * alpha))
        phase = pos @ kv.T
        s_re = (q[:, None] * torch.cos(phase)).sum(0)
        s_im = -(q[:, None] * torch.sin(phase)).sum(0)
        return ewald.KE * (g * (s_re * s_re + s_im * s_im)).sum()
    monkeypatch.setattr(ewald, "reciprocal_energy", wrong)
    _fails(t_es.test_nacl_madelung_constant)


def test_alias_sum_with_the_printed_sign(monkeypatch):
    orig = pppm.alias_sum

    def printed(n, mesh, order, terms=None):
        if terms is None and order == 5:
            z2 = np.sin(math.pi * n / mesh) ** 2
            return 1.0 - 5.0 / 3.0 * z2 + 7.0 / 9.0 * z2 ** 2 + 17.0 / 189.0 * z2 ** 3 + 2.0 / 2835.0 * z2 ** 4
        return orig(n, mesh, order, terms)
    monkeypatch.setattr(pppm, "alias_sum", printed)
    _fails(t_es.test_alias_sum_closed_form_and_sign)


def test_field_force_with_z_transposed(monkeypatch, cluster):  # noqa: F811
    monkeypatch.setattr(field, "electric_force",
                        lambda bec, e: np.einsum("b,iab->ia", np.asarray(e, float), np.asarray(bec).reshape(-1, 3, 3)))
    _fails(t_field.test_cluster_electric_force_is_gradient_of_field_energy, cluster)


def test_polarization_current_with_z_transposed(monkeypatch, cluster):  # noqa: F811
    monkeypatch.setattr(field, "polarization_current",
                        lambda bec, v: np.einsum("iba,ib->a", np.asarray(bec).reshape(-1, 3, 3), np.asarray(v)))
    _fails(t_field.test_cluster_polarization_current_is_time_derivative, cluster)


def test_utilities_without_the_baseline(monkeypatch):
    def wrong(n):
        k = np.arange(1, n + 1, dtype=np.float64)
        w = np.maximum(0.0, math.log(n / 2.0 + 1.0) - np.log(k))
        return w / w.sum()
    monkeypatch.setattr(training, "utilities", wrong)
    _fails(t_tr.test_utilities_and_ranks)


def test_snes_sigma_step_with_the_wrong_sign(monkeypatch):
    def wrong(mu, sigma, s, fitness, eta_mu=None, eta_sigma=None):
        s = np.asarray(s, dtype=np.float64)
        em, es = training.default_rates(s.shape[1])
        u = training.utilities(s.shape[0])[training.ranks(fitness)]
        return (np.asarray(mu) + em * np.asarray(sigma) * (u @ s),
                np.asarray(sigma) * np.exp(-0.5 * es * (u @ (s * s - 1.0))))
    monkeypatch.setattr(training, "update", wrong)
    _fails(t_tr.test_snes_minimises_separable_quadratic)


def test_per_atom_virial_given_to_the_central_atom(monkeypatch):
    def wrong(w, ent, g):
        if len(ent.i):
            np.add.at(w, ent.i, -np.einsum("ea,eb->eab", ent.vec, g))
    monkeypatch.setattr(virial, "_entry_term", wrong)
    _fails(t_vir.test_energy_moment_identity_fixes_the_convention)


def test_bec_without_the_half(monkeypatch):
    def doubled(qt_c, entry_derivs):
        bec = np.asarray(qt_c)[:, None, None] * np.eye(3)[None]
        for ent, a in entry_derivs:
            full = np.einsum("ea,eb->eab", ent.vec, a)
            np.add.at(bec, ent.i, full)
            np.subtract.at(bec, ent.j, full)
        return bec
    monkeypatch.setattr(forcecall, "periodic_bec", doubled)
    _fails(t_forces.test_periodic_bec_is_dp_dr_for_an_isolated_dimer)


def test_network_bias_added(monkeypatch):
    from oracle import network

    def wrong(d, types, model):
        t = torch.as_tensor(types, dtype=torch.long)
        h = torch.tanh(torch.einsum("imn,in->im", model.w0[t], d) + model.b0[t])
        return (model.w1e[t] * h).sum(1) - model.b1e[t], (model.w1q[t] * h).sum(1) - model.b1q[t]
    monkeypatch.setattr(network, "site_energy_and_charge", wrong)
    _fails(t_desc.test_network_matches_explicit_loop)


def test_bspline_of_the_wrong_order(monkeypatch):
    def one_order_up(order, x):
        # the centred cardinal B-spline of order p + 1 from truncated powers (not recursive, so the
        # oracle's own recursion is not re-entered)
        p = order + 1
        x = np.asarray(x, dtype=np.float64)
        terms = [(-1) ** k * math.comb(p, k) * np.clip(x + p / 2.0 - k, 0.0, None) ** (p - 1) for k in range(p + 1)]
        return sum(terms) / math.factorial(p - 1)
    monkeypatch.setattr(pppm, "bspline", one_order_up)
    _fails(t_es.test_bspline_identities)


def test_influence_function_with_the_printed_single_power(monkeypatch):
    orig = pppm.influence
    monkeypatch.setattr(pppm, "influence", lambda lengths, mesh, order, alpha, printed_form=False:
                        orig(lengths, mesh, order, alpha, True))
    _fails(t_es.test_pppm_converges_to_ewald)


def test_neighbour_search_without_periodic_images(monkeypatch):
    from oracle import geometry
    orig = geometry.neighbor_entries

    def no_images(pos, box, rc, chunk=256):
        ent = orig(pos, box, rc, chunk)
        return ent.select(np.all(ent.shift == 0, axis=1))
    monkeypatch.setattr(geometry, "neighbor_entries", no_images)
    _fails(t_desc.test_image_enumeration_counts_and_kdtree)
    _fails(t_desc.test_descriptor_supercell_replication_small_box)


def test_charge_correction_with_the_wrong_sign(monkeypatch, batio3_subcell):  # noqa: F811
    monkeypatch.setattr(forcecall, "correct_charges", lambda qt, q_total: qt - (q_total - qt.sum()) / len(qt))
    _fails(t_forces.test_charge_correction_and_bec_sum_rule, batio3_subcell)


def test_four_body_as_the_cube_of_the_trace(monkeypatch):
    monkeypatch.setattr(dm, "four_body", lambda t_n: torch.einsum("inaa->in", t_n) ** 3)
    _fails(t_desc.test_four_body_brute_force_triple_sum)


def test_heyes_kernel_with_half_the_gaussian_term(monkeypatch):
    def wrong(pos, box, q, alpha, kmax, chunk=2048):
        pos, q, box = np.asarray(pos, float), np.asarray(q, float), np.asarray(box, float)
        nvec = ewald.kspace_integers(box, kmax)
        kv = 2.0 * math.pi * nvec @ np.linalg.inv(box).T
        k2 = np.einsum("kd,kd->k", kv, kv)
        g = (2.0 * math.pi / abs(np.linalg.det(box))) * np.exp(-k2 / (4.0 * alpha * alpha)) / k2
        th = pos @ kv.T
        s_re, s_im = (q[:, None] * np.cos(th)).sum(0), -(q[:, None] * np.sin(th)).sum(0)
        re = q[:, None] * (np.cos(th) * s_re[None] - np.sin(th) * s_im[None])
        fac = 1.0 / (4.0 * alpha * alpha) + 2.0 / k2
        bmat = np.eye(3)[None] - fac[:, None, None] * np.einsum("ka,kb->kab", kv, kv)
        return ewald.KE * np.einsum("ik,k,kab->iab", re, g, bmat)
    monkeypatch.setattr(virial, "kspace_static_ewald", wrong)
    s = wl.batio3_supercell(2, seed=31)
    cell = (s.positions.astype(np.float64), s.box, s.types, None, None)
    _fails(t_vir.test_kspace_per_atom_sums_to_the_mesh_and_ewald_totals, cell)


def test_ranks_with_nan_first(monkeypatch):
    def wrong(fitness):
        f = np.asarray(fitness, dtype=np.float64)
        order = sorted(range(len(f)), key=lambda c: (not np.isnan(f[c]), np.nan_to_num(f[c]), c))
        r = np.empty(len(f), dtype=np.int64)
        for k, c in enumerate(order):
            r[c] = k
        return r
    monkeypatch.setattr(training, "ranks", wrong)
    _fails(t_tr.test_utilities_and_ranks)


def test_energy_error_per_structure_not_per_atom(monkeypatch):
    orig = training.loss_terms

    def wrong(energy, forces, energy_ref, forces_ref, atom_offsets, params):
        d_e, d_f, l1, l2 = orig(energy, forces, energy_ref, forces_ref, atom_offsets, params)
        off = np.asarray(atom_offsets)
        has = np.diff(off) > 0
        de = np.asarray(energy)[:, has] - np.asarray(energy_ref)[None, has]
        return np.sqrt((de ** 2).mean(1)), d_f, l1, l2
    monkeypatch.setattr(training, "loss_terms", wrong)
    _fails(t_tr.test_loss_closed_forms)


def test_virial_rmse_over_all_nine_components(monkeypatch):
    """Averaging over all nine components (lower triangle counted too) fails the six-component pins."""
    def wrong(virial, virial_ref, atom_offsets):
        off = np.asarray(atom_offsets, dtype=np.int64)
        n_s = np.diff(off)
        has = n_s > 0
        w = np.asarray(virial, dtype=np.float64).reshape(-1, len(n_s), 3, 3)
        wr = np.asarray(virial_ref, dtype=np.float64).reshape(len(n_s), 3, 3)
        dv = (w[:, has] - wr[None, has]) / n_s[None, has, None, None]
        return np.sqrt((dv ** 2).reshape(w.shape[0], -1).mean(axis=1))
    monkeypatch.setattr(training, "virial_rmse", wrong)
    with pytest.raises(AssertionError):
        t_tr.test_virial_rmse_closed_forms()


def test_bec_rmse_over_every_structure(monkeypatch):
    """Counting the structures without reference BEC fails the closed forms."""
    def wrong(bec, bec_ref, atom_offsets, has_ref):
        off = np.asarray(atom_offsets, dtype=np.int64)
        z = np.asarray(bec, dtype=np.float64).reshape(-1, off[-1], 9)
        zr = np.asarray(bec_ref, dtype=np.float64).reshape(off[-1], 9)
        return np.sqrt(((z - zr[None]) ** 2).reshape(z.shape[0], -1).mean(axis=1))
    monkeypatch.setattr(training, "bec_rmse", wrong)
    _fails(t_tr.test_bec_rmse_closed_forms)


def test_total_charge_after_the_correction(monkeypatch):
    """Reporting the corrected charges' sum (the target, by construction) fails the closed form."""
    orig = forcecall.force_call

    def wrong(*args, **kw):
        out = orig(*args, **kw)
        out["total_charge_raw"] = float(out["qtilde"].sum())
        return out
    monkeypatch.setattr(forcecall, "force_call", wrong)
    _fails(t_tr.test_force_call_total_charge_before_the_correction)


def test_general_cell_pppm_gradient_with_h_inverse_transposed(monkeypatch):
    """Mapping the fractional gradients with H^-1 instead of H^-T fails the PPPM -> Ewald pin."""
    from tests import test_oracle_triclinic as t_tri
    orig = np.linalg.inv

    def general(pos, box, q, mesh, order, alpha, printed_form=False, chunk=65536):
        # the module's code with the transposed map: d/dr = gf @ H^-1
        pos = np.asarray(pos, np.float64)
        q = np.asarray(q, np.float64)
        hinv = orig(np.asarray(box, np.float64))
        out = pppm_general_orig(pos, box, q, mesh, order, alpha, printed_form, chunk)
        lengths = np.linalg.norm(box, axis=1)
        mesh_t = tuple(int(m) for m in mesh)
        ntot = int(np.prod(mesh_t))
        s = np.fft.fftn(out["rho"])
        gopt, k, k2, nyq, n = pppm.influence(lengths, mesh_t, order, alpha, printed_form, box=box)
        sg = s * gopt
        ff = []
        for c in range(3):
            comp = 1j * (2.0 * math.pi * n[c]) * sg
            comp[nyq[c]] = 0.0
            ff.append((np.fft.ifftn(comp) * ntot).real.ravel())
        pts, w = pppm._gather_weights(pos, lengths, mesh_t, order, hinv)
        flat, wt = pppm._flat_stencil(pts, w, mesh_t)
        gf = np.stack([(wt * ff[c][flat]).sum(1) for c in range(3)], -1)
        out["force"] = -2.0 * pppm.KE * q[:, None] * (gf @ hinv)
        return out
    pppm_general_orig = pppm.pppm_general
    monkeypatch.setattr(pppm, "pppm_general", general)
    _fails(t_tri.test_pppm_in_a_general_cell_converges_to_ewald)


def test_network_slips_fail_the_zero_weight_closed_form(monkeypatch, batio3_subcell):  # noqa: F811
    """The closed form with W0 = 0 catches, without restating Eq. U_i, the hidden bias added and
    the output layer taken from the first species for every atom."""
    from oracle import network

    def bias_added(d, types, model):
        t = torch.as_tensor(types, dtype=torch.long)
        h = torch.tanh(torch.einsum("imn,in->im", model.w0[t], d) + model.b0[t])
        return (model.w1e[t] * h).sum(1) - model.b1e[t], (model.w1q[t] * h).sum(1) - model.b1q[t]

    def first_species_output(d, types, model):
        t = torch.as_tensor(types, dtype=torch.long)
        h = torch.tanh(torch.einsum("imn,in->im", model.w0[t], d) - model.b0[t])
        z = torch.zeros_like(t)
        return (model.w1e[z] * h).sum(1) - model.b1e[z], (model.w1q[z] * h).sum(1) - model.b1q[z]

    for wrong in (bias_added, first_species_output):
        monkeypatch.setattr(network, "site_energy_and_charge", wrong)
        _fails(t_forces.test_network_with_zero_input_weights_is_a_closed_form, batio3_subcell)
    monkeypatch.undo()
    t_forces.test_network_with_zero_input_weights_is_a_closed_form(batio3_subcell)


def test_general_cell_wave_vectors_with_h_inverse_transposed(monkeypatch):
    """k = 2 pi n H^-1 (transposed) instead of 2 pi H^-1 n: the forces-and-virial differences in a
    sheared cell cannot see it (energy and derivatives share it), the unimodular change of cell
    and PPPM -> Ewald in a sheared box do."""
    from tests import test_oracle_triclinic as t_tri

    def wrong(pos, box, q, alpha, nvec):
        inv = torch.linalg.inv(box)
        kv = 2.0 * math.pi * torch.as_tensor(nvec, dtype=torch.float64) @ inv
        k2 = (kv * kv).sum(1)
        omega = torch.abs(torch.linalg.det(box))
        g = (2.0 * math.pi / omega) * torch.exp(-k2 / (4.0 * alpha * alpha)) / k2
        phase = pos @ kv.T
        s_re = (q[:, None] * torch.cos(phase)).sum(0)
        s_im = -(q[:, None] * torch.sin(phase)).sum(0)
        return ewald.KE * (g * (s_re * s_re + s_im * s_im)).sum()
    monkeypatch.setattr(ewald, "reciprocal_energy", wrong)
    _fails(t_tri.test_unimodular_change_of_cell_leaves_the_force_call_unchanged, 1)
    _fails(t_tri.test_pppm_in_a_general_cell_converges_to_ewald)


def test_drift_without_the_half(monkeypatch):
    def wrong(x, v, f, masses, h):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
        return x + h * v + h * h * md.acceleration(f, masses)
    monkeypatch.setattr(md, "positions_after_step", wrong)
    _fails(t_md.test_harmonic_well_follows_the_closed_form_of_the_map, 1.2)
    _fails(t_md.test_energy_error_is_second_order_in_the_step)


def test_velocity_half_step_with_the_old_forces_only(monkeypatch):
    def wrong(v, f_old, f_new, masses, h):
        return np.asarray(v, dtype=np.float64).reshape(-1, 3) + h * md.acceleration(f_old, masses)
    monkeypatch.setattr(md, "velocities_after_step", wrong)
    _fails(t_md.test_harmonic_well_follows_the_closed_form_of_the_map, 1.2)
    _fails(t_md.test_reversing_the_velocities_retraces_the_trajectory)


def test_kinetic_energy_conversion_mistyped(monkeypatch):
    monkeypatch.setattr(md, "KE_UNIT", md.DALTON / md.E_CHARGE * 1e10 * 1.0001)
    _fails(t_md.test_unit_conversions)
