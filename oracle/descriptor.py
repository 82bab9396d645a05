"""NEP descriptor (oracle, float64 torch).

The paper states that each atom's descriptor has radial and angular
components with species-dependent trainable coefficients and defers the
definition to its NEP references (Sec. II.A, "Details on the descriptor
components ...").  The oracle uses the published NEP3/NEP4 form:

  cutoff      f_c(r) = 1/2 [1 + cos(pi r / r_c)]                  (r < r_c)
  basis       f_k(r) = 1/2 [T_k(x) + 1] f_c(r),  x = 2 (r/r_c - 1)^2 - 1
  radial fn   g_n(r) = sum_k c[t_i][t_j][n][k] f_k(r)   (own c and r_c for radial / angular)
  radial      D^R_n      = sum_j g^R_n(r_ij)
  angular     D^A_{n,l}  = sum_j sum_k g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk),  l = 1..l_max,
                           the diagonal j = k included (Legendre double sum)
  4-body      D^4b_n     = tr(T_n^3),  T_n = sum_j g^A_n(r_ij) (u_ij u_ij^T - I/3)
  order       [D^R_0..n | D^A (l-major, then n) | D^4b_0..n], each component times scaler[nu]

T_k are Chebyshev polynomials of the first kind, P_l Legendre polynomials and
u_ij = r_ij / |r_ij|.  This is a direct evaluation of the double sum over
neighbour pairs; the CUDA path evaluates the same quantity through an
expansion in spherical harmonics instead.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def cutoff_function(r: torch.Tensor, rc: float) -> torch.Tensor:
    return 0.5 * (1.0 + torch.cos(math.pi * r / rc))


def chebyshev_t(x: torch.Tensor, count: int) -> torch.Tensor:
    """T_0..T_{count-1}(x) by the three-term recurrence, stacked on the last axis."""
    polys = [torch.ones_like(x), x]
    while len(polys) < count:
        polys.append(2.0 * x * polys[-1] - polys[-2])
    return torch.stack(polys[:count], dim=-1)


def basis_functions(r: torch.Tensor, rc: float, count: int) -> torch.Tensor:
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    return 0.5 * (chebyshev_t(x, count) + 1.0) * cutoff_function(r, rc)[..., None]


def radial_functions(r: torch.Tensor, ti: np.ndarray, tj: np.ndarray, coeff: torch.Tensor,
                     rc: float) -> torch.Tensor:
    """g_n(r) for every entry: [E, n]."""
    f = basis_functions(r, rc, coeff.shape[-1])
    return torch.einsum("enk,ek->en", coeff[ti, tj], f)


def legendre(c: torch.Tensor, l_max: int) -> torch.Tensor:
    """P_1..P_{l_max}(c) (Bonnet recurrence), stacked on the last axis."""
    p = [torch.ones_like(c), c]
    for l in range(1, l_max):
        p.append(((2 * l + 1) * c * p[l] - l * p[l - 1]) / (l + 1))
    return torch.stack(p[1:l_max + 1], dim=-1)


def _pair_indices(counts: np.ndarray, starts: np.ndarray):
    """All ordered pairs (e1, e2) of entries that share a central atom."""
    sq = counts * counts
    total = int(sq.sum())
    owner = np.repeat(np.arange(len(counts)), sq)
    first = np.repeat(np.cumsum(sq) - sq, sq)
    local = np.arange(total) - first
    c_rep = np.repeat(counts, sq)
    s_rep = np.repeat(starts, sq)
    return owner, s_rep + local // np.maximum(c_rep, 1), s_rep + local % np.maximum(c_rep, 1)


def four_body(t_n: torch.Tensor) -> torch.Tensor:
    """D^4b_n = tr(T_n^3) of the traceless tensors T_n = sum_j g_n (u u^T - I/3), [atoms, n]."""
    return torch.einsum("inab,inbc,inca->in", t_n, t_n, t_n)


def descriptor(vec_r: torch.Tensor, i_r: np.ndarray, j_r: np.ndarray,
               vec_a: torch.Tensor, i_a: np.ndarray, j_a: np.ndarray,
               types: np.ndarray, atoms: np.ndarray, model) -> torch.Tensor:
    """Descriptor of the central atoms ``atoms`` (sorted, contiguous ids allowed).

    vec_r / vec_a are the pair vectors of the radial / angular entries whose
    central atom is in ``atoms`` (entries sorted by central atom).
    Returns [len(atoms), n_des].
    """
    n_loc = len(atoms)
    local = np.full(int(atoms.max()) + 1 if n_loc else 1, -1, dtype=np.int64)
    local[atoms] = np.arange(n_loc)
    li_r = torch.as_tensor(local[i_r])
    li_a_np = local[i_a]
    li_a = torch.as_tensor(li_a_np)

    # radial
    r = torch.linalg.norm(vec_r, dim=1)
    g_r = radial_functions(r, types[i_r], types[j_r], model.c_radial, model.rc_radial)
    n_r = g_r.shape[1]
    d_rad = torch.zeros(n_loc, n_r, dtype=torch.float64).index_add(0, li_r, g_r)

    # angular: Legendre double sum over ordered neighbour pairs, diagonal included
    ra = torch.linalg.norm(vec_a, dim=1)
    u = vec_a / ra[:, None]
    g_a = radial_functions(ra, types[i_a], types[j_a], model.c_angular, model.rc_angular)
    n_a = g_a.shape[1]
    counts = np.bincount(li_a_np, minlength=n_loc)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    owner, e1, e2 = _pair_indices(counts, starts)
    owner_t = torch.as_tensor(owner)
    cos = (u[e1] * u[e2]).sum(1).clamp(-1.0, 1.0)
    pl = legendre(cos, model.l_max)                                  # [P, l]
    gg = g_a[e1] * g_a[e2]                                           # [P, n]
    contrib = (pl[:, :, None] * gg[:, None, :]).reshape(len(owner), model.l_max * n_a)  # l-major, then n
    d_ang = torch.zeros(n_loc, model.l_max * n_a, dtype=torch.float64).index_add(0, owner_t, contrib)

    parts = [d_rad, d_ang]
    if model.use_4body:
        eye = torch.eye(3, dtype=torch.float64)
        outer = u[:, :, None] * u[:, None, :] - eye / 3.0               # [E, 3, 3]
        t_e = g_a[:, :, None, None] * outer[:, None, :, :]               # [E, n, 3, 3]
        t_n = torch.zeros(n_loc, n_a, 3, 3, dtype=torch.float64).index_add(0, li_a, t_e)
        parts.append(four_body(t_n))
    return torch.cat(parts, dim=1) * model.scaler[None, :]
