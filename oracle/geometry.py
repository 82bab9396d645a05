"""Neighbour entries with periodic images (oracle, float64).

The paper never describes neighbour search; it needs the pair vectors
r_ij = r_j - r_i (Sec. II.C, per-atom virial paragraph) for every j within the
cutoff (radial / angular cutoffs of Sec. II.A, real-space cutoff r_c of
Sec. II.B).  Under periodic boundary conditions the oracle takes every image:
all (j, T) != (i, 0) with |r_j + T.box - r_i| < r_c, T an integer triple.
Small boxes (edge < 2 r_c) therefore hold several images of the same j, and
self images of i.

Rows of ``box`` are the lattice vectors; any cell shape is accepted by the
brute-force enumeration (the k-d tree shortcut needs an orthorhombic box).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np


@dataclasses.dataclass
class Entries:
    i: np.ndarray       # (E,) central atom
    j: np.ndarray       # (E,) neighbour atom
    shift: np.ndarray   # (E, 3) integer image T
    vec: np.ndarray     # (E, 3) r_ij = r_j + T.box - r_i  (float64)

    def select(self, mask: np.ndarray) -> "Entries":
        return Entries(self.i[mask], self.j[mask], self.shift[mask], self.vec[mask])

    @property
    def dist(self) -> np.ndarray:
        return np.sqrt(np.einsum("ed,ed->e", self.vec, self.vec))


def box_lengths(box: np.ndarray) -> np.ndarray:
    """Edge lengths of an orthorhombic box (raises for a sheared one)."""
    box = np.asarray(box, dtype=np.float64)
    if np.any(np.abs(box - np.diag(np.diag(box))) > 0):
        raise NotImplementedError("orthorhombic box required here")
    return np.diag(box).copy()


def perpendicular_widths(box: np.ndarray) -> np.ndarray:
    """Distances between opposite faces of the cell spanned by the rows of ``box``."""
    box = np.asarray(box, dtype=np.float64)
    vol = abs(np.linalg.det(box))
    return np.array([vol / np.linalg.norm(np.cross(box[(d + 1) % 3], box[(d + 2) % 3]))
                     for d in range(3)])


def neighbor_entries(pos: np.ndarray, box: np.ndarray, rc: float, chunk: int = 256) -> Entries:
    """Brute-force enumeration of all image pairs within ``rc``, sorted by (i, j, T).

    Works for any cell (rows of ``box`` = lattice vectors).  For each pair the
    separation is first wrapped to the nearest image in fractional
    coordinates; then every shift with |T_d| <= M_d is tried, M_d large enough
    (from the perpendicular widths) that no image within rc is missed.
    """
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    inv = np.linalg.inv(box)
    n = len(pos)
    widths = perpendicular_widths(box)
    reach = [int(np.floor(rc / w + 0.5)) for w in widths]   # |T_d| < rc / w_d + 1/2
    shifts = np.array(list(itertools.product(*[range(-m, m + 1) for m in reach])), dtype=np.int64)
    out_i, out_j, out_t = [], [], []
    rc2 = rc * rc
    for a0 in range(0, n, chunk):
        a1 = min(n, a0 + chunk)
        d = pos[None, :, :] - pos[a0:a1, None, :]            # (c, N, 3)
        base = -np.round(d @ inv)                              # nearest image, fractional
        d = d + base @ box
        for t in shifts:
            v = d + t @ box
            r2 = np.einsum("cnd,cnd->cn", v, v)
            ci, cj = np.nonzero(r2 < rc2)
            tt = base[ci, cj].astype(np.int64) + t
            keep = ~((cj == ci + a0) & np.all(tt == 0, axis=1))
            out_i.append(ci[keep] + a0)
            out_j.append(cj[keep])
            out_t.append(tt[keep])
    i = np.concatenate(out_i)
    j = np.concatenate(out_j)
    t = np.concatenate(out_t).reshape(-1, 3)
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0], j, i))
    i, j, t = i[order], j[order], t[order]
    # the vector from the integer image: r_ij = r_j + T.box - r_i
    v = pos[j] + t @ box - pos[i]
    return Entries(i, j, t, v)


def offsets(i: np.ndarray, n_atoms: int) -> np.ndarray:
    """CSR offsets of entries grouped by central atom (entries sorted by i)."""
    return np.concatenate([[0], np.cumsum(np.bincount(i, minlength=n_atoms))]).astype(np.int64)


def neighbor_entries_kdtree(pos: np.ndarray, box: np.ndarray, rc: float) -> Entries:
    """Same entries as ``neighbor_entries`` for boxes with every edge > 2 rc.

    There each pair has at most one image within rc (the minimum image), so a
    periodic k-d tree (scipy) finds the pairs; used for large systems where the
    brute-force enumeration is too slow.
    """
    from scipy.spatial import cKDTree

    pos = np.asarray(pos, dtype=np.float64)
    lengths = box_lengths(box)
    if np.any(lengths <= 2.0 * rc):
        raise ValueError("k-d tree path needs every box edge > 2 rc")
    wrapped = pos - np.floor(pos / lengths) * lengths
    wrapped = np.where(wrapped >= lengths, wrapped - lengths, wrapped)
    tree = cKDTree(wrapped, boxsize=lengths)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    i = np.concatenate([pairs[:, 0], pairs[:, 1]]).astype(np.int64)
    j = np.concatenate([pairs[:, 1], pairs[:, 0]]).astype(np.int64)
    d = pos[j] - pos[i]
    t = -np.round(d / lengths).astype(np.int64)
    v = pos[j] + t * lengths - pos[i]
    keep = np.einsum("ed,ed->e", v, v) < rc * rc
    i, j, t, v = i[keep], j[keep], t[keep], v[keep]
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0], j, i))
    return Entries(i[order], j[order], t[order], v[order])


def find_entries(pos: np.ndarray, box: np.ndarray, rc: float) -> Entries:
    """Brute force for small systems or small / sheared boxes, k-d tree otherwise."""
    box = np.asarray(box, dtype=np.float64)
    ortho = not np.any(np.abs(box - np.diag(np.diag(box))) > 0)
    if ortho and len(pos) > 4000 and np.all(np.diag(box) > 2.0 * rc):
        return neighbor_entries_kdtree(pos, box, rc)
    return neighbor_entries(pos, box, rc)
