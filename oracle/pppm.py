"""PPPM reciprocal-space electrostatics (oracle, float64 numpy).

Sec. II.F.  Conventions (the paper fixes none of them; these are the readings):
  mesh points       r_s = (s_x h_x, s_y h_y, s_z h_z), h_d = L_d / N_d, s_d in [0, N_d)
  assignment W      separable W(x) W(y) W(z); W is the order-P cardinal B-spline of
                    Deserno and Holm in mesh units (support P points), centred on the
                    atom: odd P uses the nearest mesh point and the (P-1)/2 points on
                    each side, even P the P points around the atom
  charge mesh       rho_s = sum_i q_i W(r_i - r_s)
  structure factor  S(k) = sum_s rho_s exp(-i k.r_s)  (forward FFT)
  wave vectors      k_d = 2 pi n_d / L_d, -N_d/2 <= n_d < N_d/2, k = 0 excluded
  energy            U^k = k_e sum_{k != 0} G_opt(k) |S(k)|^2
  influence         G_opt = G(k) [prod_d sinc^P(pi n_d/N_d)]^2 / [prod_d A(z_d)]^2,
                    z_d = sin(pi n_d / N_d), A(z) = sum_m sinc^{2P}(pi (n/N + m));
                    for P = 5, A(z) = 1 - 5/3 z^2 + 7/9 z^4 - 17/189 z^6 + 2/2835 z^8.
                    The paper prints +17/189 and the denominator to the first power;
                    both are read as typesetting slips (the alias sum is the squared
                    denominator of the Hockney-Eastwood optimal influence function with
                    the numerator alias sum truncated to m = 0, and the printed sign
                    does not reproduce the sum).  ``printed_form=True`` keeps the
                    single power for comparison.
  inverse transform unnormalised: F^-1[X](r_s) = sum_k X(k) exp(i k.r_s)
  static force      Eq. (force-static-fft): F_i = -2 k_e q_i sum_s W(r_i - r_s) F^-1[i k S G_opt](r_s),
                    the Nyquist plane n_d = -N_d/2 of the d-th component set to zero
  potential         phi_i = dU^k/dq_i = 2 k_e sum_s W(r_i - r_s) F^-1[S G_opt](r_s)
                    (the factor of Eq. force-dynamic-fft)
  virial            W^k = k_e sum_k G_opt |S|^2 B,  B = I - (2/(4 alpha^2) + 2/k^2) k k^T,
                    as the Ewald total virial (Eq. virial-kspace-total)
General (triclinic) cells, rows of H the lattice vectors a_d (the paper treats orthorhombic
meshes only; this is the reading that reduces to the above when H is diagonal):
  mesh points       r_s = sum_d (s_d / N_d) a_d; an atom's mesh-unit coordinates are its
                    fractional coordinates (r H^-1) times N_d, the stencil and weights as above
  wave vectors      k = 2 pi H^-1 n (k . r_s = 2 pi sum_d n_d s_d / N_d: the same FFT),
                    G(k) with V = det H; the alias sums depend on n_d / N_d only (unchanged)
  field             the three fractional gradients F^-1[i 2 pi n_c S G_opt] (Nyquist plane of
                    n_c zeroed in the c-th), combined at the atom into the Cartesian
                    d/dr_a = sum_c H^-1[a][c] d/ds_c; for a diagonal H this is the ik form above
"""
from __future__ import annotations

import math

import numpy as np

KE = 14.3996454784


def bspline(order: int, x: np.ndarray) -> np.ndarray:
    """Centred cardinal B-spline M_P(x) (support |x| < P/2) by the order recurrence.

    M_1 is the unit box; M_P(x) = [(P/2 + x) M_{P-1}(x + 1/2) + (P/2 - x) M_{P-1}(x - 1/2)] / (P - 1).
    """
    x = np.asarray(x, dtype=np.float64)
    if order == 1:
        return ((x >= -0.5) & (x < 0.5)).astype(np.float64)
    p = order
    return ((p / 2.0 + x) * bspline(p - 1, x + 0.5) + (p / 2.0 - x) * bspline(p - 1, x - 0.5)) / (p - 1)


def stencil(u: np.ndarray, order: int):
    """Mesh points and weights of the assignment for mesh-unit coordinates u: [..., P]."""
    if order % 2:
        s0 = np.rint(u).astype(np.int64)
        offs = np.arange(-(order // 2), order // 2 + 1)
    else:
        s0 = np.floor(u).astype(np.int64)
        offs = np.arange(-(order // 2) + 1, order // 2 + 1)
    pts = s0[..., None] + offs
    return pts, bspline(order, u[..., None] - pts)


def alias_sum(n: np.ndarray, mesh: int, order: int, terms: int | None = None) -> np.ndarray:
    """A = sum_m sinc^{2P}(pi (n/N + m)): closed form for P = 5, else brute force."""
    if terms is None and order == 5:
        z2 = np.sin(math.pi * n / mesh) ** 2
        return 1.0 - 5.0 / 3.0 * z2 + 7.0 / 9.0 * z2 ** 2 - 17.0 / 189.0 * z2 ** 3 + 2.0 / 2835.0 * z2 ** 4
    terms = terms or 200
    x = n / mesh
    total = np.zeros_like(x, dtype=np.float64)
    for m in range(-terms, terms + 1):
        total += np.sinc(x + m) ** (2 * order)   # np.sinc(t) = sin(pi t)/(pi t)
    return total


def mesh_integers(mesh: int) -> np.ndarray:
    return np.fft.fftfreq(mesh, 1.0 / mesh).round().astype(np.int64)   # [0..N/2-1, -N/2..-1]


def influence(lengths, mesh, order: int, alpha: float, printed_form: bool = False, box=None):
    """G_opt on the full FFT grid, and the wave-vector components (box: a general cell, rows the
    lattice vectors; then k = 2 pi H^-1 n and the volume is det H)."""
    ns = [mesh_integers(m) for m in mesh]
    n = np.meshgrid(*ns, indexing="ij")
    if box is None:
        k = [2.0 * math.pi * n[d] / lengths[d] for d in range(3)]
        omega = float(np.prod(lengths))
    else:
        hinv = np.linalg.inv(np.asarray(box, np.float64))
        k = [2.0 * math.pi * (hinv[a, 0] * n[0] + hinv[a, 1] * n[1] + hinv[a, 2] * n[2]) for a in range(3)]
        omega = float(abs(np.linalg.det(np.asarray(box, np.float64))))
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, (2.0 * math.pi / omega) * np.exp(-k2 / (4 * alpha * alpha)) / k2, 0.0)
    u2 = np.ones_like(k2)
    den = np.ones_like(k2)
    for d in range(3):
        u2 = u2 * np.sinc(n[d] / mesh[d]) ** (2 * order)
        den = den * alias_sum(n[d], mesh[d], order)
    gopt = g * u2 / (den if printed_form else den * den)
    nyq = [n[d] == -(mesh[d] // 2) if mesh[d] % 2 == 0 else np.zeros_like(k2, bool) for d in range(3)]
    if box is not None:
        return gopt, k, k2, nyq, n
    return gopt, k, k2, nyq


def _gather_weights(pos, lengths, mesh, order, hinv=None):
    if hinv is None:
        u = pos / (lengths / np.asarray(mesh))        # mesh units, [N, 3]
    else:
        u = (pos @ hinv) * np.asarray(mesh)           # fractional coordinates times N_d
    pts, w = stencil(u, order)                         # [N, 3, P]
    for d in range(3):
        pts[:, d] %= mesh[d]
    return pts, w


def _flat_stencil(pts, w, mesh):
    ix = pts[:, 0, :, None, None]
    iy = pts[:, 1, None, :, None]
    iz = pts[:, 2, None, None, :]
    flat = (ix * mesh[1] + iy) * mesh[2] + iz          # [N, P, P, P]
    wt = w[:, 0, :, None, None] * w[:, 1, None, :, None] * w[:, 2, None, None, :]
    return flat.reshape(len(pts), -1), wt.reshape(len(pts), -1)


def pppm(pos: np.ndarray, box: np.ndarray, q: np.ndarray, mesh, order: int, alpha: float,
         printed_form: bool = False, chunk: int = 65536) -> dict:
    box = np.asarray(box, np.float64)
    if np.count_nonzero(box - np.diag(np.diag(box))):
        return pppm_general(pos, box, q, mesh, order, alpha, printed_form, chunk)
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    lengths = np.diag(np.asarray(box, np.float64)).copy()
    mesh = tuple(int(m) for m in mesh)
    ntot = int(np.prod(mesh))
    rho = np.zeros(ntot)
    for a0 in range(0, len(pos), chunk):
        pts, w = _gather_weights(pos[a0:a0 + chunk], lengths, mesh, order)
        flat, wt = _flat_stencil(pts, w, mesh)
        np.add.at(rho, flat.ravel(), (wt * q[a0:a0 + chunk, None]).ravel())
    rho = rho.reshape(mesh)
    s = np.fft.fftn(rho)
    gopt, k, k2, nyq = influence(lengths, mesh, order, alpha, printed_form)
    s2 = (s * np.conj(s)).real
    energy = KE * float((gopt * s2).sum())
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(k2 > 0, 2.0 / (4 * alpha * alpha) + 2.0 / k2, 0.0)
    virial = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            bab = (1.0 if a == b else 0.0) - fac * k[a] * k[b]
            virial[a, b] = KE * float((gopt * s2 * bab).sum())
    sg = s * gopt
    phi_mesh = (np.fft.ifftn(sg) * ntot).real.ravel()
    fields = []
    for d in range(3):
        comp = 1j * k[d] * sg
        comp[nyq[d]] = 0.0
        fields.append((np.fft.ifftn(comp) * ntot).real.ravel())
    phi = np.zeros(len(pos))
    force = np.zeros((len(pos), 3))
    for a0 in range(0, len(pos), chunk):
        pts, w = _gather_weights(pos[a0:a0 + chunk], lengths, mesh, order)
        flat, wt = _flat_stencil(pts, w, mesh)
        phi[a0:a0 + chunk] = 2.0 * KE * (wt * phi_mesh[flat]).sum(1)
        for d in range(3):
            force[a0:a0 + chunk, d] = -2.0 * KE * q[a0:a0 + chunk] * (wt * fields[d][flat]).sum(1)
    return {"e_kspace": energy, "phi": phi, "force": force, "virial": virial, "rho": rho}


def pppm_general(pos: np.ndarray, box: np.ndarray, q: np.ndarray, mesh, order: int, alpha: float,
                 printed_form: bool = False, chunk: int = 65536) -> dict:
    """PPPM in a general cell (rows of box the lattice vectors), the conventions of the module
    docstring: fractional mesh, k = 2 pi H^-1 n, fractional gradients mapped by H^-1."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    box = np.asarray(box, np.float64)
    hinv = np.linalg.inv(box)
    lengths = np.linalg.norm(box, axis=1)
    mesh = tuple(int(m) for m in mesh)
    ntot = int(np.prod(mesh))
    rho = np.zeros(ntot)
    for a0 in range(0, len(pos), chunk):
        pts, w = _gather_weights(pos[a0:a0 + chunk], lengths, mesh, order, hinv)
        flat, wt = _flat_stencil(pts, w, mesh)
        np.add.at(rho, flat.ravel(), (wt * q[a0:a0 + chunk, None]).ravel())
    rho = rho.reshape(mesh)
    s = np.fft.fftn(rho)
    gopt, k, k2, nyq, n = influence(lengths, mesh, order, alpha, printed_form, box=box)
    s2 = (s * np.conj(s)).real
    energy = KE * float((gopt * s2).sum())
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(k2 > 0, 2.0 / (4 * alpha * alpha) + 2.0 / k2, 0.0)
    virial = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            bab = (1.0 if a == b else 0.0) - fac * k[a] * k[b]
            virial[a, b] = KE * float((gopt * s2 * bab).sum())
    sg = s * gopt
    phi_mesh = (np.fft.ifftn(sg) * ntot).real.ravel()
    frac_fields = []
    for c in range(3):
        comp = 1j * (2.0 * math.pi * n[c]) * sg
        comp[nyq[c]] = 0.0
        frac_fields.append((np.fft.ifftn(comp) * ntot).real.ravel())
    phi = np.zeros(len(pos))
    force = np.zeros((len(pos), 3))
    for a0 in range(0, len(pos), chunk):
        pts, w = _gather_weights(pos[a0:a0 + chunk], lengths, mesh, order, hinv)
        flat, wt = _flat_stencil(pts, w, mesh)
        phi[a0:a0 + chunk] = 2.0 * KE * (wt * phi_mesh[flat]).sum(1)
        gf = np.stack([(wt * frac_fields[c][flat]).sum(1) for c in range(3)], -1)   # d/ds_c
        grad = gf @ hinv.T                                                            # d/dr_a
        force[a0:a0 + chunk] = -2.0 * KE * q[a0:a0 + chunk, None] * grad
    return {"e_kspace": energy, "phi": phi, "force": force, "virial": virial, "rho": rho}
