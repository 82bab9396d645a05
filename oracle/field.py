"""Response to an external electric field from the Born effective charges (oracle, float64).

Test infrastructure only (see the package docstring).

Sec. II.D gives two uses of the Born effective charges Z_i,ab = dP_a/dr_ib:
  Eq. (electric_force):          F^ext_i,b = sum_a E_a Z_i,ab
      the force on ion i from a uniform external field E (V/A, so F is in eV/A
      when Z is in e);
  Eq. (polarization_derivative): Pdot_a = sum_i sum_b Z_i,ab v_i,b
      the time derivative of the polarization along a trajectory with atomic
      velocities v (the ionic current; e A per unit of time of v).
Both are plain contractions, written here with one einsum each.  The first
index of Z is the polarization component a, the second the position component b.

Pins (tests/test_oracle_field.py): for a cluster, where P = sum_i q~^c_i r_i is
well defined, F^ext equals the central finite difference of E . P(r) with
respect to r_i and Pdot equals that of P(r + t v) in t, with Z the jacobian of
P; for a periodic structure with the charges constrained to Q, sum_i F^ext_i = Q E
and a uniform velocity v gives Pdot = Q v (acoustic sum rule of Eq. bec_2); and
sum_i F^ext_i . v_i = E . Pdot for any Z.
"""
from __future__ import annotations

import numpy as np


def electric_force(bec: np.ndarray, efield) -> np.ndarray:
    """F^ext [N, 3] of Eq. (electric_force): F_i,b = sum_a E_a Z_i,ab."""
    z = np.asarray(bec, dtype=np.float64).reshape(-1, 3, 3)
    e = np.asarray(efield, dtype=np.float64).reshape(3)
    return np.einsum("a,iab->ib", e, z)


def polarization_current(bec: np.ndarray, velocities: np.ndarray) -> np.ndarray:
    """Pdot [3] of Eq. (polarization_derivative): Pdot_a = sum_i sum_b Z_i,ab v_i,b."""
    z = np.asarray(bec, dtype=np.float64).reshape(-1, 3, 3)
    v = np.asarray(velocities, dtype=np.float64).reshape(-1, 3)
    return np.einsum("iab,ib->a", z, v)
