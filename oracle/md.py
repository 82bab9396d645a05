"""Velocity-Verlet NVE integration around a force call (oracle, float64).

Test infrastructure only (see the package docstring).

The paper runs its molecular dynamics with a time step of 0.5 fs (Sec. III, the speed
comparison of the water models) and does not print the integrator.  The NVE integrator taken
here is velocity Verlet (Swope, Andersen, Berens and Wilson, J. Chem. Phys. 76, 637 (1982)):
with a_i = F_i / m_i,
    x(t + h) = x(t) + h v(t) + h^2 / 2 a(t),
    v(t + h) = v(t) + h / 2 (a(t) + a(t + h)),
the forces a(t + h) taken at the new positions.  Units are those of the force call: positions in
A, time in fs, masses in amu (daltons), energies in eV, forces in eV/A.  The two conversions follow
from the SI definitions: 1 eV = 1.602176634e-19 J (exact), 1 Da = 1.66053906660e-27 kg (CODATA
2018), 1 A = 1e-10 m, 1 fs = 1e-15 s, so
    (eV/A)/amu = (e / m_u) 1e-10 A/fs^2     (ACC_UNIT, ~9.6485e-3),
    amu A^2/fs^2 = (m_u / e) 1e10 eV       (KE_UNIT, ~103.64),
and ACC_UNIT * KE_UNIT = 1 (energy = force x length).

Pins (tests/test_oracle_md.py): for one atom in a harmonic well the map has the exact solution
    x_n = x_0 cos(n theta) + D sin(n theta),   cos theta = 1 - (omega h)^2 / 2,   D = h v_0 / sin theta,
    v_n = (x_{n+1} - x_{n-1}) / 2h = (sin theta / h) (D cos(n theta) - x_0 sin(n theta));
running n steps, reversing the velocities and running n more steps returns to the start; the
total energy error of a smooth many-body potential falls as h^2; the two unit conversions are
inverse to each other.
"""
from __future__ import annotations

import numpy as np

E_CHARGE = 1.602176634e-19       # C: 1 eV = E_CHARGE J
DALTON = 1.66053906660e-27       # kg
ACC_UNIT = E_CHARGE / DALTON * 1e-10     # (eV/A)/amu in A/fs^2
KE_UNIT = DALTON / E_CHARGE * 1e10       # amu A^2/fs^2 in eV


def acceleration(forces, masses):
    """a_i = F_i / m_i in A/fs^2 for forces [N, 3] (eV/A) and masses [N] (amu)."""
    f = np.asarray(forces, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(masses, dtype=np.float64).reshape(-1)
    return f * (ACC_UNIT / m)[:, None]


def kinetic_energy(velocities, masses) -> float:
    """K = 1/2 sum_i m_i |v_i|^2 in eV for velocities in A/fs."""
    v = np.asarray(velocities, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(masses, dtype=np.float64).reshape(-1)
    return float(0.5 * KE_UNIT * (m[:, None] * v * v).sum())


def positions_after_step(x, v, f, masses, h):
    """x(t + h) = x + h v + h^2 / 2 a(t)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    return x + h * v + 0.5 * h * h * acceleration(f, masses)


def velocities_after_step(v, f_old, f_new, masses, h):
    """v(t + h) = v + h / 2 (a(t) + a(t + h))."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    return v + 0.5 * h * (acceleration(f_old, masses) + acceleration(f_new, masses))


def step(x, v, f, masses, h, forces_of):
    """One step; forces_of(x) -> (U, F) is the force call.  Returns (x, v, F, U) at t + h."""
    x1 = positions_after_step(x, v, f, masses, h)
    u1, f1 = forces_of(x1)
    v1 = velocities_after_step(v, f, f1, masses, h)
    return x1, v1, np.asarray(f1, dtype=np.float64).reshape(-1, 3), float(u1)


def run(x, v, masses, h, n_steps, forces_of):
    """n_steps steps from (x, v).  Returns the final (x, v, F) and energies [n_steps + 1, 2] holding
    (U, K) of the initial state and after every step, the layout of the NVE entry point."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    u, f = forces_of(x)
    f = np.asarray(f, dtype=np.float64).reshape(-1, 3)
    energies = np.zeros((n_steps + 1, 2))
    energies[0] = (float(u), kinetic_energy(v, masses))
    for k in range(n_steps):
        x, v, f, u = step(x, v, f, masses, h, forces_of)
        energies[k + 1] = (u, kinetic_energy(v, masses))
    return x, v, f, energies
