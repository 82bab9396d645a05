"""FP64 CPU oracle for the qNEP force call (test infrastructure only).

This package is the checker, not the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path
(``paper_2601_19034_gb300``): both only read the seeded inputs from
``paper_2601_19034_gb300.workloads``, which holds none of the method.

Everything is plain float64 (numpy / torch CPU).  Derivatives are taken with
torch autograd of the energy as written in the paper, never with the paper's
hand-derived partial-force formulas (those are what the CUDA path follows);
the PPPM static force is the one exception, because the paper defines it by the
ik-differentiation scheme rather than as an energy gradient.

Modules
  geometry    neighbour entries with periodic images (explicit enumeration)
  descriptor  NEP radial / angular / 4-body descriptor (reading of Sec. II.A)
  network     two-output network, Eq. (U_i) plus the charge node (Sec. II.B)
  ewald       real-space, reciprocal-space (direct k sum) and self energies
  pppm        PPPM mesh energy, potential and ik-differentiated force (Sec. II.F)
  forcecall   the full force call: energy, forces, virial, charges, BEC, P
  field       external-field force and polarization current from the BEC (Sec. II.D)
  training    population loss terms of Sec. II.E and the SNES update it drives
  virial      per-atom virial of Eq. per-atom_virial (Ewald and PPPM)
  md          velocity-Verlet NVE steps around a force call (the 0.5 fs runs of Sec. III)
  params      unpacking of the documented parameter blob

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, library routines, brute force or finite differences; the
absolute values of the descriptor are fixed only by the reading of Sec. II.A
the oracle and the CUDA path share (the paper defers the definition to its
references), which the tests pin by invariances and independent forms.
"""
