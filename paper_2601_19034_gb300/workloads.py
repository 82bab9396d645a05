"""Seeded synthetic inputs shaped like the paper's systems (Sec. III).

This module only builds inputs: atomic positions, species, boxes and randomly
drawn model parameters.  It holds none of the qNEP arithmetic (no descriptor,
network, electrostatics or derivative), so both the CUDA path and the FP64
oracle may import it without sharing any of the method.

Units: Angstrom, e, eV, amu, fs.  Boxes are row-vector matrices (rows are the
lattice vectors a, b, c); every box generated here is orthorhombic.

The parameter blob layout (one candidate) is the documented interface of
``qnep_create`` in ``include/qnep.h``; each side unpacks it with its own code.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Species lists used by the synthetic systems (order = type index).
WATER_SPECIES = ("O", "H")
BATIO3_SPECIES = ("Ba", "Ti", "O")
LLZO_SPECIES = ("Li", "La", "Zr", "O")
MGWATER_SPECIES = ("Mg", "O", "H")
MASSES = {"H": 1.008, "O": 15.999, "Mg": 24.305, "Li": 6.94, "La": 138.905, "Zr": 91.224, "Ba": 137.327,
          "Ti": 47.867}   # amu

AVOGADRO = 6.02214076e23

# Atom count of the field-response measurement (Born effective charges [N][3][3],
# velocities and forces [N][3], float32: 252 MB, above the 129 MB L2 of the GPU).
FIELD_RESPONSE_ATOMS = 4_194_304
M_H2O = 18.01528  # g/mol


@dataclasses.dataclass
class HParams:
    """Descriptor / network sizes (defaults: the paper's water-type model).

    n_radial / n_angular are the numbers of radial functions g_n (n_max + 1);
    basis_radial / basis_angular are the numbers of Chebyshev terms
    (basis size + 1).
    """
    n_species: int
    rc_radial: float = 6.0
    rc_angular: float = 4.0
    n_radial: int = 5
    n_angular: int = 5
    basis_radial: int = 9
    basis_angular: int = 9
    l_max: int = 4
    use_4body: int = 1
    n_neurons: int = 30

    @property
    def n_des(self) -> int:
        return self.n_radial + self.n_angular * self.l_max + (self.n_angular if self.use_4body else 0)

    @property
    def n_params(self) -> int:
        s = self.n_species
        return (s * s * (self.n_radial * self.basis_radial + self.n_angular * self.basis_angular)
                + self.n_des + s * (self.n_neurons * (self.n_des + 3) + 2) + 1)


@dataclasses.dataclass
class Elec:
    """Electrostatics settings. mode 1: real + k + self, mode 2: k only.

    kind: "ewald" or "pppm".  kmax is the strict Ewald wave-vector cutoff;
    mesh/order are the PPPM mesh and assignment order.
    """
    mode: int = 1
    kind: str = "ewald"
    alpha: float = 0.3
    rc_real: float = 6.0
    kmax: float = 2.0 * 0.3 * math.sqrt(math.log(1e6))
    mesh: tuple = (0, 0, 0)
    order: int = 5
    q_total: float = 0.0


@dataclasses.dataclass
class System:
    positions: np.ndarray   # (N, 3) float32
    types: np.ndarray       # (N,) int32
    box: np.ndarray         # (3, 3) float64, rows = lattice vectors
    species: tuple

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def random_params(hp: HParams, rng: np.random.Generator, sigma: float = 0.1,
                  sqrt_eps_inf: float = 1.53, n_candidates: int = 1) -> np.ndarray:
    """Draw candidate-major parameter blobs, every entry N(0, sigma).

    The descriptor scaler is fixed to 1 and sqrt(eps_inf) to ``sqrt_eps_inf``
    (the water mode-2 value of Sec. III.A).  Returns float32 [n_candidates, n_params].
    """
    out = rng.normal(0.0, sigma, size=(n_candidates, hp.n_params)).astype(np.float32)
    s = hp.n_species
    off_scaler = s * s * (hp.n_radial * hp.basis_radial + hp.n_angular * hp.basis_angular)
    out[:, off_scaler:off_scaler + hp.n_des] = 1.0
    out[:, -1] = sqrt_eps_inf
    return out


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform SO(3) rotations from normalised Gaussian quaternions."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _water_molecules(rng, centres: np.ndarray) -> np.ndarray:
    """Rigid H2O (O-H 0.96 A, 104.5 deg), random orientation, O at each centre."""
    half = math.radians(104.5) / 2.0
    ref = np.array([[0.0, 0.0, 0.0],
                     [0.96 * math.sin(half), 0.0, 0.96 * math.cos(half)],
                     [-0.96 * math.sin(half), 0.0, 0.96 * math.cos(half)]])
    rot = _random_rotations(rng, len(centres))
    return (centres[:, None, :] + np.einsum("mab,kb->mka", rot, ref)).reshape(-1, 3)


def water_box(n_side: int, length: float | None = None, jitter: float = 0.1,
              seed: int = 1000) -> System:
    """n_side^3 rigid waters on a grid in a cube at 1.0 g/cm^3, per-atom N(0, jitter)."""
    rng = np.random.default_rng(seed)
    n_mol = n_side ** 3
    if length is None:
        length = (n_mol * M_H2O / AVOGADRO / 1.0 * 1e24) ** (1.0 / 3.0)
    g = (np.arange(n_side) + 0.5) * (length / n_side)
    centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = _water_molecules(rng, centres)
    pos += rng.normal(0.0, jitter, size=pos.shape)
    pos %= length
    types = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    return System(pos.astype(np.float32), types, np.diag([length] * 3).astype(np.float64),
                  WATER_SPECIES)


def batio3_supercell(n: int, a: float = 4.0, sigma: float = 0.05, seed: int = 1001) -> System:
    """Cubic perovskite BaTiO3 n x n x n supercell with N(0, sigma) displacements."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0.5], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    btypes = np.array([0, 1, 2, 2, 2], np.int32)
    cells = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)
    pos += rng.normal(0.0, sigma, size=pos.shape)
    pos %= n * a
    types = np.tile(btypes, len(cells))
    return System(pos.astype(np.float32), types, np.diag([n * a] * 3).astype(np.float64),
                  BATIO3_SPECIES)


def llzo_base_cell(a: float = 12.97, seed: int = 1003, min_sep: float = 1.5) -> System:
    """Random 192-atom Li56 La24 Zr16 O96 cell (rejection sampling, min separation)."""
    rng = np.random.default_rng(seed)
    counts = (56, 24, 16, 96)
    types = np.concatenate([np.full(c, t, np.int32) for t, c in enumerate(counts)])
    pos = np.zeros((len(types), 3))
    k = 0
    while k < len(types):
        p = rng.uniform(0.0, a, size=3)
        if k:
            d = pos[:k] - p
            d -= a * np.round(d / a)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        pos[k] = p
        k += 1
    return System(pos.astype(np.float32), types, np.diag([a] * 3), LLZO_SPECIES)


def llzo_batch(n_struct: int = 512, a: float = 12.97, sigma: float = 0.1,
               seed: int = 1003) -> list:
    """Supercells n1 x n2 x n3 (n in {1, 2}) of the random LLZO cell, N(0, sigma) moves."""
    base = llzo_base_cell(a, seed)
    rng = np.random.default_rng(seed + 7)
    out = []
    for _ in range(n_struct):
        reps = rng.integers(1, 3, size=3)
        shifts = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
        pos = (base.positions[None].astype(np.float64) + shifts[:, None, :] * a).reshape(-1, 3)
        pos += rng.normal(0.0, sigma, size=pos.shape)
        lengths = reps * a
        pos %= lengths
        types = np.tile(base.types, len(shifts))
        out.append(System(pos.astype(np.float32), types, np.diag(lengths.astype(np.float64)),
                          LLZO_SPECIES))
    return out


def mg_water_interface(nx: int = 112, ny: int = 65, n_layers: int = 15, water_thickness: float = 60.0,
                       gap: float = 1.5, a: float = 3.21, c: float = 5.21, seed: int = 1004) -> System:
    """hcp Mg slab ((0001) normal to z) under a water layer at 1.0 g/cm^3.

    Orthohexagonal lateral cell nx*a by ny*sqrt(3)*a; periodic in all three
    directions with the water layer on top of the slab.
    """
    rng = np.random.default_rng(seed)
    lx, ly = nx * a, ny * math.sqrt(3.0) * a
    # orthohexagonal 4-atom cell: A layer (0,0),(1/2,1/2); B layer (1/2,1/6),(0,2/3)
    ortho_b = math.sqrt(3.0) * a
    la = np.array([[0.0, 0.0], [0.5, 0.5]])
    lb = np.array([[0.5, 1.0 / 6.0], [0.0, 2.0 / 3.0]])
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel()], -1).astype(np.float64)
    mg = []
    for layer in range(n_layers):
        frac = la if layer % 2 == 0 else lb
        xy = ((cells[:, None, :] + frac[None]) * np.array([a, ortho_b])).reshape(-1, 2)
        z = np.full((len(xy), 1), layer * c / 2.0)
        mg.append(np.concatenate([xy, z], 1))
    mg = np.concatenate(mg)
    slab_top = (n_layers - 1) * c / 2.0
    z0 = slab_top + gap + 1.0
    n_mol_target = int(round(lx * ly * water_thickness * 1.0 / M_H2O * AVOGADRO * 1e-24))
    spacing = (lx * ly * water_thickness / n_mol_target) ** (1.0 / 3.0)
    gx = int(lx / spacing); gy = int(ly / spacing); gz = int(math.ceil(n_mol_target / (gx * gy)))
    centres = np.stack(np.meshgrid((np.arange(gx) + 0.5) * lx / gx, (np.arange(gy) + 0.5) * ly / gy,
                                   z0 + (np.arange(gz) + 0.5) * water_thickness / gz, indexing="ij"),
                       -1).reshape(-1, 3)[:n_mol_target]
    water = _water_molecules(rng, centres)
    water += rng.normal(0.0, 0.05, size=water.shape)
    lz = z0 + water_thickness + gap
    pos = np.concatenate([mg, water])
    pos %= np.array([lx, ly, lz])
    types = np.concatenate([np.zeros(len(mg), np.int32), np.tile(np.array([1, 2, 2], np.int32), len(centres))])
    return System(pos.astype(np.float32), types, np.diag([lx, ly, lz]), MGWATER_SPECIES)


def maxwell_boltzmann(masses: np.ndarray, temperature: float, seed: int = 1005) -> np.ndarray:
    """Velocities (A/fs) from a Maxwell-Boltzmann distribution with zero total momentum.

    1 amu A^2 fs^-2 = 103.6427 eV, so sigma_v = sqrt(k_B T / (103.6427 m)).
    """
    kb = 8.617333262e-5  # eV/K
    rng = np.random.default_rng(seed)
    sig = np.sqrt(kb * temperature / (103.6427 * masses))
    v = rng.normal(size=(len(masses), 3)) * sig[:, None]
    v -= (masses[:, None] * v).sum(0) / masses.sum()
    return v


# --- the five benchmark configurations -------------------------------------------------

def config_water_small(seed: int = 1000):
    """64 H2O (192 atoms), 12.42 A box, Ewald alpha 0.3, mode 1."""
    sysm = water_box(4, length=12.42, seed=seed)
    hp = HParams(n_species=2)
    params = random_params(hp, np.random.default_rng(seed + 100))
    return sysm, hp, params[0], Elec(mode=1, kind="ewald")


def config_batio3(seed: int = 1001, n: int = 10):
    """BaTiO3 n^3 perovskite cells (5 n^3 atoms), Ewald alpha 0.3, mode 1."""
    sysm = batio3_supercell(n, seed=seed)
    hp = HParams(n_species=3)
    params = random_params(hp, np.random.default_rng(seed + 100))
    return sysm, hp, params[0], Elec(mode=1, kind="ewald")


def config_water_pppm(seed: int = 1002, n_side: int = 20, mesh: int = 64):
    """n_side^3 H2O at 1.0 g/cm^3 with PPPM (mesh^3, order 5, alpha 0.3)."""
    sysm = water_box(n_side, seed=seed)
    hp = HParams(n_species=2)
    params = random_params(hp, np.random.default_rng(seed + 100))
    return sysm, hp, params[0], Elec(mode=1, kind="pppm", mesh=(mesh, mesh, mesh), order=5)


def config_llzo_batch(seed: int = 1003, n_struct: int = 512, n_candidates: int = 64):
    """512 LLZO-shaped cells x 64 candidate parameter vectors, Ewald per cell."""
    systems = llzo_batch(n_struct, seed=seed)
    hp = HParams(n_species=4)
    params = random_params(hp, np.random.default_rng(seed + 100), n_candidates=n_candidates)
    return systems, hp, params, Elec(mode=1, kind="ewald")


def scale_charge_head(params: np.ndarray, hp: HParams, factor: float) -> np.ndarray:
    """Multiply the charge output layer (w1_q and b1_q of every species) by ``factor``."""
    p = np.array(params, dtype=np.float32, copy=True)
    s = hp.n_species
    mlp = s * s * (hp.n_radial * hp.basis_radial + hp.n_angular * hp.basis_angular) + hp.n_des
    block = hp.n_neurons * hp.n_des + 3 * hp.n_neurons + 2
    for t in range(s):
        w1q = mlp + t * block + hp.n_neurons * hp.n_des + 2 * hp.n_neurons
        p[..., w1q:w1q + hp.n_neurons] *= factor
        p[..., mlp + t * block + block - 1] *= factor        # b1_q
    return p


def config_mg_water(seed: int = 1004, nx: int = 112, ny: int = 65, mesh=(256, 256, 384)):
    """Mg-water interface (~1.0 M atoms at the default size), PPPM, mode 1, 3 species.

    Weights N(0, 0.1) except the charge output layer, N(0, 0.01): with a full-size random
    charge head the per-species offsets charge the slab against the water layer (about
    100 V/A across the interface) and the NVE run is not integrable at 0.5 fs.
    """
    sysm = mg_water_interface(nx, ny, seed=seed)
    hp = HParams(n_species=3)
    params = scale_charge_head(random_params(hp, np.random.default_rng(seed + 100)), hp, 0.1)
    return sysm, hp, params[0], Elec(mode=1, kind="pppm", mesh=tuple(mesh), order=5)


def species_masses(species) -> np.ndarray:
    return np.array([MASSES[s] for s in species], dtype=np.float64)
