"""Seeded synthetic inputs: molecular boxes, velocities and the sp tight-binding model data.

This module produces inputs only.  It holds none of the method's arithmetic
(no Hamiltonian, no Coulomb sum, no graph, no density matrix), so both the
FP64 oracle and the CUDA path may draw their inputs from it.

Workloads stand in for the paper's LATTE water boxes (2,955 / 30,840 / 2,088
atoms, Sec. "Accuracy Control via Graph Thresholding" and "Scalability") and
for a liquid methanol/water mixture:

* molecules sit on the sites of an fcc lattice with m = ceil((N_mol/4)^(1/3))
  cells per box edge; when N_mol < 4 m^3 a seeded subset of sites is used;
* every molecule centre gets a uniform +-0.2 A jitter per axis and a uniform
  (Haar) orientation drawn from a normalised Gaussian quaternion;
* an orientation is redrawn (up to 100 times) while any intermolecular atom
  pair is closer than 1.2 A (minimum image);
* water: O-H 0.96 A, H-O-H 104.5 deg; methanol: C-O 1.43, O-H 0.96, C-H 1.09 A,
  tetrahedral carbon, C-O-H 108.5 deg.

Units: positions in Angstrom, velocities in Angstrom/fs, masses in amu.
Species codes: 0 = H, 1 = C, 2 = O.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

H, C, O = 0, 1, 2
SPECIES_NAMES = ("H", "C", "O")

# --------------------------------------------------------------------------------------
# Model data of the synthetic sp Slater-Koster SCC tight-binding model.
# Energies in Hartree, lengths in Angstrom.  The same numbers go to both sides as input.
# --------------------------------------------------------------------------------------


@dataclass(frozen=True)
class SKModel:
    """Constants of the synthetic sp SCC-TB model (input data, no arithmetic).

    Hopping radial functions are V_X(r) = V0_X * exp(-r / decay) * sw(r) for
    X in (ss sigma, sp sigma, pp sigma, pp pi), with sw the quintic switch from
    ``r_on`` to ``r_off``.  The overlap uses the same form with every V0
    multiplied by ``overlap_scale``.  ``v0`` is indexed [species_i, species_j, X]
    where, for sp sigma, species_i carries the s orbital and species_j the p.
    Repulsion: A_ij * exp(-r / rep_decay) * sw(r).
    """

    n_orb: tuple = (1, 4, 4)                 # H: s ; C, O: s px py pz
    eps_s: tuple = (-0.24, -0.50, -0.88)     # on-site s energies
    eps_p: tuple = (0.0, -0.19, -0.33)       # on-site p energies (unused for H)
    hubbard_u: tuple = (0.40, 0.36, 0.50)    # Hubbard U (Ha)
    z_val: tuple = (1.0, 4.0, 6.0)           # valence electrons
    mass: tuple = (1.008, 12.011, 15.999)    # amu
    v0: tuple = field(default_factory=lambda: tuple(
        tuple((-1.5, 1.8, 1.6, -0.6) for _ in range(3)) for _ in range(3)))
    decay: float = 0.6                       # A
    overlap_scale: float = -0.1              # S = overlap_scale * V / (1 Ha)
    r_on: float = 5.0                        # A, switch start
    r_off: float = 6.0                       # A, switch end (pair cutoff r_hs)
    rep_a: tuple = field(default_factory=lambda: tuple(tuple(0.0 for _ in range(3)) for _ in range(3)))
    rep_decay: float = 0.3                   # A

    def v0_array(self) -> np.ndarray:
        return np.asarray(self.v0, dtype=np.float64)

    def rep_array(self) -> np.ndarray:
        return np.asarray(self.rep_a, dtype=np.float64)


def default_model() -> SKModel:
    """The model with the repulsive amplitudes fitted once by ``oracle/fit_repulsion.py``.

    The amplitudes make an isolated water molecule force-free at its input geometry
    (O-H 0.96 A, 104.5 deg), so dynamics keeps its bonds.  The fitted numbers are
    stored in ``oracle/repulsion_fit.json``; they are model data like the V0 table.
    """
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "oracle", "repulsion_fit.json")
    rep = [[0.0] * 3 for _ in range(3)]
    if os.path.exists(path):
        with open(path) as fh:
            fit = json.load(fh)
        for key, val in fit["A"].items():
            a, b = (SPECIES_NAMES.index(s) for s in key.split("-"))
            rep[a][b] = rep[b][a] = float(val)
    return SKModel(rep_a=tuple(tuple(r) for r in rep))


# --------------------------------------------------------------------------------------
# Molecule templates (body frame, Angstrom)
# --------------------------------------------------------------------------------------

def _water_template() -> tuple[np.ndarray, np.ndarray]:
    half = math.radians(104.5) / 2.0
    r = 0.96
    pos = np.array([[0.0, 0.0, 0.0],
                    [r * math.sin(half), 0.0, r * math.cos(half)],
                    [-r * math.sin(half), 0.0, r * math.cos(half)]])
    return np.array([O, H, H], dtype=np.int32), pos


def _methanol_template() -> tuple[np.ndarray, np.ndarray]:
    # C at origin, O along +z; three H on C tetrahedral; hydroxyl H in the xz plane.
    r_co, r_oh, r_ch = 1.43, 0.96, 1.09
    tet = math.acos(-1.0 / 3.0)            # 109.47 deg
    c = np.zeros(3)
    o = np.array([0.0, 0.0, r_co])
    hs = []
    for k in range(3):
        phi = 2.0 * math.pi * k / 3.0
        hs.append(r_ch * np.array([math.sin(tet) * math.cos(phi), math.sin(tet) * math.sin(phi), math.cos(tet)]))
    ang = math.radians(108.5)              # C-O-H angle
    # direction from O making angle `ang` with O->C (which is -z), in the xz plane, anti to H0
    ho = o + r_oh * np.array([-math.sin(math.pi - ang), 0.0, math.cos(math.pi - ang)])
    pos = np.vstack([c, o, hs[0], hs[1], hs[2], ho])
    return np.array([C, O, H, H, H, H], dtype=np.int32), pos


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class System:
    """A periodic orthorhombic box of atoms (input data)."""

    species: np.ndarray          # int32 [N]
    R: np.ndarray                # float64 [N, 3], Angstrom
    box: np.ndarray              # float64 [3], Angstrom
    mol_ptr: np.ndarray          # int64 [n_mol + 1], atom ranges per molecule
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.species.shape[0])


def molecular_box(n_water: int, n_methanol: int, box_len: float, seed: int, name: str = "") -> System:
    """Seeded fcc-lattice box of rigid water / methanol molecules (see module docstring)."""
    rng = np.random.default_rng(seed)
    n_mol = n_water + n_methanol
    m = int(math.ceil((n_mol / 4.0) ** (1.0 / 3.0) - 1e-12))
    a = box_len / m
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.array([[i, j, k] for i in range(m) for j in range(m) for k in range(m)], dtype=np.float64)
    sites = ((cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) + 0.25) * a
    if n_mol < sites.shape[0]:
        pick = np.sort(rng.choice(sites.shape[0], size=n_mol, replace=False))
        sites = sites[pick]
    kinds = np.array([1] * n_methanol + [0] * n_water)
    rng.shuffle(kinds)
    templates = {0: _water_template(), 1: _methanol_template()}
    box = np.array([box_len] * 3, dtype=np.float64)

    species, coords, ptr = [], [], [0]
    placed = np.zeros((0, 3))
    for im in range(n_mol):
        sp, body = templates[int(kinds[im])]
        body = body - body.mean(axis=0)
        centre = sites[im] + rng.uniform(-0.2, 0.2, size=3)
        for _ in range(100):
            xyz = centre + body @ _random_rotation(rng).T
            if placed.shape[0] == 0:
                break
            d = xyz[:, None, :] - placed[None, :, :]
            d -= box * np.round(d / box)
            if np.min(np.einsum("ijk,ijk->ij", d, d)) >= 1.2 * 1.2:
                break
        species.append(sp)
        coords.append(xyz)
        placed = np.vstack([placed, xyz])
        ptr.append(ptr[-1] + len(sp))
    return System(species=np.concatenate(species).astype(np.int32),
                  R=np.vstack(coords).astype(np.float64), box=box,
                  mol_ptr=np.asarray(ptr, dtype=np.int64), name=name)


# Named workloads (seed 20260603 + k for workload k).
WORKLOADS = {
    "water96": dict(n_water=32, n_methanol=0, box_len=9.86, seed=20260604),
    "water9000": dict(n_water=3000, n_methanol=0, box_len=44.8, seed=20260605),
    "mix9999": dict(n_water=1111, n_methanol=1111, box_len=46.82, seed=20260606),
    "water30000": dict(n_water=10000, n_methanol=0, box_len=67.2, seed=20260608),
}


def workload(name: str) -> System:
    kw = WORKLOADS[name]
    return molecular_box(name=name, **kw)


def small_water_box(n_water: int, box_len: float, seed: int) -> System:
    return molecular_box(n_water, 0, box_len, seed, name=f"water{3 * n_water}")


def maxwell_boltzmann(species: np.ndarray, temperature_k: float, seed: int, model: SKModel | None = None) -> np.ndarray:
    """Seeded Maxwell-Boltzmann velocities (A/fs), COM momentum removed, rescaled to exactly T over 3N-3 dof."""
    model = model or SKModel()
    rng = np.random.default_rng(seed)
    m = np.asarray(model.mass, dtype=np.float64)[species]              # amu
    kb_ev = 8.617333262e-5                                             # eV/K
    amu_a2_fs2_to_ev = 103.642696562                                   # 1 amu A^2/fs^2 in eV
    kt = kb_ev * temperature_k / amu_a2_fs2_to_ev                      # amu A^2/fs^2
    v = rng.standard_normal((species.shape[0], 3)) * np.sqrt(kt / m)[:, None]
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    ekin = 0.5 * np.sum(m[:, None] * v * v)
    dof = 3 * species.shape[0] - 3
    v *= math.sqrt(0.5 * dof * kt / ekin)
    return v


def random_charges(n_atoms: int, seed: int, scale: float = 0.05) -> np.ndarray:
    """Seeded zero-sum charge vector (e), used as the trial density n in tests."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n_atoms) * scale
    return x - x.mean()
