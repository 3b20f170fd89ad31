"""Seeded synthetic inputs for the NEP3 energy/force/virial path (arXiv:2205.10046).

This module only generates inputs: crystal lattices and supercells, Gaussian position
jitter, random model weights and Maxwell-Boltzmann velocities. It holds none of the
NEP arithmetic (no descriptor, network, force or integrator code), so both the CUDA
path and the FP64 oracle can consume the same arrays without sharing any method code.

Conventions (all FP64 numpy arrays):
  * positions ``pos`` [N, 3] in Angstrom, cell ``box`` [3, 3] whose ROWS are the cell
    vectors a, b, c (a position is r = s @ box for fractional s in [0, 1)^3);
  * ``types`` [N] int32 in [0, n_types);
  * model weights follow the ordering of Sec. II of the paper: c_radial[t_i][t_j][n][k]
    (ordered type pair, Eq. g_n), c_angular likewise, w0[mu][nu] neuron-major (Eq. Ui,
    the neuron-major layout of Appendix B), b0[mu], w1[mu], scalar b1.

Random draws: one numpy PCG64 stream per purpose. The model uses the workload seed;
displacements use seed + 1000 and velocities seed + 2000. Weights are drawn in the order
c_radial, c_angular, w0, b0, w1, b1, each U(-1, 1) / sqrt(fan_in) with fan_in = K_R + 1
(c_radial), K_A + 1 (c_angular), N_des (w0, b0) and N_neu (w1, b1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Unit conventions (Angstrom, fs, eV, atomic mass unit, K): CODATA 2018 exact/recommended.
_EV_J = 1.602176634e-19
_AMU_KG = 1.66053906660e-27
#: 1 u * Angstrom^2 / fs^2 expressed in eV (about 103.6427).
AMU_A2_PER_FS2_IN_EV = _AMU_KG * 1e-20 / 1e-30 / _EV_J
#: Boltzmann constant in eV/K.
KB_EV = 8.617333262e-5

MASS_SI = 28.085
MASS_PB = 207.2
MASS_TE = 127.60
MASS_GE = 72.630
MASS_C = 12.011


@dataclass
class NepModel:
    """Hyper-parameters and weights of one NEP3 model (the nep.in keywords of Sec. III)."""

    n_types: int
    rc_radial: float
    rc_angular: float
    n_max_radial: int
    n_max_angular: int
    basis_radial: int
    basis_angular: int
    l_max_3b: int
    l_max_4b: int
    l_max_5b: int
    n_neuron: int
    c_radial: np.ndarray = field(repr=False, default=None)
    c_angular: np.ndarray = field(repr=False, default=None)
    w0: np.ndarray = field(repr=False, default=None)
    b0: np.ndarray = field(repr=False, default=None)
    w1: np.ndarray = field(repr=False, default=None)
    b1: float = 0.0
    mass: np.ndarray = field(repr=False, default=None)

    @property
    def n_angular_blocks(self) -> int:
        """Blocks of (n_max_angular + 1) angular components: l = 1..l_max_3b, 4-body, 5-body."""
        return self.l_max_3b + (1 if self.l_max_4b >= 2 else 0) + (1 if self.l_max_5b >= 1 else 0)

    @property
    def n_des(self) -> int:
        """Descriptor length (the N_des enumeration at the end of Sec. II C)."""
        return (self.n_max_radial + 1) + (self.n_max_angular + 1) * self.n_angular_blocks

    @property
    def n_par(self) -> int:
        """Trainable parameter count N_par of NEP3 (Sec. II E)."""
        t2 = self.n_types ** 2
        return ((self.n_des + 2) * self.n_neuron + 1
                + t2 * (self.n_max_radial + 1) * (self.basis_radial + 1)
                + t2 * (self.n_max_angular + 1) * (self.basis_angular + 1))

    def hyper(self) -> dict:
        return dict(n_types=self.n_types, rc_radial=self.rc_radial, rc_angular=self.rc_angular,
                    n_max_radial=self.n_max_radial, n_max_angular=self.n_max_angular,
                    basis_radial=self.basis_radial, basis_angular=self.basis_angular,
                    l_max_3b=self.l_max_3b, l_max_4b=self.l_max_4b, l_max_5b=self.l_max_5b,
                    n_neuron=self.n_neuron)

    def to_vector(self) -> np.ndarray:
        """Flatten the trainable parameters in the draw order (c_R, c_A, w0, b0, w1, b1)."""
        return np.concatenate([self.c_radial.ravel(), self.c_angular.ravel(), self.w0.ravel(),
                               self.b0.ravel(), self.w1.ravel(), np.array([self.b1])])

    def with_vector(self, z) -> "NepModel":
        """A model with these hyper-parameters and masses and the parameters z (to_vector order)."""
        z = np.asarray(z, dtype=np.float64).reshape(-1)
        if z.shape[0] != self.n_par:
            raise ValueError(f"z has {z.shape[0]} values, N_par = {self.n_par}")
        T, nR, nA, KR, KA, H, D = (self.n_types, self.n_max_radial, self.n_max_angular, self.basis_radial,
                                   self.basis_angular, self.n_neuron, self.n_des)
        m = NepModel(**self.hyper())
        sizes = [T * T * (nR + 1) * (KR + 1), T * T * (nA + 1) * (KA + 1), H * D, H, H, 1]
        parts = np.split(z, np.cumsum(sizes)[:-1])
        m.c_radial = parts[0].reshape(T, T, nR + 1, KR + 1).copy()
        m.c_angular = parts[1].reshape(T, T, nA + 1, KA + 1).copy()
        m.w0 = parts[2].reshape(H, D).copy()
        m.b0 = parts[3].copy()
        m.w1 = parts[4].copy()
        m.b1 = float(parts[5][0])
        m.mass = None if self.mass is None else np.array(self.mass)
        return m


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_model(hyper: dict, seed: int, mass) -> NepModel:
    """Random NEP3 weights, U(-1, 1)/sqrt(fan_in), drawn from one PCG64(seed) stream."""
    m = NepModel(**hyper)
    rng = _rng(seed)
    T, nR, nA, KR, KA, H = (m.n_types, m.n_max_radial, m.n_max_angular, m.basis_radial,
                            m.basis_angular, m.n_neuron)
    D = m.n_des
    m.c_radial = rng.uniform(-1.0, 1.0, (T, T, nR + 1, KR + 1)) / math.sqrt(KR + 1)
    m.c_angular = rng.uniform(-1.0, 1.0, (T, T, nA + 1, KA + 1)) / math.sqrt(KA + 1)
    m.w0 = rng.uniform(-1.0, 1.0, (H, D)) / math.sqrt(D)
    m.b0 = rng.uniform(-1.0, 1.0, H) / math.sqrt(D)
    m.w1 = rng.uniform(-1.0, 1.0, H) / math.sqrt(H)
    m.b1 = float(rng.uniform(-1.0, 1.0) / math.sqrt(H))
    m.mass = np.asarray(mass, dtype=np.float64).reshape(T)
    return m


# --------------------------------------------------------------------------- lattices
_FCC = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
_BCC = np.array([[0, 0, 0], [.5, .5, .5]], dtype=np.float64)


def _basis(kind: str):
    """Fractional basis of a conventional cubic cell and the sublattice label of each site."""
    if kind == "diamond":
        return np.vstack([_FCC, _FCC + 0.25]), np.zeros(8, np.int32)
    if kind == "rocksalt":  # cation on the FCC sites, anion at +(1/2, 0, 0)
        return np.vstack([_FCC, _FCC + [0.5, 0, 0]]) % 1.0, np.r_[np.zeros(4), np.ones(4)].astype(np.int32)
    if kind == "fcc":
        return _FCC.copy(), np.zeros(4, np.int32)
    if kind == "bcc":
        return _BCC.copy(), np.zeros(2, np.int32)
    raise ValueError(kind)


def lattice(kind: str, a: float, reps) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Cubic supercell of ``reps`` = (nx, ny, nz) conventional cells.

    Atom index = ((ix * ny + iy) * nz + iz) * n_basis + b. Returns (pos, box, sublattice).
    """
    nx, ny, nz = reps
    frac, sub = _basis(kind)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + frac[None, :, :]).reshape(-1, 3) * a
    box = np.diag([nx * a, ny * a, nz * a]).astype(np.float64)
    return pos, box, np.tile(sub, nx * ny * nz)


def jitter(pos: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    return pos + _rng(seed).normal(0.0, sigma, pos.shape)


def maxwell_boltzmann(masses_per_atom: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Velocities (Angstrom/fs) ~ N(0, k_B T / m); centre-of-mass motion removed; rescaled so
    the kinetic temperature with 3N - 3 degrees of freedom is exactly ``temperature``."""
    m = np.asarray(masses_per_atom, dtype=np.float64)
    n = m.shape[0]
    if n < 2 or temperature <= 0.0:
        return np.zeros((n, 3))
    sig = np.sqrt(KB_EV * temperature / (m * AMU_A2_PER_FS2_IN_EV))
    v = _rng(seed).normal(0.0, 1.0, (n, 3)) * sig[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    ke = 0.5 * AMU_A2_PER_FS2_IN_EV * float((m[:, None] * v * v).sum())
    t_now = 2.0 * ke / ((3 * n - 3) * KB_EV)
    return v * math.sqrt(temperature / t_now)


def shear_box(box: np.ndarray, max_strain: float, seed: int) -> np.ndarray:
    """box <- box @ (I + E) with off-diagonal E ~ U(-max_strain, max_strain)."""
    e = _rng(seed).uniform(-max_strain, max_strain, (3, 3))
    np.fill_diagonal(e, 0.0)
    return box @ (np.eye(3) + e)


@dataclass
class Workload:
    name: str
    model: NepModel
    pos: np.ndarray
    types: np.ndarray
    box: np.ndarray
    vel: np.ndarray | None = None
    dt_fs: float = 1.0
    n_steps: int = 0
    temperature: float = 0.0

    @property
    def n_atoms(self) -> int:
        return self.pos.shape[0]

    def masses(self) -> np.ndarray:
        return self.model.mass[self.types]


# Model shapes of the workloads (K = n_max, since every example in the paper uses
# N_bas = n_max; l_max 4 with the 4-body (l = 2) and 5-body (l = 1) terms).
SI_MODEL = dict(n_types=1, rc_radial=5.0, rc_angular=4.0, n_max_radial=8, n_max_angular=4,
                basis_radial=8, basis_angular=4, l_max_3b=4, l_max_4b=2, l_max_5b=1, n_neuron=50)
PBTE_MODEL = dict(n_types=2, rc_radial=6.0, rc_angular=4.0, n_max_radial=10, n_max_angular=6,
                  basis_radial=10, basis_angular=6, l_max_3b=4, l_max_4b=2, l_max_5b=1, n_neuron=30)
MIXED_MODEL = dict(n_types=3, rc_radial=5.5, rc_angular=4.0, n_max_radial=8, n_max_angular=4,
                   basis_radial=8, basis_angular=4, l_max_3b=4, l_max_4b=2, l_max_5b=1, n_neuron=40)


def si_diamond(reps: int = 3, seed: int = 0, sigma: float = 0.05, temperature: float = 300.0,
               n_steps: int = 100, dt_fs: float = 1.0, with_velocities: bool = True) -> Workload:
    """Si diamond, reps^3 conventional cells, a = 5.43 A (216 atoms at reps = 3;
    8,000,000 atoms at reps = 100)."""
    pos, box, _ = lattice("diamond", 5.43, (reps, reps, reps))
    pos = jitter(pos, sigma, seed + 1000)
    types = np.zeros(pos.shape[0], np.int32)
    model = random_model(SI_MODEL, seed, [MASS_SI])
    vel = maxwell_boltzmann(model.mass[types], temperature, seed + 2000) if with_velocities else None
    return Workload(f"si_diamond_{reps}x{reps}x{reps}", model, pos, types, box, vel, dt_fs,
                    n_steps, temperature)


def pbte_rocksalt(reps: int = 32, seed: int = 1, sigma: float = 0.1, temperature: float = 300.0,
                  n_steps: int = 1000, dt_fs: float = 2.0, with_velocities: bool = True) -> Workload:
    """Rocksalt PbTe, reps^3 conventional cells, a = 6.46 A (262,144 atoms at reps = 32)."""
    pos, box, sub = lattice("rocksalt", 6.46, (reps, reps, reps))
    pos = jitter(pos, sigma, seed + 1000)
    types = sub.astype(np.int32)
    model = random_model(PBTE_MODEL, seed, [MASS_PB, MASS_TE])
    vel = maxwell_boltzmann(model.mass[types], temperature, seed + 2000) if with_velocities else None
    return Workload(f"pbte_rocksalt_{reps}x{reps}x{reps}", model, pos, types, box, vel, dt_fs,
                    n_steps, temperature)


def random_structure(seed: int, n_atoms: int, n_types_model: int = 3, sigma: float = 0.1,
                     max_shear: float = 0.1):
    """One random periodic structure: FCC (a = 4.05 A), BCC (3.30 A) or diamond (5.43 A),
    lattice constant scaled by U(0.95, 1.05); the smallest near-cubic supercell with at
    least ``n_atoms`` sites, random sites deleted down to ``n_atoms``; 1..n_types_model
    species drawn uniformly; cell sheared by U(-max_shear, max_shear) off-diagonal strain;
    Gaussian jitter sigma. Returns (pos, types, box)."""
    rng = _rng(seed)
    kind = ["fcc", "bcc", "diamond"][int(rng.integers(0, 3))]
    a0 = {"fcc": 4.05, "bcc": 3.30, "diamond": 5.43}[kind] * float(rng.uniform(0.95, 1.05))
    nb = {"fcc": 4, "bcc": 2, "diamond": 8}[kind]
    cells = int(math.ceil(n_atoms / nb))
    best = None
    for nx in range(1, cells + 1):
        if int(math.ceil(cells / (nx * nx))) < nx:
            break  # nz >= ny >= nx is impossible from here on
        for ny in range(nx, cells + 1):
            nz = int(math.ceil(cells / (nx * ny)))
            if nz < ny:
                break  # nz only falls and ny only grows along this loop
            key = (nx * ny * nz, nz - nx)
            if best is None or key < best[0]:
                best = (key, (nx, ny, nz))
    reps = best[1]
    pos, box, _ = lattice(kind, a0, reps)
    keep = np.sort(rng.permutation(pos.shape[0])[:n_atoms])
    pos = pos[keep]
    n_species = int(rng.integers(1, n_types_model + 1))
    species = np.sort(rng.permutation(n_types_model)[:n_species])
    types = species[rng.integers(0, n_species, n_atoms)].astype(np.int32)
    frac = pos @ np.linalg.inv(box)
    box = shear_box(box, max_shear, int(rng.integers(0, 2**31)))
    pos = frac @ box
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    return pos, types, box


def mixed_model(seed: int = 0) -> NepModel:
    """The three-species model of the batch and serving workloads (rc 5.5 / 4.0 A,
    n_max 8 / 4, N_neu = 40; types 0, 1, 2 with the masses of Si, Ge and C)."""
    return random_model(MIXED_MODEL, seed, [MASS_SI, MASS_GE, MASS_C])


@dataclass
class Batch:
    """Concatenated independent structures: structure s owns atoms [offsets[s], offsets[s+1])."""
    offsets: np.ndarray  # [S+1] int32
    pos: np.ndarray      # [N, 3]
    types: np.ndarray    # [N] int32
    boxes: np.ndarray    # [S, 3, 3]
    seeds: np.ndarray    # [S] structure seeds

    @property
    def n_struct(self) -> int:
        return self.boxes.shape[0]

    @property
    def n_atoms(self) -> int:
        return int(self.offsets[-1])

    def structure(self, s: int):
        a, b = int(self.offsets[s]), int(self.offsets[s + 1])
        return self.pos[a:b], self.types[a:b], self.boxes[s]

    def subset(self, idx) -> "Batch":
        parts = [self.structure(int(s)) for s in idx]
        return concat_structures(parts, self.seeds[np.asarray(idx, dtype=np.int64)])


def concat_structures(parts, seeds=None) -> Batch:
    """Batch from a list of (pos, types, box)."""
    sizes = [p[0].shape[0] for p in parts]
    offsets = np.zeros(len(parts) + 1, np.int32)
    offsets[1:] = np.cumsum(sizes)
    pos = np.concatenate([p[0] for p in parts]) if parts else np.zeros((0, 3))
    types = np.concatenate([p[1] for p in parts]).astype(np.int32) if parts else np.zeros(0, np.int32)
    boxes = np.stack([p[2] for p in parts]) if parts else np.zeros((0, 3, 3))
    seeds = np.asarray(seeds if seeds is not None else np.arange(len(parts)), dtype=np.int64)
    return Batch(offsets, np.ascontiguousarray(pos, dtype=np.float64), np.ascontiguousarray(types),
                 np.ascontiguousarray(boxes, dtype=np.float64), seeds)


def batch_structures(n_struct: int = 4096, seed: int = 3, n_min: int = 8, n_max: int = 512,
                     n_types_model: int = 3, sigma: float = 0.1, max_shear: float = 0.1) -> Batch:
    """The structure batch: n_struct random structures (``random_structure``) with atom
    counts uniform in [n_min, n_max]; structure s uses seed 1000003 * seed + s."""
    rng = _rng(seed)
    sizes = rng.integers(n_min, n_max + 1, n_struct)
    seeds = 1000003 * seed + np.arange(n_struct, dtype=np.int64)
    parts = [random_structure(int(seeds[s]), int(sizes[s]), n_types_model, sigma, max_shear)
             for s in range(n_struct)]
    return concat_structures(parts, seeds)


def subcell_cluster(w: Workload, reps: int, cells: int = 8, halo: float | None = None):
    """The atoms of conventional cells [0, cells)^3 of a cubic ``reps``^3 supercell workload
    (lattice index order of ``lattice``), cut out with every atom within ``halo`` (default
    2 r_c^R: the neighbours of the neighbours) as an open cluster in a cubic box wide enough
    that no periodic image comes within r_c^R. Positions are the workload's own, taken by the
    minimum image relative to the subcell centre.

    Returns (pos [M, 3], types [M], box [3, 3], inner [n_inner] indices into the cluster,
    sel [n_inner] the same atoms' indices in the workload), inner and sel in workload order."""
    L = float(w.box[0, 0])
    if not np.allclose(w.box, np.diag(np.diag(w.box))) or not np.allclose(np.diag(w.box), L):
        raise ValueError("subcell_cluster needs a cubic box")
    a = L / reps
    nb = w.n_atoms // reps ** 3
    rc = w.model.rc_radial
    halo = 2.0 * rc if halo is None else float(halo)
    ix, iy, iz = np.meshgrid(np.arange(cells), np.arange(cells), np.arange(cells), indexing="ij")
    cell_idx = ((ix * reps + iy) * reps + iz).ravel()
    sel = np.sort((cell_idx[:, None] * nb + np.arange(nb)[None, :]).ravel())
    centre = np.full(3, 0.5 * cells * a)
    d = w.pos - centre
    d -= L * np.round(d / L)
    half = 0.5 * cells * a + halo
    keep = np.nonzero(np.all(np.abs(d) < half, axis=1))[0]
    side = 2.0 * half + 2.0 * rc + 5.0
    inner = np.searchsorted(keep, sel)
    if not np.array_equal(keep[inner], sel):
        raise ValueError("subcell atoms moved outside the cut")
    return d[keep] + 0.5 * side, w.types[keep].copy(), np.eye(3) * side, inner, sel
