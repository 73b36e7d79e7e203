"""Seeded synthetic LSMS workloads (fcc NiAu-like random alloys).

This module generates *inputs only*: lattice positions, species, well depths,
spin directions and contour energies.  It holds none of the method's
arithmetic (no Bessel functions, harmonics, t-matrices, structure constants or
linear algebra), so both the CUDA library's tests and the CPU oracle can draw
from it without sharing any of the computation they are checked on.

Stand-ins for the paper's NiAu / CoCrFeMnNi systems (arXiv 2308.16317,
Sec. 4.1: fcc alloys, N_LIZ = 135 or 249, complex double), whose potentials
are not available: square wells on an fcc lattice with the paper's shapes.

Units: Rydberg atomic units (lengths in bohr, energies in Ry).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
A_LAT_ANGSTROM = 3.75
A_LAT = A_LAT_ANGSTROM * BOHR_PER_ANGSTROM          # fcc lattice constant, bohr
R_MT = A_LAT / (2.0 * np.sqrt(2.0))                 # touching spheres, bohr
V_SPECIES = (-1.0, -1.4)                            # well depths of species A, B (Ry)
SPIN_SPLIT = 0.05                                   # up = V - 0.05 (deeper), down = V + 0.05
E_BOT, E_F = -0.3, 0.7                              # semicircle contour end points (Ry)
SEED_BASE = 16317


def fcc_shell_table(max_shell: int):
    """Integer offsets (i,j,k), i+j+k even, of the fcc lattice through `max_shell`
    neighbour shells, in units of a/2, sorted by (shell, x, y, z); centre first.
    Returns (offsets [N,3] int, shell index [N] int, shell squared radii)."""
    lim = 2 * max_shell + 2
    pts = [p for p in itertools.product(range(-lim, lim + 1), repeat=3) if sum(p) % 2 == 0]
    r2 = sorted({p[0] ** 2 + p[1] ** 2 + p[2] ** 2 for p in pts})
    radii = r2[: max_shell + 1]
    keep = [p for p in pts if p[0] ** 2 + p[1] ** 2 + p[2] ** 2 <= radii[-1]]
    shell_of = {v: s for s, v in enumerate(radii)}
    keep.sort(key=lambda p: (shell_of[p[0] ** 2 + p[1] ** 2 + p[2] ** 2], p[0], p[1], p[2]))
    off = np.array(keep, dtype=np.int64)
    shell = np.array([shell_of[int((o ** 2).sum())] for o in off], dtype=np.int64)
    return off, shell, radii


def fcc_cluster(max_shell: int):
    """Positions (bohr) of a centred fcc cluster through `max_shell` shells."""
    off, shell, _ = fcc_shell_table(max_shell)
    return off.astype(np.float64) * (A_LAT / 2.0), shell


def semicircle_contour(n_e: int, e_bot: float = E_BOT, e_f: float = E_F, im_min: float | None = None):
    """Gauss-Legendre nodes in the angle of the semicircle from e_bot to e_f in
    the upper half plane, ordered from e_bot to e_f.  If im_min is given, the
    imaginary part is clamped from below (the end nodes only)."""
    x, _ = np.polynomial.legendre.leggauss(n_e)
    theta = 0.5 * np.pi * (1.0 - x)                 # x ascending -> theta from ~pi to ~0
    c, r = 0.5 * (e_bot + e_f), 0.5 * (e_f - e_bot)
    E = c + r * np.exp(1j * theta)
    if im_min is not None:
        E = E.real + 1j * np.maximum(E.imag, im_min)
    return E.astype(np.complex128)


def random_unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@dataclasses.dataclass
class Liz:
    """One local interaction zone: positions (centre first) and species."""
    pos: np.ndarray          # [N,3] float64, bohr, pos[0] = centre
    species: np.ndarray      # [N] int32 in {0, 1}
    dirs: np.ndarray | None = None   # [N,3] unit moment directions (canted), or None

    @property
    def n_sites(self) -> int:
        return int(self.pos.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    lmax: int
    lizs: list
    energies: np.ndarray             # [nE] complex128
    v_species: np.ndarray            # [nspin][n_species] well depth per spin channel
    r_mt: float
    canted: bool = False

    @property
    def nspin(self) -> int:
        return int(self.v_species.shape[0])

    def kappa(self) -> int:
        return (self.lmax + 1) ** 2 * (2 if self.canted else 1)

    def n_of(self, liz: Liz) -> int:
        return liz.n_sites * (self.lmax + 1) ** 2 * (2 if self.canted else 1)

    def site_depths(self, liz: Liz, spin: int) -> np.ndarray:
        return self.v_species[spin][liz.species]


def spin_depths(nspin: int) -> np.ndarray:
    v = np.array(V_SPECIES)
    if nspin == 1:
        return v[None, :]
    return np.stack([v - SPIN_SPLIT, v + SPIN_SPLIT])


def first_shell_small(seed: int = SEED_BASE + 1) -> Workload:
    """13-site first-shell cluster, lmax = 2 (n = 117), 8 contour energies,
    one spin, species A/B drawn Bernoulli(1/2) per site."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(1)
    species = rng.integers(0, 2, size=pos.shape[0]).astype(np.int32)
    return Workload("fcc13_lmax2_8E", 2, [Liz(pos, species)], semicircle_contour(8),
                    spin_depths(1), R_MT)


def liz135(seed: int = SEED_BASE + 2, n_e: int = 32, im_min: float | None = 0.005) -> Workload:
    """135-site LIZ (fcc shells 1-7), lmax = 3 (n = 2160), random 50/50 alloy,
    32 contour energies (Im E clamped at 0.005), two collinear spins."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(7)
    species = rng.integers(0, 2, size=pos.shape[0]).astype(np.int32)
    return Workload("fcc135_lmax3_32E_2spin", 3, [Liz(pos, species)], semicircle_contour(n_e, im_min=im_min),
                    spin_depths(2), R_MT)


def supercell_species(rng: np.random.Generator, ncell: int = 4):
    """fcc supercell of ncell^3 conventional cells, exact 50/50 shuffle.
    Returns (integer site coordinates in units of a/2 [Ns,3], species [Ns])."""
    basis = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]])
    cells = np.array(list(itertools.product(range(ncell), repeat=3)))
    sites = (2 * cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    ns = sites.shape[0]
    species = np.array([0] * (ns // 2) + [1] * (ns - ns // 2), dtype=np.int32)
    rng.shuffle(species)
    return sites, species


def batched_supercell(seed: int = SEED_BASE + 3, n_e: int = 32, ncell: int = 4,
                      n_sites: int | None = None) -> Workload:
    """Per-site LIZs of a 256-site periodic supercell with random vacancies:
    shell cutoff S uniform in {3..7}; a fraction f ~ U[0, 0.2] of the sites in
    shells 4..S is removed (centre and shells 1-3 are never vacant), so
    N_LIZ spans 43..135 and n = 688..2160 at lmax = 3."""
    rng = np.random.default_rng(seed)
    sites, species = supercell_species(rng, ncell)
    box = 2 * ncell
    index = {tuple(s): k for k, s in enumerate(sites)}
    off7, shell7, _ = fcc_shell_table(7)
    lizs = []
    count = sites.shape[0] if n_sites is None else min(n_sites, sites.shape[0])
    for k in range(count):
        S = int(rng.integers(3, 8))
        f = float(rng.uniform(0.0, 0.2))
        sel = np.nonzero(shell7 <= S)[0]
        outer = sel[shell7[sel] >= 4]
        n_vac = int(np.floor(f * outer.size))
        vac = set(rng.choice(outer, size=n_vac, replace=False).tolist()) if n_vac else set()
        keep = np.array([s for s in sel if s not in vac])
        off = off7[keep]
        nbr = [index[tuple(((sites[k] + o) % box).tolist())] for o in off]
        pos = off.astype(np.float64) * (A_LAT / 2.0)
        lizs.append(Liz(pos, species[nbr].astype(np.int32)))
    return Workload("supercell256_vacancies_lmax3_32E_2spin", 3, lizs, semicircle_contour(n_e, im_min=0.005),
                    spin_depths(2), R_MT)


def canted135(seed: int = SEED_BASE + 4, n_e: int = 32) -> Workload:
    """Config-2 geometry with a random unit moment direction per site (spin
    canting, M of order 2n = 4320); contour nodes unclamped (Im E >= 0.00215)."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(7)
    species = rng.integers(0, 2, size=pos.shape[0]).astype(np.int32)
    dirs = random_unit_vectors(rng, pos.shape[0])
    return Workload("fcc135_lmax3_32E_canted", 3, [Liz(pos, species, dirs)], semicircle_contour(n_e),
                    spin_depths(2), R_MT, canted=True)


def random_liz(seed: int, max_shell: int = 7) -> Liz:
    """A random 50/50 LIZ (used for the learned warm start's training set)."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(max_shell)
    return Liz(pos, rng.integers(0, 2, size=pos.shape[0]).astype(np.int32))


# ---------------------------------------------------------------------------
# The paper's own matrix shapes (Sec. 4.1): lmax = 4 (kappa = 25 per spin).
# The alloys' potentials are not available; square wells of graded depths
# stand in for the species, on the paper's lattice type, LIZ sizes and ranks.

def _depths(n_species: int, nspin: int) -> np.ndarray:
    """Well depths evenly spread over [V_A, V_B], split by spin as elsewhere."""
    v = np.linspace(V_SPECIES[0], V_SPECIES[1], n_species)
    if nspin == 1:
        return v[None, :]
    return np.stack([v - SPIN_SPLIT, v + SPIN_SPLIT])


def niau249(seed: int = SEED_BASE + 6, n_e: int = 8) -> Workload:
    """Ni30Au70-shaped LIZ: 249 sites (fcc shells 1-12), lmax = 4, rank
    n = 6225; species Ni with probability 0.3 per site; two collinear spins."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(12)
    species = (rng.random(pos.shape[0]) >= 0.3).astype(np.int32)   # 0 = Ni, 1 = Au
    return Workload("niau249_lmax4", 4, [Liz(pos, species)], semicircle_contour(n_e, im_min=0.005),
                    _depths(2, 2), R_MT)


def cocrfemnni135_canted(seed: int = SEED_BASE + 7, n_e: int = 8) -> Workload:
    """CoCrFeMnNi-shaped LIZ: 135 sites (shells 1-7), lmax = 4, five species
    drawn uniformly, random moment directions: canted rank 2n = 6750."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(7)
    species = rng.integers(0, 5, size=pos.shape[0]).astype(np.int32)
    dirs = random_unit_vectors(rng, pos.shape[0])
    return Workload("cocrfemnni135_lmax4_canted", 4, [Liz(pos, species, dirs)], semicircle_contour(n_e),
                    _depths(5, 2), R_MT, canted=True)


def niau249_canted(seed: int = SEED_BASE + 8, n_e: int = 8) -> Workload:
    """Ni30Au70-shaped LIZ with spin canting: 249 sites (fcc shells 1-12),
    lmax = 4, random moment directions, canted rank 2n = 12450 (the paper's
    largest rank, Sec. 4.1); contour nodes unclamped."""
    rng = np.random.default_rng(seed)
    pos, _ = fcc_cluster(12)
    species = (rng.random(pos.shape[0]) >= 0.3).astype(np.int32)   # 0 = Ni, 1 = Au
    dirs = random_unit_vectors(rng, pos.shape[0])
    return Workload("niau249_lmax4_canted", 4, [Liz(pos, species, dirs)], semicircle_contour(n_e),
                    _depths(2, 2), R_MT, canted=True)


# ---------------------------------------------------------------------------
# Periodic crystals for the full-KKR path (the paper's Sec. 5 target): the
# same square wells on a lattice with a basis instead of a finite LIZ.

@dataclasses.dataclass
class Crystal:
    """One periodic crystal: primitive vectors (rows), basis sites, species."""
    name: str
    lattice: np.ndarray              # [3,3] rows a1, a2, a3 (bohr)
    basis: np.ndarray                # [N_b,3] (bohr)
    species: np.ndarray              # [N_b] int32
    lmax: int
    n_k: int                         # mesh points per reciprocal axis
    energies: np.ndarray             # [nE] complex128
    v_species: np.ndarray            # [nspin][n_species]
    r_mt: float

    @property
    def nspin(self) -> int:
        return int(self.v_species.shape[0])

    @property
    def n_basis(self) -> int:
        return int(self.basis.shape[0])

    def site_depths(self, spin: int) -> np.ndarray:
        return self.v_species[spin][self.species]


FCC_PRIMITIVE = 0.5 * A_LAT * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
FCC_CUBIC_BASIS = A_LAT * np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def fcc_crystal(species: int = 0, lmax: int = 3, n_e: int = 32, n_k: int = 16) -> Crystal:
    """Pure fcc element on the primitive cell (one site), lmax = 3 (M(k) of
    order 16), 32 contour energies (Im E >= 0.005), two spins."""
    return Crystal("fcc1_lmax%d_nk%d" % (lmax, n_k), FCC_PRIMITIVE.copy(), np.zeros((1, 3)),
                   np.array([species], np.int32), lmax, n_k, semicircle_contour(n_e, im_min=0.005),
                   spin_depths(2), R_MT)


def l12_crystal(lmax: int = 3, n_e: int = 32, n_k: int = 8) -> Crystal:
    """Ordered Ni3Au-like L1_2 alloy on the 4-site simple-cubic cell of the fcc
    lattice (species B at the cube corner, A on the face centres), lmax = 3
    (M(k) of order 64), 32 contour energies (Im E >= 0.005), two spins."""
    return Crystal("l12_cell4_lmax%d_nk%d" % (lmax, n_k), A_LAT * np.eye(3), FCC_CUBIC_BASIS.copy(),
                   np.array([1, 0, 0, 0], np.int32), lmax, n_k, semicircle_contour(n_e, im_min=0.005),
                   spin_depths(2), R_MT)
