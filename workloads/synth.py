"""Seeded synthetic workloads (geometry, basis, MM charges, density matrix).

Recipe (all lengths converted to bohr with 1 bohr = 0.52917721092 Angstrom):

* MM water: rigid TIP3P geometry (O-H 0.9572 A, H-O-H 104.52 deg), charges O -0.834,
  H +0.417, uniformly random orientations (random unit quaternions); oxygens on a cubic lattice
  with a half-spacing offset, jittered uniformly by +-0.3 A; waters whose oxygen lies within
  2.0 A of a QM atom are dropped.  The box spans [-L/2, L/2)^3 and the QM region sits at the
  origin.
* Basis: per shell, exponents log-uniform in [0.1, 50] bohr^-2, raw coefficients uniform in
  [0.1, 1] (the library normalises them).
* Density matrix: gamma = X X^T with X an nao x nao standard normal matrix, scaled to a trace.

Nothing in here evaluates the method; it only draws inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.52917721092
SEED_BASE = 2408032730

Z_OF = {"H": 1.0, "C": 6.0, "N": 7.0, "O": 8.0}
L_OF = {"s": 0, "p": 1, "d": 2, "f": 3}


@dataclasses.dataclass
class System:
    """One QM/MM geometry plus basis, MM charges, Ewald parameters and a density matrix.

    All lengths are in bohr.  Shell arrays follow the C ABI layout: shell i sits on atom
    ``shell_atom[i]`` with angular momentum ``shell_l[i]`` and primitives
    ``prim_exp/prim_coeff[shell_prim_offset[i] : shell_prim_offset[i] + shell_nprim[i]]``.
    ``mm_sigma <= 0`` marks a point charge; otherwise the charge is a normalised Gaussian with
    exponent 1/sigma^2.
    """

    name: str
    atom_xyz: np.ndarray
    atom_Z: np.ndarray
    shell_atom: np.ndarray
    shell_l: np.ndarray
    shell_nprim: np.ndarray
    shell_prim_offset: np.ndarray
    prim_exp: np.ndarray
    prim_coeff: np.ndarray
    mm_xyz: np.ndarray
    mm_q: np.ndarray
    mm_sigma: np.ndarray
    box: np.ndarray
    cutoff: float
    ewald_alpha: float
    kmax: tuple
    ewald_rcut: float = 0.0  # <= 0 means "equal to cutoff"
    dm: np.ndarray | None = None
    seed: int = 0

    @property
    def natm(self) -> int:
        return int(self.atom_xyz.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nmm(self) -> int:
        return int(self.mm_xyz.shape[0])

    @property
    def nao(self) -> int:
        return int(sum((l + 1) * (l + 2) // 2 for l in self.shell_l))

    def copy(self) -> "System":
        return dataclasses.replace(
            self,
            **{f.name: (getattr(self, f.name).copy() if isinstance(getattr(self, f.name), np.ndarray)
                        else getattr(self, f.name)) for f in dataclasses.fields(self)})


# ----------------------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------------------

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly random rotation matrices from random unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random((3, n))
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _tip3p_local() -> np.ndarray:
    """TIP3P water in its own frame (Angstrom): O at the origin, H-O-H 104.52 deg."""
    r, th = 0.9572, math.radians(104.52)
    return np.array([[0.0, 0.0, 0.0],
                     [r * math.sin(th / 2), r * math.cos(th / 2), 0.0],
                     [-r * math.sin(th / 2), r * math.cos(th / 2), 0.0]])


def mm_water_box(rng: np.random.Generator, box_A: float, n_per_side: int, n_waters: int | None,
                 qm_xyz_A: np.ndarray, drop_within_A: float = 2.0, jitter_A: float = 0.3):
    """Rigid TIP3P waters on a jittered cubic lattice in [-L/2, L/2)^3 (positions in Angstrom).

    ``n_waters`` lattice sites are drawn without replacement from the ``n_per_side^3`` sites
    (all sites when None).  Returns (xyz[n,3], q[n]).
    """
    a = box_A / n_per_side
    idx = np.arange(n_per_side)
    g = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), axis=-1).reshape(-1, 3)
    sites = (g + 0.5) * a - box_A / 2
    if n_waters is not None and n_waters < len(sites):
        pick = np.sort(rng.choice(len(sites), size=n_waters, replace=False))
        sites = sites[pick]
    sites = sites + rng.uniform(-jitter_A, jitter_A, size=sites.shape)
    rot = _random_rotations(rng, len(sites))
    local = _tip3p_local()
    mol = sites[:, None, :] + np.einsum("nij,kj->nki", rot, local)
    if len(qm_xyz_A):
        d = np.linalg.norm(mol[:, 0, None, :] - qm_xyz_A[None, :, :], axis=-1)
        keep = d.min(axis=1) >= drop_within_A
        mol = mol[keep]
    q = np.tile(np.array([-0.834, 0.417, 0.417]), len(mol))
    return mol.reshape(-1, 3), q


def random_shells(rng: np.random.Generator, atom_elems, recipe: dict, nprim):
    """Seeded contracted Cartesian shells.

    recipe maps an element to a shell string such as "3s2p1d"; ``nprim`` is an int or a
    (lo, hi) inclusive range drawn per shell.
    """
    shell_atom, shell_l, shell_nprim, prim_exp, prim_coeff = [], [], [], [], []
    for ia, el in enumerate(atom_elems):
        spec = recipe[el]
        i = 0
        while i < len(spec):
            j = i
            while spec[j].isdigit():
                j += 1
            count, l = int(spec[i:j]), L_OF[spec[j]]
            i = j + 1
            for _ in range(count):
                n = nprim if isinstance(nprim, int) else int(rng.integers(nprim[0], nprim[1] + 1))
                shell_atom.append(ia)
                shell_l.append(l)
                shell_nprim.append(n)
                prim_exp.extend(np.exp(rng.uniform(math.log(0.1), math.log(50.0), size=n)))
                prim_coeff.extend(rng.uniform(0.1, 1.0, size=n))
    shell_nprim = np.array(shell_nprim, dtype=np.int32)
    off = np.zeros_like(shell_nprim)
    off[1:] = np.cumsum(shell_nprim)[:-1]
    return (np.array(shell_atom, dtype=np.int32), np.array(shell_l, dtype=np.int32), shell_nprim,
            off.astype(np.int32), np.array(prim_exp), np.array(prim_coeff))


def random_density(rng: np.random.Generator, nao: int, trace: float) -> np.ndarray:
    """Random symmetric positive semi-definite density matrix X X^T scaled to a given trace."""
    X = rng.standard_normal((nao, nao))
    dm = X @ X.T
    dm *= trace / np.trace(dm)
    return 0.5 * (dm + dm.T)


def cluster_in_sphere(rng: np.random.Generator, n: int, radius_A: float, min_dist_A: float) -> np.ndarray:
    """n points uniform in a sphere of given radius, rejecting any closer than min_dist."""
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("could not place QM atoms")
        p = rng.uniform(-radius_A, radius_A, size=3)
        if p @ p > radius_A * radius_A:
            continue
        if pts and np.min(np.linalg.norm(np.asarray(pts) - p, axis=1)) < min_dist_A:
            continue
        pts.append(p)
    return np.asarray(pts)


def _assemble(name, seed, qm_xyz_A, elems, shells, mm_xyz_A, mm_q, sigma_A, box_A, cutoff_A,
              alpha_invA, kmax, dm_trace, rng, ewald_rcut_A=0.0) -> System:
    sa, sl, sn, so, pe, pc = shells
    sysm = System(
        name=name,
        atom_xyz=np.ascontiguousarray(qm_xyz_A * ANGSTROM_TO_BOHR),
        atom_Z=np.array([Z_OF[e] for e in elems]),
        shell_atom=sa, shell_l=sl, shell_nprim=sn, shell_prim_offset=so,
        prim_exp=pe, prim_coeff=pc,
        mm_xyz=np.ascontiguousarray(mm_xyz_A * ANGSTROM_TO_BOHR),
        mm_q=np.ascontiguousarray(mm_q, dtype=np.float64),
        mm_sigma=np.full(len(mm_q), sigma_A * ANGSTROM_TO_BOHR),
        box=np.full(3, box_A * ANGSTROM_TO_BOHR),
        cutoff=cutoff_A * ANGSTROM_TO_BOHR,
        ewald_alpha=alpha_invA / ANGSTROM_TO_BOHR,
        kmax=tuple(int(k) for k in kmax),
        ewald_rcut=ewald_rcut_A * ANGSTROM_TO_BOHR,
        seed=seed,
    )
    sysm.dm = random_density(rng, sysm.nao, dm_trace if dm_trace is not None else float(sysm.atom_Z.sum()))
    return sysm


# ----------------------------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------------------------

def config1_water(seed: int | None = None) -> System:
    """QM water (O at origin, H at 0.96 A, 104.5 deg), O 3s2p1d + H 2s1p (12 shells, 25 AOs),
    3 primitives per shell; 216 TIP3P waters (6^3 lattice, 3.1 A) in an 18.6 A box; sigma 0.2 A,
    cutoff 9 A, alpha 0.35 A^-1, kmax 7; density trace 10."""
    seed = SEED_BASE + 1 if seed is None else seed
    rng = np.random.default_rng(seed)
    th = math.radians(104.5)
    qm = np.array([[0.0, 0.0, 0.0],
                   [0.96 * math.sin(th / 2), 0.96 * math.cos(th / 2), 0.0],
                   [-0.96 * math.sin(th / 2), 0.96 * math.cos(th / 2), 0.0]])
    elems = ["O", "H", "H"]
    shells = random_shells(rng, elems, {"O": "3s2p1d", "H": "2s1p"}, 3)
    mm, q = mm_water_box(rng, 18.6, 6, None, qm, drop_within_A=2.0)
    return _assemble("water_c1", seed, qm, elems, shells, mm, q, 0.2, 18.6, 9.0, 0.35, (7, 7, 7), 10.0, rng)


def make_cluster_system(name, seed, n_atoms, elem_counts, radius_A, recipe, nprim, box_A, n_side,
                        n_waters, sigma_A, cutoff_A, alpha_invA, kmax, dm_trace=None) -> System:
    """Generic active-site-like system: QM atoms uniform in a sphere (min spacing 1.0 A) at the
    box centre, a seeded basis from ``recipe`` and a TIP3P water box."""
    rng = np.random.default_rng(seed)
    qm = cluster_in_sphere(rng, n_atoms, radius_A, 1.0)
    elems = []
    for el, c in elem_counts.items():
        elems += [el] * c
    assert len(elems) == n_atoms
    elems = [elems[i] for i in rng.permutation(n_atoms)]
    shells = random_shells(rng, elems, recipe, nprim)
    mm, q = mm_water_box(rng, box_A, n_side, n_waters, qm, drop_within_A=2.0)
    return _assemble(name, seed, qm, elems, shells, mm, q, sigma_A, box_A, cutoff_A, alpha_invA, kmax,
                     dm_trace, rng)


def config2_active_site(seed: int | None = None) -> System:
    """60 QM atoms (C20 N4 O6 H30) in a 10 A sphere; heavy 6s4p3d, H 4s2p1d (600 shells,
    1560 AOs), 1-5 primitives per shell; 20000 TIP3P waters (60000 charges) in a 58 A box;
    sigma 0.2 A, cutoff 12 A, alpha 0.3 A^-1, kmax 16."""
    seed = SEED_BASE + 2 if seed is None else seed
    return make_cluster_system("active_site_c2", seed, 60, {"C": 20, "N": 4, "O": 6, "H": 30}, 10.0,
                               {"C": "6s4p3d", "N": "6s4p3d", "O": "6s4p3d", "H": "4s2p1d"}, (1, 5),
                               58.0, 28, 20000, 0.2, 12.0, 0.3, (16, 16, 16))


def config4_large_site(seed: int | None = None) -> System:
    """150 QM atoms (C50 N10 O15 H75) in a 13.6 A sphere; heavy 6s4p3d2f, H 3s1p1d (1500 shells,
    5100 AOs); 66667 TIP3P waters (~200000 charges) in an 86 A box; cutoff 12 A, alpha 0.3 A^-1,
    kmax 24."""
    seed = SEED_BASE + 4 if seed is None else seed
    return make_cluster_system("large_site_c4", seed, 150, {"C": 50, "N": 10, "O": 15, "H": 75}, 13.6,
                               {"C": "6s4p3d2f", "N": "6s4p3d2f", "O": "6s4p3d2f", "H": "3s1p1d"}, (1, 5),
                               86.0, 41, 66667, 0.2, 12.0, 0.3, (24, 24, 24))


def config5_frames(n_frames: int = 64, seed: int | None = None):
    """Uneven frames: QM water clusters of 20-120 atoms (multiples of 3, config-1 shell recipe),
    20000-120000 MM charges in a cubic box at water density (0.1003 charges/A^3), cutoff 12 A,
    alpha 0.3 A^-1, kmax = ceil(16 L / 58)."""
    seed = SEED_BASE + 5 if seed is None else seed
    rng = np.random.default_rng(seed)
    frames = []
    for f in range(n_frames):
        n_qm = 3 * int(rng.integers(7, 41))
        n_mm = int(rng.integers(20000, 120001))
        n_w = n_mm // 3
        box = (n_w * 3 / 0.1003) ** (1.0 / 3.0)
        n_side = int(math.ceil(n_w ** (1.0 / 3.0)))
        fseed = int(rng.integers(0, 2**31))
        frng = np.random.default_rng(fseed)
        radius = max(3.0, (n_qm / 3 / 0.0334 * 3 / (4 * math.pi)) ** (1.0 / 3.0))
        # QM water cluster: oxygens in a sphere, each with a randomly oriented TIP3P geometry
        o = cluster_in_sphere(frng, n_qm // 3, radius, 2.6)
        rot = _random_rotations(frng, len(o))
        qm = (o[:, None, :] + np.einsum("nij,kj->nki", rot, _tip3p_local())).reshape(-1, 3)
        elems = ["O", "H", "H"] * (n_qm // 3)
        shells = random_shells(frng, elems, {"O": "3s2p1d", "H": "2s1p"}, 3)
        mm, q = mm_water_box(frng, box, n_side, n_w, qm, drop_within_A=2.0)
        k = int(math.ceil(16 * box / 58.0))
        frames.append(_assemble(f"frame{f}", fseed, qm, elems, shells, mm, q, 0.2, box, 12.0, 0.3,
                                (k, k, k), None, frng))
    return frames


def small_system(seed: int, n_atoms: int = 3, lmax: int = 2, nprim=(1, 3), n_waters: int = 12,
                 box_A: float = 12.0, cutoff_A: float = 5.5, alpha_invA: float = 0.45, kmax=(5, 5, 5),
                 sigma_A: float = 0.2, radius_A: float = 1.6, point_charges: bool = False,
                 shells_per_atom=None) -> System:
    """Tiny seeded system for the oracle pins and parity tests (a few atoms, a handful of
    waters).  ``lmax`` caps the shell angular momenta; every atom gets one shell per l <= lmax
    unless ``shells_per_atom`` (a recipe string) is given."""
    rng = np.random.default_rng(seed)
    qm = cluster_in_sphere(rng, n_atoms, radius_A, 0.9)
    elems = [["O", "C", "N", "H"][i % 4] for i in range(n_atoms)]
    spec = shells_per_atom or "".join(f"1{'spdf'[l]}" for l in range(lmax + 1))
    shells = random_shells(rng, elems, {e: spec for e in "HCNO"}, nprim)
    n_side = max(2, int(math.ceil(n_waters ** (1.0 / 3.0))))
    mm, q = mm_water_box(rng, box_A, n_side, n_waters, qm, drop_within_A=2.0)
    s = _assemble(f"small{seed}", seed, qm, elems, shells, mm, q, sigma_A, box_A, cutoff_A, alpha_invA,
                  kmax, None, rng)
    if point_charges:
        s.mm_sigma[:] = 0.0
    return s
