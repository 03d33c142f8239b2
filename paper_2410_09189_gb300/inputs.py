"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds *inputs only*: atom geometries, pseudo-atom parameters, occupations,
random draws (KB energies, jitter) and smooth random starting orbitals.  It contains none
of the method's arithmetic (no stencil, no potentials on the grid, no Hamiltonian, no
propagation), so both sides of a parity test start from identical numbers without sharing
any code that computes a result.

Workloads (units: bohr, hartree, atomic time units):

* ``small``  -- two Z=1 Gaussian-erf wells 1.4 bohr apart on a 24^3 grid at h=0.4,
  1 doubly occupied orbital + 15 virtual, kick along z (the smallest system the
  propagation of Algorithm 1 is meaningful for).
* ``ring``   -- planar hexagonal ring: 6 Z=4 atoms at radius 2.6 and 6 Z=1 atoms at
  radius 4.6, one s-type Kleinman-Bylander projector per Z=4 atom, 64^3 grid at h=0.35,
  15 doubly occupied + 15 virtual orbitals, kicks along x, y and z.  A benzene-like
  stand-in (30 valence electrons) for the paper's benzene benchmark (Section 4.1).
* ``icosa``  -- 147-atom Mackay icosahedron (shells 1+12+42+92) scaled to a 5.4 bohr
  minimum distance, Z=1 plus one s-type projector each, 128^3 grid at h=0.4,
  74 doubly occupied + 74 virtual orbitals: a metal-cluster stand-in for the paper's
  silver nanoparticles (Section 4.3).
* ``cluster(i)`` -- the batched workload's eight random clusters (20-150 atoms, 48^3-96^3).
* ``fcc_large`` -- the large workload: the 1,024 sites of an FCC lattice (nearest-neighbour
  distance 5.4 bohr) nearest the box centre, jittered, Z=2 each with one s and three p
  projectors, 192^3 grid at h=0.4, 1,024 doubly occupied + 1,024 virtual orbitals: the
  stand-in for the paper's largest silver clusters (Section 4.3).

Seeds are ``241009189 + 1000*workload_index + sub_index``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 241009189


@dataclasses.dataclass
class System:
    """Everything that defines one propagation problem (inputs only)."""

    name: str
    n: tuple                 # (nx, ny, nz) grid points
    h: float                 # grid spacing (bohr)
    pos: np.ndarray          # (natoms, 3) atom positions, origin = box centre
    Z: np.ndarray            # (natoms,) valence charges of the local wells
    rc_loc: np.ndarray       # (natoms,) erf radius of the local wells
    proj_atom: np.ndarray    # (nproj,) int atom index of each KB projector
    proj_l: np.ndarray       # (nproj,) int angular momentum (0 = s, 1 = p)
    proj_m: np.ndarray       # (nproj,) int component for l=1 (0=x, 1=y, 2=z)
    proj_rc: np.ndarray      # (nproj,) Gaussian radius of each projector
    E_kb: np.ndarray         # (nproj,) KB energies (hartree), seeded draws
    nocc: int
    nvirt: int
    dt: float = 0.05
    kappa: float = 1e-3
    kick_axes: tuple = (2,)
    nsteps: int = 200
    hartree_xc: bool = True  # False: independent electrons in V_loc (+ v_ext)
    v_ext_omega: float = 0.0  # >0 adds a harmonic well 0.5*omega^2*r^2 (test mode)
    seed: int = SEED_BASE
    rho_core: Optional[np.ndarray] = None  # frozen core density (nz, ny, nx), xc only

    @property
    def N(self) -> int:
        return self.nocc + self.nvirt

    @property
    def Ng(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nproj(self) -> int:
        return int(len(self.proj_atom))

    @property
    def occupations(self) -> np.ndarray:
        """f_i = 2 for the doubly occupied orbitals, 0 for the virtual ones."""
        f = np.zeros(self.N)
        f[: self.nocc] = 2.0
        return f

    @property
    def n_electrons(self) -> float:
        return 2.0 * self.nocc


def _no_proj():
    return (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
            np.zeros(0), np.zeros(0))


def small(n: int = 24, h: float = 0.4, nvirt: int = 15) -> System:
    """Two Z=1 wells at (0,0,+-0.7) with r_c=0.5, no nonlocal part."""
    pos = np.array([[0.0, 0.0, -0.7], [0.0, 0.0, 0.7]])
    pa, pl, pm, prc, ekb = _no_proj()
    return System("small", (n, n, n), h, pos, np.ones(2), np.full(2, 0.5),
                  pa, pl, pm, prc, ekb, nocc=1, nvirt=nvirt, kick_axes=(2,),
                  nsteps=200, seed=SEED_BASE + 1000 * 1)


def ring(n: int = 64, h: float = 0.35, nvirt: int = 15) -> System:
    """Hexagonal ring of 6 Z=4 and 6 Z=1 wells; s-type KB on the Z=4 atoms."""
    seed = SEED_BASE + 1000 * 2
    rng = np.random.default_rng(seed)
    ang = np.arange(6) * (math.pi / 3.0)
    heavy = np.stack([2.6 * np.cos(ang), 2.6 * np.sin(ang), np.zeros(6)], axis=1)
    light = np.stack([4.6 * np.cos(ang), 4.6 * np.sin(ang), np.zeros(6)], axis=1)
    pos = np.concatenate([heavy, light])
    Z = np.concatenate([np.full(6, 4.0), np.ones(6)])
    ekb = rng.uniform(0.5, 2.0, size=6)
    return System("ring", (n, n, n), h, pos, Z, np.full(12, 0.5),
                  np.arange(6, dtype=np.int32), np.zeros(6, np.int32),
                  np.zeros(6, np.int32), np.full(6, 1.2), ekb,
                  nocc=15, nvirt=nvirt, kick_axes=(0, 1, 2), nsteps=2000, seed=seed)


def _icosahedron_vertices() -> np.ndarray:
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    return np.array(v)


def mackay_icosahedron(shells: int) -> np.ndarray:
    """Centre atom plus `shells` Mackay shells (10k^2+2 sites in shell k)."""
    V = _icosahedron_vertices()
    edge = np.min([np.linalg.norm(V[i] - V[j]) for i in range(12) for j in range(i)])
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            for k in range(j + 1, 12):
                if (abs(np.linalg.norm(V[i] - V[j]) - edge) < 1e-9
                        and abs(np.linalg.norm(V[j] - V[k]) - edge) < 1e-9
                        and abs(np.linalg.norm(V[i] - V[k]) - edge) < 1e-9):
                    faces.append((i, j, k))
    pts = [np.zeros(3)]
    for s in range(1, shells + 1):
        shell = []
        for (a, b, c) in faces:
            for i in range(s + 1):
                for j in range(s + 1 - i):
                    l = s - i - j
                    shell.append((i * V[a] + j * V[b] + l * V[c]))
        shell = np.array(shell)
        keys = {}
        for p in shell:
            keys[tuple(np.round(p, 8))] = p
        pts += list(keys.values())
    return np.array(pts)


def icosa(n: int = 128, h: float = 0.4, nvirt: int = 74, shells: int = 3) -> System:
    """147-atom Mackay icosahedron, min distance 5.4 bohr, Z=1 + s-KB on every atom."""
    seed = SEED_BASE + 1000 * 3
    rng = np.random.default_rng(seed)
    p = mackay_icosahedron(shells)
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    dmin = d[np.triu_indices(len(p), 1)].min()
    pos = p * (5.4 / dmin)
    na = len(pos)
    ekb = rng.uniform(0.5, 2.0, size=na)
    nocc = (na + 1) // 2
    return System("icosa", (n, n, n), h, pos, np.ones(na), np.full(na, 0.5),
                  np.arange(na, dtype=np.int32), np.zeros(na, np.int32),
                  np.zeros(na, np.int32), np.full(na, 1.2), ekb,
                  nocc=nocc, nvirt=nvirt, kick_axes=(2,), nsteps=1000, seed=seed)


# the eight clusters of the batched workload: atom counts and grids (edge points)
CLUSTER_ATOMS = (20, 38, 56, 75, 93, 112, 131, 150)
CLUSTER_GRIDS = (48, 56, 64, 64, 72, 80, 88, 96)


def cluster(index: int, natoms: Optional[int] = None, n: Optional[int] = None,
            h: float = 0.4) -> System:
    """Cluster `index` (0..7) of the batched workload: atoms uniform in a sphere with a
    minimum distance of 4.0 bohr (rejection sampling, seeded), Z = 1 local well (r_c = 0.5)
    plus an s-type KB projector (r_c = 1.2, E_KB ~ U[0.5, 2]) on every atom, h = 0.4,
    N_occ = ceil(natoms / 2), N = 2 N_occ."""
    natoms = CLUSTER_ATOMS[index] if natoms is None else natoms
    n = CLUSTER_GRIDS[index] if n is None else n
    seed = SEED_BASE + 1000 * 4 + index
    rng = np.random.default_rng(seed)
    half = 0.5 * (n - 1) * h
    # 80 % of the half-width, enlarged (up to 95 %) where the atoms would fill more than a
    # quarter of the spheres of radius 2 around them (random placement jams near 38 %)
    radius = min(max(0.8 * half, 2.0 * (4.0 * natoms) ** (1.0 / 3.0) - 2.0), 0.95 * half)
    pts = []
    tries = 0
    while len(pts) < natoms:
        tries += 1
        if tries > 200000:
            raise ValueError("cluster: could not place the atoms at the minimum distance")
        p = rng.uniform(-radius, radius, 3)
        if np.linalg.norm(p) > radius:
            continue
        if all(np.linalg.norm(p - q) >= 4.0 for q in pts):
            pts.append(p)
    pos = np.array(pts)
    nocc = (natoms + 1) // 2
    ekb = rng.uniform(0.5, 2.0, size=natoms)
    return System(f"cluster{index}", (n, n, n), h, pos, np.ones(natoms), np.full(natoms, 0.5),
                  np.arange(natoms, dtype=np.int32), np.zeros(natoms, np.int32),
                  np.zeros(natoms, np.int32), np.full(natoms, 1.2), ekb,
                  nocc=nocc, nvirt=nocc, kick_axes=(0, 1, 2), nsteps=200, seed=seed)


def fcc_sites(nsites: int, nn: float = 5.4) -> np.ndarray:
    """The `nsites` sites of an FCC lattice with nearest-neighbour distance `nn` (cube edge
    a = nn * sqrt(2), a site at the origin) nearest the origin; equidistant sites are taken
    in lexicographic order of (x, y, z), so the selection is deterministic."""
    a = nn * math.sqrt(2.0)
    m = int(math.ceil((nsites / 4.0) ** (1.0 / 3.0))) + 2
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    r = np.arange(-m, m + 1, dtype=float)
    cells = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    d2 = np.round((pts * pts).sum(1), 9)
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], d2))
    return pts[order[:nsites]]


def fcc_large(n: int = 192, h: float = 0.4, nsites: int = 1024, jitter: float = 0.1) -> System:
    """The large workload: `fcc_sites(nsites)` each moved by N(0, jitter^2) per coordinate
    (seeded), Z = 2 local wells (r_c = 0.5) with one s and three p KB projectors (x, y, z)
    on every atom (r_c = 1.2, E_KB ~ U[0.5, 2] per projector), n^3 grid at h; two valence
    electrons per atom: N_occ = nsites, N = 2 N_occ; kick along z, 200 steps."""
    seed = SEED_BASE + 1000 * 5
    rng = np.random.default_rng(seed)
    pos = fcc_sites(nsites) + rng.normal(0.0, jitter, size=(nsites, 3))
    atoms = np.repeat(np.arange(nsites, dtype=np.int32), 4)
    pl = np.tile(np.array([0, 1, 1, 1], np.int32), nsites)
    pm = np.tile(np.array([0, 0, 1, 2], np.int32), nsites)
    ekb = rng.uniform(0.5, 2.0, size=4 * nsites)
    return System("fcc_large", (n, n, n), h, pos, np.full(nsites, 2.0), np.full(nsites, 0.5),
                  atoms, pl, pm, np.full(4 * nsites, 1.2), ekb, nocc=nsites, nvirt=nsites,
                  kick_axes=(2,), nsteps=200, seed=seed)


def harmonic(n: int = 32, h: float = 0.4, omega: float = 0.5, nvirt: int = 3) -> System:
    """Test mode: one doubly occupied orbital in V = 0.5*omega^2*r^2, no Hartree/xc."""
    pa, pl, pm, prc, ekb = _no_proj()
    return System("harmonic", (n, n, n), h, np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                  pa, pl, pm, prc, ekb, nocc=1, nvirt=nvirt, kick_axes=(2,),
                  nsteps=200, hartree_xc=False, v_ext_omega=omega,
                  seed=SEED_BASE + 7)


def scaled(base: System, n: int, h: Optional[float] = None, nocc: Optional[int] = None,
           nvirt: Optional[int] = None) -> System:
    """Same atoms and parameters on another grid / active space (parity-test sizes)."""
    out = dataclasses.replace(base, n=(n, n, n), h=base.h if h is None else h)
    if nocc is not None:
        out.nocc = nocc
    if nvirt is not None:
        out.nvirt = nvirt
    return out


def grid_shape(sys: System) -> tuple:
    """Array shape of a grid function: (nz, ny, nx), x fastest in memory."""
    return (sys.n[2], sys.n[1], sys.n[0])


def smooth_random_orbitals(sys: System, sub_index: int = 0, sigma_pts: float = 2.0,
                           window_frac: float = 0.8) -> np.ndarray:
    """Seeded smooth random starting orbitals, shape (N, nz, ny, nx), NOT orthonormal.

    A white-noise field per orbital is smoothed with a Gaussian of `sigma_pts` grid
    points and multiplied by a smooth window that vanishes at the box faces, so every
    column is a smooth function that respects the zero boundary condition.  These are
    random draws, not an eigen-solve: callers orthonormalise them themselves.
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(sys.seed + sub_index)
    shape = grid_shape(sys)
    out = np.empty((sys.N,) + shape)
    wins = []
    for ax, npts in zip((2, 1, 0), sys.n):
        t = (np.arange(npts) + 0.5) / npts           # (0,1)
        u = np.clip((t - 0.5) / (0.5 * window_frac), -1.0, 1.0)
        wins.append(np.cos(0.5 * math.pi * u) ** 2)
    win = wins[2][:, None, None] * wins[1][None, :, None] * wins[0][None, None, :]
    for i in range(sys.N):
        w = rng.standard_normal(shape)
        out[i] = gaussian_filter(w, sigma_pts, mode="constant") * win
    return out


def gaussian_core_density(sys: System, charge: float = 0.5, width: float = 0.6) -> np.ndarray:
    """A model frozen core density, shape (nz, ny, nx): a normalised Gaussian of `charge`
    electrons and `width` bohr on every atom (an input field, like the orbitals)."""
    x = (np.arange(sys.n[0]) - 0.5 * (sys.n[0] - 1)) * sys.h
    y = (np.arange(sys.n[1]) - 0.5 * (sys.n[1] - 1)) * sys.h
    z = (np.arange(sys.n[2]) - 0.5 * (sys.n[2] - 1)) * sys.h
    out = np.zeros(grid_shape(sys))
    norm = charge / (math.pi * width * width) ** 1.5
    for p in sys.pos:
        out += (norm * np.exp(-((z[:, None, None] - p[2]) ** 2) / width ** 2)
                * np.exp(-((y[None, :, None] - p[1]) ** 2) / width ** 2)
                * np.exp(-((x[None, None, :] - p[0]) ** 2) / width ** 2))
    return out


def random_matrix(n: int, seed: int) -> np.ndarray:
    """A seeded standard-normal n x n matrix (test inputs for the subspace kernels)."""
    return np.random.default_rng(seed).standard_normal((n, n))


def random_grid(sys: System, seed: int, positive: bool = False) -> np.ndarray:
    """A seeded random grid function of shape (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(grid_shape(sys))
    return np.abs(x) if positive else x


ALL = {"small": small, "ring": ring, "icosa": icosa, "harmonic": harmonic,
       "fcc_large": fcc_large}


def by_name(name: str, **kw) -> System:
    return ALL[name](**kw)


def workload_names() -> List[str]:
    return list(ALL)
