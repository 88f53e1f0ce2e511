"""Seeded synthetic inputs: diamond / zincblende boxes, displacements,
vacancies, Maxwell-Boltzmann velocities and the serving job stream.

This module holds none of the potential's arithmetic; both the CUDA path and
the FP64 oracle consume what it generates.  The paper's own benchmark (a
carbon-nanotube stretching run, Sec. 5) is not available, so these boxes stand
in for it: diamond Si keeps its ~4 in-cutoff neighbours per atom, and 3C-SiC
adds the skin-dominated neighbour lists that Sec. 3 is about.

Units: Angstrom, amu, ps, K.
"""
from dataclasses import dataclass, field

import numpy as np

K_B = 8.617333262e-5          # eV/K
EV_J = 1.602176634e-19        # J per eV
AMU_KG = 1.66053906660e-27    # kg per amu
# (eV/A)/amu expressed in A/ps^2
ACCEL = EV_J / AMU_KG * 1e-4

MASS = {"Si": 28.0855, "C": 12.011}

_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_SHIFT = np.array([0.25, 0.25, 0.25])


@dataclass
class System:
    pos: np.ndarray                 # [N, 3] float64
    types: np.ndarray               # [N] int32
    box: np.ndarray                 # [3] float64
    species: tuple                  # type index -> element name
    vel: np.ndarray = None          # [N, 3] float64, A/ps
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.pos.shape[0])

    def masses(self):
        return np.array([MASS[s] for s in self.species], dtype=np.float64)


def diamond(nx, ny, nz, a, species=("Si",)):
    """Diamond (one species) or zincblende (two species: first on the FCC
    sublattice, second on the shifted one) lattice of nx*ny*nz cubic cells,
    8 atoms per cell, in cell order."""
    basis = np.concatenate([_FCC, _FCC + _SHIFT])
    btype = np.array([0] * 4 + [1 if len(species) > 1 else 0] * 4, dtype=np.int32)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    types = np.tile(btype, cells.shape[0])
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return System(pos=pos, types=types, box=box, species=tuple(species))


def displace_uniform(s, amp, rng):
    s.pos = s.pos + rng.uniform(-amp, amp, size=s.pos.shape)
    return s


def displace_gaussian(s, sigma, rng):
    s.pos = s.pos + rng.normal(0.0, sigma, size=s.pos.shape)
    return s


def vacancies(s, frac, rng):
    """Remove floor(frac * N) sites chosen by a seeded shuffle."""
    nrem = int(np.floor(frac * s.n))
    if nrem == 0:
        return s
    keep = np.sort(rng.permutation(s.n)[nrem:])
    s.pos = s.pos[keep]
    s.types = s.types[keep]
    if s.vel is not None:
        s.vel = s.vel[keep]
    return s


def wrap(s):
    s.pos = s.pos - np.floor(s.pos / s.box) * s.box
    return s


def temperature(vel, types, masses):
    m = masses[types]
    ke = 0.5 * np.sum(m[:, None] * vel * vel) / ACCEL
    dof = 3 * len(types) - 3
    return 2.0 * ke / (dof * K_B)


def maxwell_boltzmann(s, T, rng):
    """v ~ N(0, k_B T / m) per component, zero total momentum, rescaled to
    exactly T with 3N - 3 degrees of freedom."""
    m = s.masses()[s.types]
    sig = np.sqrt(K_B * T / m * ACCEL)
    v = rng.normal(size=s.pos.shape) * sig[:, None]
    p = np.sum(m[:, None] * v, axis=0)
    v -= p / np.sum(m)
    if s.n > 1 and T > 0:
        v *= np.sqrt(T / temperature(v, s.types, s.masses()))
    s.vel = v
    return s


# ---- the named workloads ---------------------------------------------------

def si_512(seed=1):
    """Si diamond a = 5.432, 4x4x4 cells = 512 atoms, uniform +-0.05 A."""
    rng = np.random.default_rng(seed)
    s = displace_uniform(diamond(4, 4, 4, 5.432), 0.05, rng)
    s.meta = dict(name="Si diamond 4x4x4 = 512 atoms, uniform +-0.05 A", seed=seed)
    return wrap(s)


def si_box(nx, ny, nz, seed, T=1000.0, sigma=0.05, a=5.432):
    rng = np.random.default_rng(seed)
    s = displace_gaussian(diamond(nx, ny, nz, a), sigma, rng)
    s = maxwell_boltzmann(wrap(s), T, rng)
    s.meta = dict(name=f"Si diamond {nx}x{ny}x{nz} = {s.n} atoms, sigma {sigma} A, {T:g} K",
                  seed=seed, T=T, dt=1e-3)
    return s


def si_32k(seed=2):
    """Si diamond 20x20x10 = 32,000 atoms, Gaussian sigma 0.05 A, 1000 K."""
    return si_box(20, 20, 10, seed)


def si_512k(seed=3):
    """Si diamond 40x40x40 = 512,000 atoms, Gaussian sigma 0.05 A, 1000 K."""
    return si_box(40, 40, 40, seed)


def sic_box(n, seed, T=1500.0, vac=0.05, sigma=0.05, a=4.36):
    rng = np.random.default_rng(seed)
    s = diamond(n, n, n, a, species=("Si", "C"))
    s = vacancies(s, vac, rng)
    s = displace_gaussian(s, sigma, rng)
    s = maxwell_boltzmann(wrap(s), T, rng)
    s.meta = dict(name=f"3C-SiC {n}^3 cells, {vac:.0%} vacancies = {s.n} atoms, {T:g} K",
                  seed=seed, T=T, dt=0.5e-3)
    return s


def sic_1m(seed=4):
    """3C-SiC a = 4.36, 50^3 cells = 1,000,000 sites, 5% vacancies, 1500 K."""
    return sic_box(50, seed)


# ---- serving stream ----------------------------------------------------------

def cells_for_atoms(target, min_cells=1):
    """n_x <= n_y <= n_z, each >= min_cells, with 8 n_x n_y n_z closest to target
    (ties: most cubic)."""
    best = None
    cells = target / 8.0
    top = max(int(np.ceil(cells)), min_cells) + 1
    for nx in range(min_cells, max(int(np.ceil(cells ** (1 / 3))), min_cells) + 2):
        for ny in range(nx, max(int(np.ceil(np.sqrt(cells / nx))), nx) + 2):
            nz_f = cells / (nx * ny)
            for nz in (int(np.floor(nz_f)), int(np.ceil(nz_f)), ny):
                if nz < ny or nz > top:
                    continue
                err = abs(8 * nx * ny * nz - target)
                key = (err, nz - nx)
                if best is None or key < best[0]:
                    best = (key, (nx, ny, nz))
    return best[1]


@dataclass
class Job:
    arrival: float                  # seconds from stream start
    system: System
    steps: int
    dt: float                       # ps


def serving_stream(njobs=4096, seed=5, rate=None, min_atoms=64, max_atoms=16384, min_cells=2):
    """Poisson stream of MD jobs: Si or SiC (50/50), atoms log-uniform in
    [min_atoms, max_atoms], 5% vacancies, T ~ U(300, 2000) K, steps ~ U{50..500},
    dt 1 fs (Si) / 0.5 fs (SiC).  Boxes keep at least ``min_cells`` cubic cells per
    side.  rate (jobs/s) None gives arrival times of 0 (closed loop)."""
    rng = np.random.default_rng(seed)
    jobs = []
    t = 0.0
    for _ in range(njobs):
        sic = bool(rng.integers(0, 2))
        target = float(np.exp(rng.uniform(np.log(min_atoms), np.log(max_atoms))))
        nx, ny, nz = cells_for_atoms(target, min_cells)
        T = float(rng.uniform(300.0, 2000.0))
        steps = int(rng.integers(50, 501))
        if sic:
            s = diamond(nx, ny, nz, 4.36, species=("Si", "C"))
        else:
            s = diamond(nx, ny, nz, 5.432)
        s = vacancies(s, 0.05, rng)
        s = displace_gaussian(s, 0.05, rng)
        s = maxwell_boltzmann(wrap(s), T, rng)
        s.meta = dict(name=("SiC" if sic else "Si") + f" {nx}x{ny}x{nz}", T=T)
        if rate:
            t += float(rng.exponential(1.0 / rate))
        jobs.append(Job(arrival=t, system=s, steps=steps, dt=0.5e-3 if sic else 1e-3))
    return jobs
