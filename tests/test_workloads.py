"""The seeded input generators follow the recipe the workloads are stated with:
atom and site counts, box sizes, displacement laws, exact initial temperature
with zero total momentum, vacancy counts, and the serving stream's species,
size, temperature, step and arrival distributions.  CPU only."""
import numpy as np
import pytest

from paper_1710_00882_gb300 import workloads as wl


def site_offsets(s, sites):
    """Minimum-image displacement of each atom from its lattice site."""
    d = s.pos - sites
    return d - s.box * np.round(d / s.box)


def test_si_512_recipe():
    s = wl.si_512()
    lat = wl.diamond(4, 4, 4, 5.432)
    assert s.n == 512 and s.species == ("Si",)
    assert np.allclose(s.box, 4 * 5.432)
    off = site_offsets(s, lat.pos)
    assert np.abs(off).max() <= 0.05 and np.abs(off).max() > 0.045   # uniform on [-0.05, 0.05]
    assert abs(off.mean()) < 0.005
    assert np.all((s.pos >= 0) & (s.pos < s.box))
    assert s.vel is None


@pytest.mark.parametrize("make,cells,T", [(wl.si_32k, (20, 20, 10), 1000.0), (wl.si_512k, (40, 40, 40), 1000.0)])
def test_thermal_si_boxes_recipe(make, cells, T):
    s = make()
    lat = wl.diamond(*cells, 5.432)
    assert s.n == 8 * int(np.prod(cells))
    assert np.allclose(s.box, np.array(cells) * 5.432)
    off = site_offsets(s, lat.pos)
    assert abs(off.std() - 0.05) < 0.002 and abs(off.mean()) < 0.001   # Gaussian sigma 0.05 A
    m = s.masses()[s.types]
    p = (m[:, None] * s.vel).sum(axis=0)
    assert np.abs(p).max() <= 1e-9 * (m[:, None] * np.abs(s.vel)).sum()
    assert wl.temperature(s.vel, s.types, s.masses()) == pytest.approx(T, rel=1e-12)
    assert np.all((s.pos >= 0) & (s.pos < s.box))


def test_sic_950k_recipe():
    s = wl.sic_1m()
    sites = 8 * 50 ** 3
    assert s.n == sites - sites // 20 == 950_000
    assert s.species == ("Si", "C") and np.allclose(s.box, 50 * 4.36)
    n_si, n_c = int((s.types == 0).sum()), int((s.types == 1).sum())
    assert n_si + n_c == s.n and abs(n_si - n_c) < 2000           # half the 50,000 vacancies on each sublattice
    assert wl.temperature(s.vel, s.types, s.masses()) == pytest.approx(1500.0, rel=1e-12)
    assert s.meta["dt"] == 0.5e-3


def test_vacancies_remove_floor_fraction_by_seed():
    base = wl.diamond(3, 3, 3, 4.36, species=("Si", "C"))
    a = wl.vacancies(wl.diamond(3, 3, 3, 4.36, species=("Si", "C")), 0.05, np.random.default_rng(9))
    b = wl.vacancies(wl.diamond(3, 3, 3, 4.36, species=("Si", "C")), 0.05, np.random.default_rng(9))
    assert a.n == base.n - int(np.floor(0.05 * base.n))
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.types, b.types)
    # the kept atoms are sites of the lattice, in lattice order
    idx = [int(np.flatnonzero(np.all(base.pos == p, axis=1))[0]) for p in a.pos]
    assert idx == sorted(idx)


@pytest.mark.parametrize("min_cells", [1, 2])
def test_cells_for_atoms_is_the_closest_box(min_cells):
    for target in list(range(8, 400, 7)) + [1000.0, 5000.0, 16384.0, 777.7]:
        nx, ny, nz = wl.cells_for_atoms(target, min_cells)
        assert min_cells <= nx <= ny <= nz
        best = min(abs(8 * a * b * c - target)
                   for a in range(min_cells, 40) for b in range(a, 40) for c in range(b, 300))
        assert abs(8 * nx * ny * nz - target) == best, (target, (nx, ny, nz))


def test_serving_stream_recipe():
    jobs = wl.serving_stream(600, seed=5)
    again = wl.serving_stream(600, seed=5)
    assert all(np.array_equal(a.system.pos, b.system.pos) and a.steps == b.steps for a, b in zip(jobs, again))
    sic = np.array([j.system.species == ("Si", "C") for j in jobs])
    assert abs(sic.mean() - 0.5) < 0.07                                  # 50/50 species
    assert all(j.dt == (0.5e-3 if s else 1e-3) for j, s in zip(jobs, sic))
    steps = np.array([j.steps for j in jobs])
    assert steps.min() >= 50 and steps.max() <= 500 and abs(steps.mean() - 275) < 15
    n = np.array([j.system.n for j in jobs])
    assert n.min() >= 64 * 0.9 * 0.95 and n.max() <= 16384 * 1.1
    # log-uniform sizes: log n spread evenly over [log 64, log 16384]
    u = (np.log(n) - np.log(64)) / (np.log(16384) - np.log(64))
    assert abs(u.mean() - 0.5) < 0.05 and abs(np.mean(u < 0.25) - 0.25) < 0.06
    for j in jobs:
        s = j.system
        cells = np.round(s.box / (4.36 if s.species == ("Si", "C") else 5.432)).astype(int)
        assert cells.min() >= 2
        sites = 8 * int(np.prod(cells))
        assert s.n == sites - int(np.floor(0.05 * sites))                # 5% vacancies
        T = wl.temperature(s.vel, s.types, s.masses())
        assert T == pytest.approx(s.meta["T"], rel=1e-10) and 300.0 <= T <= 2000.0
        assert j.arrival == 0.0                                           # closed loop without a rate


def test_serving_stream_poisson_arrivals():
    jobs = wl.serving_stream(400, seed=11, rate=200.0, max_atoms=512)
    t = np.array([j.arrival for j in jobs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.15 / 200.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15                   # exponential: cv = 1
