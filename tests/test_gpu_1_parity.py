"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 energy rel <= 1e-12, force max-abs <= 1e-10 eV/A; mixed
energy rel <= 1e-6, force max-abs <= 1e-4 eV/A (the accuracy targets the
workloads are specified with); single (float32 throughout) energy rel <= 1e-5,
force max-abs <= 1e-3 eV/A (derived in gpu_common).  Virial: 1e-10 (FP64) / 1e-5
(mixed) / 1e-4 (single) eV per atom.  Every case uses these bounds except the one
stress case whose forces (up to 80 eV/A) are four times the workloads' scale: there
the float32 bounds scale with max|F| (gpu_common.force_scale).
"""
import numpy as np
import pytest

from oracle import oracle, params as oparams
from paper_1710_00882_gb300 import workloads as wl

from gpu_common import (FP64_E_REL, FP64_F_ABS, FP64_W_ATOM, MIX_E_REL, MIX_F_ABS, MIX_W_ATOM, SGL_E_REL, SGL_F_ABS,
                        SGL_W_ATOM, assert_parity, force_scale, oracle_table, product_params)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_1710_00882_gb300 import tersoff
    return tersoff


@pytest.fixture(scope="module")
def ctx(T):
    return T.Context(0)


def run_pair(T, ctx, s, species=None, prec=None, **kw):
    species = species or s.species
    P = product_params(ctx, species, **kw)
    tab, _ = oracle_table(species, **kw)
    Eo, Fo, Wo = oracle.energy_forces(s.pos, s.types, s.box, tab)
    out = {}
    for p in ([prec] if prec is not None else [T.FP64, T.MIXED, T.SINGLE]):
        E, F, W = T.compute(ctx, P, s.pos, s.types, s.box, prec=p)
        out[p] = (E, F, W)
    return out, (Eo, Fo, Wo)


def check(T, out, ref, what, f_scale=1.0, w_scale=1.0):
    """Every precision against the oracle at its bounds; f_scale, w_scale (>= 1) widen
    the float32 force and virial bounds of stress cases beyond the workloads' force
    scale."""
    Eo, Fo, Wo = ref
    if T.FP64 in out:
        E, F, W = out[T.FP64]
        assert_parity(E, F, W, Eo, Fo, Wo, FP64_E_REL, FP64_F_ABS, FP64_W_ATOM, what + " fp64")
    if T.MIXED in out:
        E, F, W = out[T.MIXED]
        assert_parity(E, F, W, Eo, Fo, Wo, MIX_E_REL, f_scale * MIX_F_ABS, w_scale * MIX_W_ATOM, what + " mixed")
    if T.SINGLE in out:
        E, F, W = out[T.SINGLE]
        assert_parity(E, F, W, Eo, Fo, Wo, SGL_E_REL, f_scale * SGL_F_ABS, w_scale * SGL_W_ATOM, what + " single")


def test_si_512_config(T, ctx):
    """512-atom Si diamond, uniform +-0.05 A displacements: the single-evaluation workload."""
    s = wl.si_512()
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "si512")


def test_sic_ragged_with_vacancies(T, ctx):
    """3C-SiC 4^3 cells with vacancies (N = 487, not a multiple of any block), 1500 K
    displacements: skin-dominated lists, two types, Si-Si pairs in the taper."""
    s = wl.sic_box(4, seed=41, T=1500.0, sigma=0.08)
    assert s.n % 32 != 0
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "sic")


@pytest.mark.parametrize("lam3,m", [(1.3, 1), (1.1, 3)])
def test_lambda3_variants(T, ctx, lam3, m):
    s = wl.sic_box(3, seed=42, T=2000.0, sigma=0.1)
    out, ref = run_pair(T, ctx, s, lambda3=lam3, m=m)
    check(T, out, ref, f"lam3={lam3},m={m}")


def test_compressed_many_neighbours(T, ctx):
    """Si compressed to a = 4.1 A with displacements: the second shell (2.90 A) sits in
    the f_C taper, ~16 in-cutoff neighbours per atom, exercises the wider slot kernels.
    Forces reach 78 eV/A, yet the workloads' absolute force bounds hold (measured mixed
    error 2.2e-5 eV/A); the virial, a sum of terms four times the workloads' size, takes
    the force-scaled bound (measured mixed error 1.8e-3 eV over 216 atoms)."""
    rng = np.random.default_rng(5)
    s = wl.diamond(3, 3, 3, 4.1)
    s.pos = s.pos + rng.normal(0, 0.12, size=s.pos.shape)
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "compressed", w_scale=force_scale(ref[1]))


def test_more_than_32_neighbours(T, ctx):
    """Si compressed to a = 2.9 A: 33-35 in-cutoff neighbours per atom, so every atom
    leaves the register kernel for the warp kernel with two slots per lane.  Energy and
    forces.  The nearest neighbours sit at 1.26 A, deep in the repulsive wall: single
    terms reach ~200 eV/A and forces 80 eV/A, four times the workloads' force scale, so
    the float32 force bounds scale with max|F| / 20 eV/A (measured mixed error 1.1e-4
    eV/A against a scaled bound of 4e-4)."""
    rng = np.random.default_rng(12)
    s = wl.diamond(4, 4, 4, 2.9)
    s.pos = s.pos + rng.normal(0, 0.03, size=s.pos.shape)
    P = product_params(ctx, s.species)
    nl = T.NeighborList(ctx, s.pos, s.box, P.cutoff, 0.0)
    counts, _ = nl.get()
    assert counts.min() > 32
    tab, _ = oracle_table(s.species)
    Eo, Fo, _ = oracle.energy_forces(s.pos, s.types, s.box, tab)
    sc = force_scale(Fo)
    assert sc > 3.5
    for prec, er, fa in ((T.FP64, FP64_E_REL, FP64_F_ABS), (T.MIXED, MIX_E_REL, sc * MIX_F_ABS),
                         (T.SINGLE, SGL_E_REL, sc * SGL_F_ABS)):
        E, F, _ = T.compute(ctx, P, s.pos, s.types, s.box, prec=prec)
        assert_parity(E, F, None, Eo, Fo, None, er, fa, 0, f"dense prec {prec}")


def test_two_cells_per_side(T, ctx):
    """Smallest legal boxes: 2 cells per side (box < 3 * r_list)."""
    s = wl.sic_box(2, seed=43, T=1000.0)
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "sic2")
    s = wl.si_box(2, 2, 2, seed=44, T=1000.0)
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "si2")


def test_positions_outside_box(T, ctx):
    s = wl.si_box(3, 3, 3, seed=45, T=1000.0)
    rng = np.random.default_rng(0)
    s.pos = s.pos + s.box * rng.integers(-3, 4, size=s.pos.shape)
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "unwrapped")


def test_edge_cases(T, ctx):
    P = product_params(ctx, ("Si",))
    box = np.array([20.0, 20.0, 20.0])
    # empty system
    E, F, W = T.compute(ctx, P, np.zeros((0, 3)), np.zeros(0, np.int32), box)
    assert E == 0.0 and F.shape == (0, 3) and np.all(W == 0)
    # isolated atom, dimer (zeta = 0 path), trimer
    for pos in ([[1.0, 2.0, 3.0]], [[5.0, 5.0, 5.0], [7.35, 5.0, 5.0]],
                [[5.0, 5.0, 5.0], [7.3, 5.0, 5.0], [4.2, 7.2, 5.0]]):
        pos = np.array(pos)
        types = np.zeros(len(pos), np.int32)
        Eo, Fo, Wo = oracle.energy_forces(pos, types, box, oracle_table(("Si",))[0])
        # the workloads' bounds hold for a lone bond too (its energy f_R + f_A is ~5x
        # smaller than its two terms; measured mixed error 1.2e-7, single 8.4e-7)
        for prec, (er, fa, wa) in ((T.FP64, (FP64_E_REL, FP64_F_ABS, FP64_W_ATOM)),
                                   (T.MIXED, (MIX_E_REL, MIX_F_ABS, MIX_W_ATOM)),
                                   (T.SINGLE, (SGL_E_REL, SGL_F_ABS, SGL_W_ATOM))):
            E, F, W = T.compute(ctx, P, pos, types, box, prec=prec)
            if Eo == 0.0:
                assert E == 0.0 and np.all(F == 0)
            else:
                assert_parity(E, F, W, Eo, Fo, Wo, er, fa, wa)


def test_errors_are_reported(T, ctx):
    P = product_params(ctx, ("Si",))
    s = wl.si_box(2, 2, 2, seed=46, T=300.0)
    with pytest.raises(T.TersoffError) as e:
        T.compute(ctx, P, s.pos, np.full(s.n, 3, np.int32), s.box)
    assert e.value.code == T.ERR_ARG
    with pytest.raises(T.TersoffError) as e:
        T.compute(ctx, P, s.pos[:10], s.types[:10], np.array([5.0, 20.0, 20.0]))
    assert e.value.code == T.ERR_BOX_TOO_SMALL
    bad = s.pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(T.TersoffError) as e:
        T.compute(ctx, P, bad, s.types, s.box)
    assert e.value.code == T.ERR_NONFINITE
    # the context stays usable after errors
    E, F, W = T.compute(ctx, P, s.pos, s.types, s.box)
    assert np.isfinite(E)


def test_deterministic(T, ctx):
    s = wl.sic_box(5, seed=47, T=1500.0)
    P = product_params(ctx, s.species)
    for prec in (T.FP64, T.MIXED, T.SINGLE):
        E1, F1, W1 = T.compute(ctx, P, s.pos, s.types, s.box, prec=prec)
        E2, F2, W2 = T.compute(ctx, P, s.pos, s.types, s.box, prec=prec)
        assert np.array_equal(F1, F2)


def test_device_pointers(T, ctx):
    import torch
    s = wl.si_box(4, 4, 4, seed=48, T=1000.0)
    P = product_params(ctx, s.species)
    pos = torch.tensor(s.pos, device="cuda")
    types = torch.tensor(s.types, device="cuda")
    E, F, W = T.compute(ctx, P, pos, types, s.box, prec=T.FP64)
    Eh, Fh, Wh = T.compute(ctx, P, s.pos, s.types, s.box, prec=T.FP64)
    assert E == Eh and np.array_equal(F.cpu().numpy(), Fh)


def test_given_neighbor_list_with_skin(T, ctx):
    """A list built with skin 0.3 A stays valid for displacements below skin/2."""
    s = wl.si_box(5, 5, 5, seed=49, T=1000.0)
    P = product_params(ctx, s.species)
    nl = T.NeighborList(ctx, s.pos, s.box, P.cutoff, 0.3)
    rng = np.random.default_rng(1)
    moved = s.pos + rng.uniform(-0.08, 0.08, size=s.pos.shape)
    tab, _ = oracle_table(s.species)
    Eo, Fo, Wo = oracle.energy_forces(moved, s.types, s.box, tab)
    E, F, W = T.compute(ctx, P, moved, s.types, s.box, prec=T.FP64, nlist=nl)
    assert_parity(E, F, W, Eo, Fo, Wo, FP64_E_REL, FP64_F_ABS, 1e-10, "given list")


@pytest.mark.parametrize("seed,box_cells,skin", [(1, 2, 0.3), (2, 3, 0.0), (3, 5, 0.5), (4, 2, 1.2)])
def test_neighbor_list_equals_brute_force(T, ctx, seed, box_cells, skin):
    s = wl.sic_box(box_cells, seed=seed, T=2000.0)
    rc = 3.0
    nl = T.NeighborList(ctx, s.pos, s.box, rc, skin)
    counts, idx = nl.get()
    off, oidx = oracle.neighbors(s.pos, s.box, rc + skin, method="brute")
    # the GPU list may also hold pairs within a relative 1e-5 above r_list
    for i in range(s.n):
        got = set(idx[i, :counts[i]].tolist())
        want = set(oidx[off[i]:off[i + 1]].tolist())
        assert want <= got
        for j in got - want:
            dj = np.linalg.norm((s.pos[j] - s.pos[i] + s.box / 2) % s.box - s.box / 2)
            assert dj < (rc + skin) * (1 + 1e-5)
        assert list(idx[i, :counts[i]]) == sorted(got)


@pytest.mark.parametrize("seed,cells,skin", [(5, 2, 0.3), (6, 4, 0.3), (7, 3, 0.0), (8, 5, 0.8)])
def test_typed_neighbor_list_equals_brute_force(T, ctx, seed, cells, skin):
    """Lists with one radius per type pair (the list the MD driver, the server and
    tersoff_compute build): j is listed for i exactly when the minimum-image distance
    is below r_C(t_i, t_j) + skin, with r_C = R + D from the oracle's own table."""
    s = wl.sic_box(cells, seed=seed, T=2000.0)
    P = product_params(ctx, s.species)
    tab, _ = oracle_table(s.species)
    nt = 2
    rows = np.asarray(tab).reshape(nt, nt, nt, -1)
    f_r, f_d = oparams.FIELDS.index("R"), oparams.FIELDS.index("D")
    rc = np.array([[rows[a, b, b, f_r] + rows[a, b, b, f_d] for b in range(nt)] for a in range(nt)])
    nl = T.NeighborList(ctx, s.pos, s.box, None, skin, types=s.types, params=P)
    counts, idx = nl.get()
    d = s.pos[None, :, :] - s.pos[:, None, :]
    d -= s.box * np.round(d / s.box)
    r = np.linalg.norm(d, axis=2)
    lim = rc[s.types[:, None], s.types[None, :]] + skin
    np.fill_diagonal(r, np.inf)
    for i in range(s.n):
        got = idx[i, :counts[i]]
        want = np.nonzero(r[i] < lim[i])[0]
        extra = set(got.tolist()) - set(want.tolist())
        assert set(want.tolist()) <= set(got.tolist()), f"atom {i}: missing {set(want.tolist()) - set(got.tolist())}"
        # float32 decisions with the build's 1e-5 relative margin
        assert all(r[i, j] < lim[i, j] * (1 + 1e-5) for j in extra), f"atom {i}: extra {extra}"
        assert list(got) == sorted(got)
    # C atoms keep only their Si neighbours: the C-C second shell (3.08 A, thermal
    # spread ~0.1 A) lies well beyond r_C(C,C) + skin = 2.1 + skin for skin <= 0.3 A
    if skin <= 0.3:
        cnt_c = counts[s.types == 1]
        assert cnt_c.max() <= 4 and cnt_c.mean() > 3.5
    # and the typed list gives the oracle's energy and forces
    Eo, Fo, Wo = oracle.energy_forces(s.pos, s.types, s.box, tab)
    E, F, W = T.compute(ctx, P, s.pos, s.types, s.box, prec=T.FP64, nlist=nl)
    assert_parity(E, F, W, Eo, Fo, Wo, FP64_E_REL, FP64_F_ABS, 1e-10, "typed list")


@pytest.mark.slow
def test_full_size_si_512k(T, ctx):
    """The 512,000-atom Si box at its full size, in the launch configuration the bench times:
    every force and the energy against the oracle."""
    s = wl.si_512k()
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "si512k")


@pytest.mark.slow
def test_full_size_sic_950k(T, ctx):
    """The 3C-SiC box at full size (950,000 atoms), in all three precisions, against the oracle."""
    s = wl.sic_1m()
    out, ref = run_pair(T, ctx, s)
    check(T, out, ref, "sic950k")


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
def test_register_and_general_kernels_agree(T, prec_name, monkeypatch):
    """The register kernel (unordered neighbour pairs, overflow queue) and the general
    kernel (ordered pairs, shared-memory slots) on a SiC box where Si atoms exceed 8
    in-cutoff neighbours: same forces within rounding."""
    prec = getattr(T, prec_name)
    s = wl.sic_box(6, seed=50, T=2500.0, sigma=0.1)
    c1 = T.Context(0)
    P1 = product_params(c1, s.species)
    E1, F1, W1 = T.compute(c1, P1, s.pos, s.types, s.box, prec=prec)
    monkeypatch.setenv("TERSOFF_FORCE_KERNEL", "general")
    c2 = T.Context(0)
    P2 = product_params(c2, s.species)
    E2, F2, W2 = T.compute(c2, P2, s.pos, s.types, s.box, prec=prec)
    if prec == T.FP64:
        assert abs(E1 - E2) <= 1e-13 * abs(E2) and np.abs(F1 - F2).max() < 1e-11
    elif prec == T.MIXED:
        assert abs(E1 - E2) <= 1e-6 * abs(E2) and np.abs(F1 - F2).max() < 1e-4
    else:
        assert abs(E1 - E2) <= 1e-5 * abs(E2) and np.abs(F1 - F2).max() < 1e-3


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
@pytest.mark.parametrize("case", ["si", "sic"])
def test_type_specialised_and_generic_tables_agree(T, prec_name, case, monkeypatch):
    """The register kernel with its table in the kernel argument (one type: Si; two
    types: SiC, lambda3 = 0) and with the shared-memory table every table can use
    (TERSOFF_FORCE_TABLE=generic): the same terms, so the same forces within rounding,
    and both match the oracle."""
    prec = getattr(T, prec_name)
    s = wl.si_box(5, 4, 3, seed=51, T=1000.0) if case == "si" else wl.sic_box(4, seed=52, T=1500.0)
    c1 = T.Context(0)
    P1 = product_params(c1, s.species)
    E1, F1, W1 = T.compute(c1, P1, s.pos, s.types, s.box, prec=prec)
    monkeypatch.setenv("TERSOFF_FORCE_TABLE", "generic")
    c2 = T.Context(0)
    P2 = product_params(c2, s.species)
    E2, F2, W2 = T.compute(c2, P2, s.pos, s.types, s.box, prec=prec)
    tab, _ = oracle_table(s.species)
    Eo, Fo, Wo = oracle.energy_forces(s.pos, s.types, s.box, tab)
    er, fa, wa = {T.FP64: (FP64_E_REL, FP64_F_ABS, FP64_W_ATOM), T.MIXED: (MIX_E_REL, MIX_F_ABS, MIX_W_ATOM),
                  T.SINGLE: (SGL_E_REL, SGL_F_ABS, SGL_W_ATOM)}[prec]
    assert_parity(E1, F1, W1, Eo, Fo, Wo, er, fa, wa, f"{case} kernel-argument table")
    assert_parity(E2, F2, W2, Eo, Fo, Wo, er, fa, wa, f"{case} generic table")
    assert_parity(E1, F1, W1, E2, F2, W2, er, fa, wa, f"{case} tables agree")
