"""The counts behind the force kernel's algorithmic flop figure (bench.py): on a
perfect diamond Si lattice every atom has 4 list entries within r_C + skin (the
second shell, 3.84 A, lies beyond 3.3 A), 4 in-cutoff neighbours, none in the f_C
taper (2.35 A < R - D = 2.7 A) and 4 * 3 = 12 ordered triplets.  CPU only."""
import numpy as np
import pytest

import bench
from paper_1710_00882_gb300 import workloads as wl


def test_perfect_diamond_counts():
    pytest.importorskip("scipy")
    s = wl.diamond(5, 5, 5, 5.432)
    n_list, P, P_taper, P_short, T = bench.workload_counts(s, 3.0, 2.7, 1.995)
    assert (n_list, P, P_taper, P_short, T) == (4 * s.n, 4 * s.n, 0, 0, 12 * s.n)
    # every pair of a lattice compressed to a = 3.9 A (bonds of 1.69 A) is short
    c = wl.diamond(5, 5, 5, 3.9)
    _, Pc, _, Pc_short, _ = bench.workload_counts(c, 3.0, 2.7, 1.995)
    assert Pc_short == 4 * c.n and Pc > Pc_short


def test_flops_per_launch_for_si_512k_counts():
    """0.379 GFLOP of the method's own work per launch for the 512,000-atom box at the
    perfect-lattice counts (740 flops per atom), plus the mixed-mode compensation
    reported apart: 14 flops per pair (head+tail exponents; 28.7 MFLOP) with no pair in
    the taper or shorter than 0.7 R, 75 per pair where the geometry is head+tail too."""
    n = 512_000
    flops = bench.C_ENTRY * 4 * n + bench.C_PAIR * 4 * n + bench.C_TAPER * 0 + bench.C_TRIPLET * 12 * n
    assert flops == pytest.approx(0.379e9, rel=1e-3)
    assert flops / n == 740
    assert bench.C_PAIR_MIXED_EXP * 4 * n == pytest.approx(28.67e6, rel=1e-3)
    assert bench.C_PAIR_MIXED_EXP + bench.C_PAIR_MIXED_GEOM == 75


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    """The guard on the recorded ncu traffic changes with the kernel's code, not with
    its comments."""
    import os
    import shutil
    csrc = os.path.join(bench.ROOT, "paper_1710_00882_gb300", "csrc")
    root = tmp_path / "repo"
    dst = root / "paper_1710_00882_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("force_kernels.cuh", "force_mixed.cu", "internal.cuh"):
        shutil.copy(os.path.join(csrc, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.force_kernel_source_hash()
    k = (dst / "force_kernels.cuh").read_text()
    (dst / "force_kernels.cuh").write_text(k.replace("#pragma once", "// a new comment line\n#pragma once", 1))
    assert bench.force_kernel_source_hash() == h0
    (dst / "force_kernels.cuh").write_text(k.replace("constexpr float L2E_F = 1.44269502f;",
                                                     "constexpr float L2E_F = 1.44269503f;", 1))
    assert bench.force_kernel_source_hash() != h0


def test_committed_capture_is_of_the_current_kernel():
    """The DRAM traffic the bench line reports comes from the committed ncu capture of
    the mixed register kernel; it is reported only while that capture was taken with the
    kernel's current source (same hash), so a kernel change without a new capture shows
    here, before a bench run reports a null traffic."""
    assert bench.force_traffic() is not None
    assert bench.force_traffic() > 0
