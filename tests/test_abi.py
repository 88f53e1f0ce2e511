"""The C-ABI library loads and exports every symbol include/tersoff.h declares;
host-side argument handling works without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(tersoff_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_00882_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tersoff_ctx_create", "tersoff_params_create", "tersoff_neighbor_build", "tersoff_compute",
              "tersoff_md_create", "tersoff_md_step", "tersoff_md_run"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1710_00882_gb300", "libtersoff.so")],
                         capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert set(declared_functions()) <= exported


def test_binding_names_match_header():
    from paper_1710_00882_gb300 import tersoff as t
    for n in declared_functions():
        assert hasattr(t, n), n


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1710_00882_gb300 import tersoff as t
    assert t.tersoff_ctx_create(0, None, None) == t.ERR_ARG
    assert t.tersoff_params_create(None, 1, None, None, None) == t.ERR_ARG
    assert t.tersoff_compute(None, None, None, 0, None, None, None, 0, 0, None, None, None) == t.ERR_ARG
    assert t.tersoff_md_step(None, 1, None) == t.ERR_ARG
    assert t.tersoff_neighbor_build_typed(None, None, None, 0, None, None, 0.3, 0, None) == t.ERR_ARG
    assert t.tersoff_version().startswith(b"tersoff-gb300")


def test_precision_values_match_header():
    """The binding's precision constants are the header's enum values."""
    from paper_1710_00882_gb300 import tersoff as t
    src = open(os.path.join(ROOT, "include", "tersoff.h")).read()
    m = re.search(r"typedef enum \{([^}]*)\} tersoff_precision;", src)
    vals = dict((k.strip(), int(v)) for k, v in re.findall(r"TERSOFF_(\w+)\s*=\s*(\d+)", m.group(1)))
    assert vals == {"FP64": t.FP64, "MIXED": t.MIXED, "SINGLE": t.SINGLE}


def test_ctx_create_fails_cleanly_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1710_00882_gb300 import tersoff as t
    h = ctypes.c_void_p()
    assert t.tersoff_ctx_create(0, None, ctypes.byref(h)) == t.ERR_CUDA
    assert not h.value


def test_product_table_layout():
    """Row (i, j, k) of the product's table: angular constants of i, pair constants of
    (i, j), cutoff of (i, k)."""
    from paper_1710_00882_gb300 import params as pp
    tab, m = pp.for_species(("Si", "C"))
    t = tab.reshape(2, 2, 2, 14)
    assert t.shape == (2, 2, 2, 14) and list(m) == [28.0855, 12.011]
    assert t[1, 0, 1, 3] == pp.CARBON.c and t[0, 1, 1, 3] == pp.SILICON.c
    assert np.isclose(t[0, 1, 0, 13], np.sqrt(pp.SILICON.A * pp.CARBON.A))
    assert np.isclose(t[0, 1, 0, 10], 2.85) and np.isclose(t[0, 1, 1, 11], (np.sqrt(6.3) - np.sqrt(4.86)) / 2)
    # pair cutoffs symmetric (the C ABI requires it)
    assert t[0, 1, 1, 10] == t[1, 0, 0, 10] and t[0, 1, 1, 11] == t[1, 0, 0, 11]


def test_server_null_arguments_rejected_without_gpu(lib):
    from paper_1710_00882_gb300 import tersoff as t
    assert t.tersoff_server_create(None, None, 0, 0.3, 1 << 20, 4, 10, None) == t.ERR_ARG
    assert t.tersoff_server_submit(None, None, None) == t.ERR_ARG
    assert t.tersoff_server_poll(None, 1, None) == t.ERR_ARG
    assert t.tersoff_server_wait(None, 1, 0.0) == t.ERR_ARG
    assert t.tersoff_server_result(None, 1, None, None, None, None) == t.ERR_ARG
    assert t.tersoff_server_get_stats(None, None) == t.ERR_ARG
    assert t.tersoff_server_last_error(None) == b"null server"
    t.tersoff_server_destroy(None)


def test_server_struct_layout_matches_header(tmp_path):
    """The binding's ctypes structures have the C compiler's sizes and offsets."""
    from paper_1710_00882_gb300 import tersoff as t
    src = tmp_path / "layout.c"
    fields_job = [f for f, _ in t.tersoff_job._fields_]
    fields_st = [f for f, _ in t.tersoff_server_stats._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tersoff.h"', "int main(void) {",
             'printf("%zu\\n", sizeof(tersoff_job));']
    lines += [f'printf("%zu\\n", offsetof(tersoff_job, {f}));' for f in fields_job]
    lines += ['printf("%zu\\n", sizeof(tersoff_server_stats));']
    lines += [f'printf("%zu\\n", offsetof(tersoff_server_stats, {f}));' for f in fields_st]
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(t.tersoff_job)] + [getattr(t.tersoff_job, f).offset for f in fields_job]
    want += [ctypes.sizeof(t.tersoff_server_stats)] + [getattr(t.tersoff_server_stats, f).offset for f in fields_st]
    assert got == want
