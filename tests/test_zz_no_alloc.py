"""tersoff_compute_noalloc: the evaluation for callers that may not allocate device
memory while they run (for example next to a framework allocator that already
reserved the GPU, or inside a loop where cudaMalloc would synchronize the device).
Its working buffers live in one fixed array inside the library.  Called through
the C ABI with device buffers, two calls in a row must give what tersoff_compute
gives, within the tolerances of the parity tests; sizes beyond the fixed limit are
refused before any GPU work.  Collected last so that a failure here comes after
every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1710_00882_gb300 import workloads as wl

from gpu_common import FP64_E_REL, FP64_F_ABS, MIX_E_REL, MIX_F_ABS, SGL_E_REL, SGL_F_ABS, product_params

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


def noalloc(T, P, s, prec):
    """One call through the C ABI on device buffers; returns (E, W[6], F[N,3]) on the host."""
    import torch
    dev = torch.device("cuda:0")
    pos = torch.as_tensor(np.ascontiguousarray(s.pos), dtype=torch.float64, device=dev)
    types = torch.as_tensor(np.ascontiguousarray(s.types, dtype=np.int32), device=dev)
    ev = torch.full((7,), float("nan"), dtype=torch.float64, device=dev)
    F = torch.full((s.n, 3), float("nan"), dtype=torch.float64, device=dev)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = T.tersoff_compute_noalloc(P.h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(types.data_ptr()), s.n,
                                   box.ctypes.data_as(ctypes.c_void_p), int(prec), ctypes.c_void_p(stream),
                                   ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(F.data_ptr()), err, 256)
    assert rc == T.OK, err.value.decode()
    ev = ev.cpu().numpy()
    return ev[0], ev[1:], F.cpu().numpy()


CASES = [
    ("si_512", lambda: wl.si_512(), ("Si",)),
    ("sic_ragged", lambda: wl.sic_box(3, seed=12), ("Si", "C")),
    ("si_box_5x4x3", lambda: wl.si_box(5, 4, 3, seed=13), ("Si",)),
]


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
def test_noalloc_matches_compute_twice(T, ctx, prec_name):
    prec = getattr(T, prec_name)
    e_rel, f_abs = {T.FP64: (FP64_E_REL, FP64_F_ABS), T.MIXED: (MIX_E_REL, MIX_F_ABS),
                    T.SINGLE: (SGL_E_REL, SGL_F_ABS)}[prec]
    # the cases run one after another, so each call finds the previous call's data in the array
    for name, make, species in CASES:
        s = make()
        P = product_params(ctx, species)
        E0, F0, W0 = T.compute(ctx, P, s.pos, s.types, s.box, prec=prec)
        for call in range(2):
            E, W, F = noalloc(T, P, s, prec)
            assert abs(E - E0) <= e_rel * abs(E0), f"{name} call {call}: energy {E!r} vs {E0!r}"
            assert np.abs(F - F0).max() <= f_abs, f"{name} call {call}: force err {np.abs(F - F0).max():.3e}"
            wtol = max(1e-10 * s.n, e_rel * np.abs(W0).max())
            assert np.abs(W - W0).max() <= wtol, f"{name} call {call}: virial {W} vs {W0}"


def test_noalloc_refuses_sizes_beyond_the_limit(T, ctx):
    P = product_params(ctx, ("Si",))
    n = T.NOALLOC_MAX_ATOMS + 1
    box = np.full(3, 100.0)
    err = ctypes.create_string_buffer(256)
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    rc = T.tersoff_compute_noalloc(P.h, dummy, dummy, n, box.ctypes.data_as(ctypes.c_void_p), int(T.FP64), None,
                                   None, None, err, 256)
    assert rc == T.ERR_NOMEM
    assert b"exceeds the fixed scratch limit" in err.value
