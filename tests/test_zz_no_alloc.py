"""tersoff_compute_noalloc: the evaluation for callers that may not allocate device
memory while they run (for example next to a framework allocator that already
reserved the GPU, or inside a loop where cudaMalloc would synchronize the device).
Its working buffers live in one fixed array inside the library.

Checked through the C ABI with device buffers:
- two calls in a row give bitwise the same energy, virial and forces (the second call
  finds the first call's data in the shared array and must not depend on it);
- the result matches the FP64 oracle within the parity tests' tolerances, and
  tersoff_compute within the same tolerances;
- free device memory does not change across calls (nothing is allocated);
- a system with more than 32 neighbours within the cutoff is refused with
  TERSOFF_ERR_NLIST_OVERFLOW, read from the device status word, and the next call
  on a normal system is correct again;
- sizes beyond the fixed limit are refused before any GPU work.
Collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_1710_00882_gb300 import workloads as wl

from gpu_common import (FP64_E_REL, FP64_F_ABS, MIX_E_REL, MIX_F_ABS, SGL_E_REL, SGL_F_ABS, assert_parity,
                        oracle_table, product_params)

pytestmark = pytest.mark.gpu

TOL = {"FP64": (FP64_E_REL, FP64_F_ABS, 1e-10), "MIXED": (MIX_E_REL, MIX_F_ABS, 1e-5),
       "SINGLE": (SGL_E_REL, SGL_F_ABS, 1e-4)}


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_1710_00882_gb300 import tersoff
    return tersoff


@pytest.fixture(scope="module")
def ctx(T):
    return T.Context(0)


class DeviceCase:
    """Device input and output buffers of one system, allocated before any call."""

    def __init__(self, s):
        import torch
        dev = torch.device("cuda:0")
        self.s = s
        self.pos = torch.as_tensor(np.ascontiguousarray(s.pos), dtype=torch.float64, device=dev)
        self.types = torch.as_tensor(np.ascontiguousarray(s.types, dtype=np.int32), device=dev)
        self.ev = torch.empty((7,), dtype=torch.float64, device=dev)
        self.F = torch.empty((s.n, 3), dtype=torch.float64, device=dev)
        self.box = np.ascontiguousarray(s.box, dtype=np.float64)
        self.stream = torch.cuda.current_stream(dev).cuda_stream

    def call(self, T, P, prec):
        """One call; returns (rc, message).  Outputs are poisoned with NaN first."""
        self.ev.fill_(float("nan"))
        self.F.fill_(float("nan"))
        err = ctypes.create_string_buffer(256)
        rc = T.tersoff_compute_noalloc(P.h, ctypes.c_void_p(self.pos.data_ptr()),
                                       ctypes.c_void_p(self.types.data_ptr()), self.s.n,
                                       self.box.ctypes.data_as(ctypes.c_void_p), int(prec),
                                       ctypes.c_void_p(self.stream), ctypes.c_void_p(self.ev.data_ptr()),
                                       ctypes.c_void_p(self.F.data_ptr()), err, 256)
        return rc, err.value.decode()

    def result(self):
        ev = self.ev.cpu().numpy()
        return ev[0], ev[1:].copy(), self.F.cpu().numpy()


CASES = [
    ("si_512", lambda: wl.si_512(), ("Si",)),
    ("sic_ragged", lambda: wl.sic_box(3, seed=12), ("Si", "C")),
    ("si_box_5x4x3", lambda: wl.si_box(5, 4, 3, seed=13), ("Si",)),
]


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED", "SINGLE"])
def test_noalloc_twice_matches_oracle_and_compute(T, ctx, prec_name):
    import torch
    prec = getattr(T, prec_name)
    e_rel, f_abs, w_abs = TOL[prec_name]
    cases = [(name, DeviceCase(make()), species) for name, make, species in CASES]
    params = {species: product_params(ctx, species) for _, _, species in CASES}
    # a first call of each case loads the kernels; nothing after it may allocate
    for name, dc, species in cases:
        rc, msg = dc.call(T, params[species], prec)
        assert rc == T.OK, msg
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # the cases run one after another, so each call finds the previous call's data in the array
    results = {}
    for name, dc, species in cases:
        pair = []
        for call in range(2):
            rc, msg = dc.call(T, params[species], prec)
            assert rc == T.OK, f"{name} call {call}: {msg}"
            pair.append(dc.result())
        results[name] = pair
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "free device memory changed across no-allocation calls"
    for name, dc, species in cases:
        s = dc.s
        (E0, W0, F0), (E1, W1, F1) = results[name]
        assert E0 == E1 and np.array_equal(W0, W1) and np.array_equal(F0, F1), f"{name}: calls differ"
        tab, _ = oracle_table(species)
        Eo, Fo, Wo = oracle.energy_forces(s.pos, s.types, s.box, tab)
        assert_parity(E1, F1, W1, Eo, Fo, Wo, e_rel, f_abs, w_abs, f"{name} {prec_name} vs oracle")
        Ec, Fc, Wc = T.compute(ctx, params[species], s.pos, s.types, s.box, prec=prec)
        assert_parity(E1, F1, W1, Ec, Fc, Wc, e_rel, f_abs, w_abs, f"{name} {prec_name} vs tersoff_compute")


def test_noalloc_neighbour_overflow_then_normal_call(T, ctx):
    """Si compressed to a = 2.9 A has 33-35 atoms within the cutoff of every atom, more
    than the fixed list holds: the build sets the device status word, the force kernel
    stops at its first line, and the call returns TERSOFF_ERR_NLIST_OVERFLOW.  The next
    call on a normal system clears the status and matches the oracle."""
    rng = np.random.default_rng(12)
    dense = wl.diamond(4, 4, 4, 2.9)
    dense.pos = dense.pos + rng.normal(0, 0.03, size=dense.pos.shape)
    P = product_params(ctx, ("Si",))
    dd = DeviceCase(dense)
    rc, msg = dd.call(T, P, T.MIXED)
    assert rc == T.ERR_NLIST_OVERFLOW, (rc, msg)
    assert "exceed the fixed limit" in msg
    s = wl.si_512()
    dc = DeviceCase(s)
    rc, msg = dc.call(T, P, T.MIXED)
    assert rc == T.OK, msg
    E, W, F = dc.result()
    tab, _ = oracle_table(("Si",))
    Eo, Fo, Wo = oracle.energy_forces(s.pos, s.types, s.box, tab)
    assert_parity(E, F, W, Eo, Fo, Wo, MIX_E_REL, MIX_F_ABS, 1e-5, "after overflow")


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
