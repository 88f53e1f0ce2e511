"""ctypes binding of libtersoff.so (include/tersoff.h).

The functions named ``tersoff_*`` mirror the C entry points one to one and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels.  The small classes below (Context, Params, NeighborList, MD, Server) own the
opaque handles and turn status codes into exceptions.

Arrays may be numpy arrays (host pointers) or CUDA torch tensors (device
pointers, TERSOFF_DEVICE_PTRS): the binding reads ``.ctypes.data`` or
``.data_ptr()`` and passes the pointer through.  There is no fallback: if the
library is missing, importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtersoff.so")

OK = 0
ERR_ARG = -1
ERR_NOMEM = -2
ERR_CUDA = -3
ERR_NLIST_OVERFLOW = -4
ERR_NONFINITE = -5
ERR_TIMEOUT = -6
ERR_BOX_TOO_SMALL = -7
ERR_BUSY = -8
ERR_NOT_FOUND = -9

FP64 = 0
MIXED = 1
SINGLE = 2

NOALLOC_MAX_ATOMS = 16384   # TERSOFF_NOALLOC_MAX_ATOMS

HOST_PTRS = 0
DEVICE_PTRS = 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtersoff.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                      "python paper_1710_00882_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


tersoff_version = _sig("tersoff_version", ctypes.c_char_p)
tersoff_ctx_create = _sig("tersoff_ctx_create", _I, _I, _P, _PP)
tersoff_ctx_destroy = _sig("tersoff_ctx_destroy", None, _P)
tersoff_last_error = _sig("tersoff_last_error", ctypes.c_char_p, _P)
tersoff_params_create = _sig("tersoff_params_create", _I, _P, _I, _P, _P, _PP)
tersoff_params_destroy = _sig("tersoff_params_destroy", None, _P)
tersoff_params_cutoff = _sig("tersoff_params_cutoff", _D, _P)
tersoff_neighbor_build = _sig("tersoff_neighbor_build", _I, _P, _P, _I64, _P, _D, _D, _I, _PP)
tersoff_neighbor_build_typed = _sig("tersoff_neighbor_build_typed", _I, _P, _P, _P, _I64, _P, _P, _D, _I, _PP)
tersoff_nlist_destroy = _sig("tersoff_nlist_destroy", None, _P)
tersoff_nlist_get = _sig("tersoff_nlist_get", _I, _P, _P, _P, _P, _P, _P)
tersoff_compute = _sig("tersoff_compute", _I, _P, _P, _P, _I64, _P, _P, _P, _I, _I, _P, _P, _P)
tersoff_md_create = _sig("tersoff_md_create", _I, _P, _P, _P, _P, _I64, _P, _P, _D, _D, _I, _I, _PP)
tersoff_md_step = _sig("tersoff_md_step", _I, _P, _I64, _P)
tersoff_md_step_async = _sig("tersoff_md_step_async", _I, _P, _I64)
tersoff_md_sync = _sig("tersoff_md_sync", _I, _P)
tersoff_md_get = _sig("tersoff_md_get", _I, _P, _P, _P, _P, _I)
tersoff_md_stats = _sig("tersoff_md_stats", _I, _P, _P, _P, _P)
tersoff_md_destroy = _sig("tersoff_md_destroy", None, _P)
tersoff_md_profile = _sig("tersoff_md_profile", _I, _P, _I)
tersoff_md_profile_read = _sig("tersoff_md_profile_read", _I, _P, _P, _P)
tersoff_md_run = _sig("tersoff_md_run", _I, _P, _P, _P, _P, _I64, _P, _P, _D, _I64, _D, _I, _I, _P)
tersoff_compute_noalloc = _sig("tersoff_compute_noalloc", _I, _P, _P, _P, _I64, _P, _I, _P, _P, _P, ctypes.c_char_p,
                               ctypes.c_size_t)


class tersoff_job(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("pos", _P), ("vel", _P), ("types", _P), ("box", ctypes.c_double * 3),
                ("dt_ps", ctypes.c_double), ("nsteps", ctypes.c_int64)]


class tersoff_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "admitted", "completed", "failed", "queued", "running",
                                              "atom_steps", "chunks", "repacks")] + \
               [("busy_s", ctypes.c_double), ("capacity_atoms", ctypes.c_int64)] + \
               [(k, ctypes.c_double) for k in ("retire_s", "repack_s", "graph_s", "run_s")] + \
               [("compactions", ctypes.c_int64), ("layout_fill", ctypes.c_double)]


_U64 = ctypes.c_uint64
tersoff_server_create = _sig("tersoff_server_create", _I, _P, _P, _I, _D, ctypes.c_size_t, _I, _I, _PP)
tersoff_server_submit = _sig("tersoff_server_submit", _I, _P, ctypes.POINTER(tersoff_job), ctypes.POINTER(_U64))
tersoff_server_poll = _sig("tersoff_server_poll", _I, _P, _U64, ctypes.POINTER(_I))
tersoff_server_wait = _sig("tersoff_server_wait", _I, _P, _U64, _D)
tersoff_server_result = _sig("tersoff_server_result", _I, _P, _U64, _P, _P, _P, _P)
tersoff_server_get_stats = _sig("tersoff_server_get_stats", _I, _P, ctypes.POINTER(tersoff_server_stats))
tersoff_server_last_error = _sig("tersoff_server_last_error", ctypes.c_char_p, _P)
tersoff_server_destroy = _sig("tersoff_server_destroy", None, _P)


class TersoffError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tersoff error {code}: {msg}")
        self.code = code


# ---- argument marshalling -----------------------------------------------------

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_flag(*arrays):
    dev = [_is_torch(a) and a.is_cuda for a in arrays if a is not None]
    if dev and all(dev):
        return DEVICE_PTRS
    if any(dev):
        raise ValueError("mix of device and host arrays")
    return HOST_PTRS


def _f64(a, shape):
    if _is_torch(a):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous() and tuple(a.shape) == shape, (a.dtype, a.shape, shape)
        return a
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape)


def _i32(a, n):
    if _is_torch(a):
        import torch
        assert a.dtype == torch.int32 and a.is_contiguous() and a.numel() == n
        return a
    return np.ascontiguousarray(a, dtype=np.int32).reshape(n)


def _box(box):
    return np.ascontiguousarray(box, dtype=np.float64).reshape(3)


# ---- handle classes -------------------------------------------------------------

class Context:
    def __init__(self, device=0, stream=None):
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(int(stream))
        rc = tersoff_ctx_create(int(device), s, ctypes.byref(h))
        if rc != OK:
            raise TersoffError(rc, "tersoff_ctx_create failed (no CUDA device?)")
        self.h = h

    def check(self, rc):
        if rc != OK:
            raise TersoffError(rc, tersoff_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            tersoff_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Params:
    def __init__(self, ctx, table, masses):
        table = np.ascontiguousarray(table, dtype=np.float64).reshape(-1, 14)
        nt = round(table.shape[0] ** (1 / 3))
        assert nt ** 3 == table.shape[0]
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        h = ctypes.c_void_p()
        ctx.check(tersoff_params_create(ctx.h, nt, ptr(table), ptr(masses), ctypes.byref(h)))
        self.h, self.ctx, self.ntypes = h, ctx, nt

    @property
    def cutoff(self):
        return tersoff_params_cutoff(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            tersoff_params_destroy(self.h)
            self.h = None


class NeighborList:
    def __init__(self, ctx, pos, box, cutoff, skin, types=None, params=None):
        """One radius cutoff + skin (tersoff_neighbor_build), or with `params` and
        `types` one radius per type pair (tersoff_neighbor_build_typed; cutoff unused)."""
        n = int(pos.shape[0])
        pos = _f64(pos, (n, 3))
        h = ctypes.c_void_p()
        if params is None:
            ctx.check(tersoff_neighbor_build(ctx.h, ptr(pos), n, ptr(_box(box)), float(cutoff), float(skin),
                                             _dev_flag(pos), ctypes.byref(h)))
        else:
            types = _i32(types, n)
            ctx.check(tersoff_neighbor_build_typed(ctx.h, ptr(pos), ptr(types), n, ptr(_box(box)), params.h,
                                                   float(skin), _dev_flag(pos, types), ctypes.byref(h)))
        self.h, self.ctx, self.n = h, ctx, n

    def rebuild(self, pos, box, cutoff, skin):
        pos = _f64(pos, (self.n, 3))
        self.ctx.check(tersoff_neighbor_build(self.ctx.h, ptr(pos), self.n, ptr(_box(box)), float(cutoff), float(skin),
                                              _dev_flag(pos), ctypes.byref(self.h)))

    def get(self):
        """(counts[N], idx[N, stride]) with -1 past each count."""
        n = ctypes.c_int64()
        stride = ctypes.c_int32()
        self.ctx.check(tersoff_nlist_get(self.ctx.h, self.h, ctypes.byref(n), ctypes.byref(stride), None, None))
        counts = np.zeros(n.value, dtype=np.int32)
        idx = np.zeros((n.value, stride.value), dtype=np.int32)
        self.ctx.check(tersoff_nlist_get(self.ctx.h, self.h, None, None, ptr(counts), ptr(idx)))
        return counts, idx

    def __del__(self):
        if getattr(self, "h", None):
            tersoff_nlist_destroy(self.h)
            self.h = None


def compute(ctx, params, pos, types, box, prec=FP64, nlist=None, forces=None, virial=True):
    """Energy (eV), forces [N,3] (eV/A) and virial (6) of one configuration.

    pos/types may be host numpy arrays or CUDA torch tensors (then ``forces``, if
    given, must be a CUDA float64 tensor [N,3]; it is written in place)."""
    n = int(pos.shape[0])
    pos = _f64(pos, (n, 3))
    types = _i32(types, n)
    flags = _dev_flag(pos, types, forces)
    if forces is None:
        if flags == DEVICE_PTRS:
            import torch
            forces = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        else:
            forces = np.zeros((n, 3))
    e = ctypes.c_double()
    w = np.zeros(6)
    ctx.check(tersoff_compute(ctx.h, ptr(pos), ptr(types), n, ptr(_box(box)), params.h,
                              nlist.h if nlist is not None else None, int(prec), flags, ctypes.byref(e),
                              ptr(forces), ptr(w) if virial else None))
    return e.value, forces, (w if virial else None)


class MD:
    """Device-resident velocity-Verlet state (tersoff_md_*)."""

    def __init__(self, ctx, params, pos, vel, types, box, dt, skin, prec=MIXED):
        n = int(pos.shape[0])
        pos = _f64(pos, (n, 3))
        vel = _f64(vel, (n, 3))
        types = _i32(types, n)
        h = ctypes.c_void_p()
        ctx.check(tersoff_md_create(ctx.h, ptr(pos), ptr(vel), ptr(types), n, ptr(_box(box)), params.h, float(dt),
                                    float(skin), int(prec), _dev_flag(pos, vel, types), ctypes.byref(h)))
        self.h, self.ctx, self.n, self.params = h, ctx, n, params

    def step(self, nsteps, trace=False):
        tr = np.zeros((nsteps + 1, 2)) if trace else None
        self.ctx.check(tersoff_md_step(self.h, int(nsteps), ptr(tr)))
        return tr

    def step_async(self, nsteps):
        self.ctx.check(tersoff_md_step_async(self.h, int(nsteps)))

    def sync(self):
        self.ctx.check(tersoff_md_sync(self.h))

    def get(self, forces=False):
        p = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        f = np.zeros((self.n, 3)) if forces else None
        self.ctx.check(tersoff_md_get(self.h, ptr(p), ptr(v), ptr(f), HOST_PTRS))
        return (p, v, f) if forces else (p, v)

    def stats(self):
        s, r, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        self.ctx.check(tersoff_md_stats(self.h, ctypes.byref(s), ctypes.byref(r), ctypes.byref(c)))
        return dict(steps=s.value, rebuilds=r.value, stride=c.value)

    def profile(self, enable=True):
        self.ctx.check(tersoff_md_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """(ms[5], launches[5]) for phases (integrator, list build, register force kernel,
        overflow force kernel + reductions, bookkeeping)."""
        ms = np.zeros(5)
        n = np.zeros(5, dtype=np.int64)
        self.ctx.check(tersoff_md_profile_read(self.h, ptr(ms), ptr(n)))
        return ms, n

    def __del__(self):
        if getattr(self, "h", None):
            tersoff_md_destroy(self.h)
            self.h = None


def md_run(ctx, params, pos, vel, types, box, dt, nsteps, skin, prec=MIXED, trace=True, inplace=False):
    """One call: returns (pos, vel, trace) after nsteps (host arrays).  inplace: pos and
    vel (C-contiguous float64 [N][3]) are updated in place, as tersoff_md_run does with
    the caller's buffers, and returned; else copies are."""
    n = int(pos.shape[0])
    if inplace:
        for a in (pos, vel):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == (n, 3)
                    and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"]):
                raise ValueError("inplace needs writeable C-contiguous float64 [N][3] pos and vel")
    else:
        pos = np.array(pos, dtype=np.float64).reshape(n, 3)
        vel = np.array(vel, dtype=np.float64).reshape(n, 3)
    types = _i32(types, n)
    tr = np.zeros((nsteps + 1, 2)) if trace else None
    ctx.check(tersoff_md_run(ctx.h, ptr(pos), ptr(vel), ptr(types), n, ptr(_box(box)), params.h, float(dt),
                             int(nsteps), float(skin), int(prec), HOST_PTRS, ptr(tr)))
    return pos, vel, tr


class Server:
    """Continuous-batching MD server (tersoff_server_*): jobs of independent
    systems run together on one device, admitted between chunks of steps."""

    def __init__(self, ctx, params, prec=MIXED, skin=0.5, budget_bytes=1 << 30, max_slots=64, chunk_steps=50):
        h = ctypes.c_void_p()
        ctx.check(tersoff_server_create(ctx.h, params.h, int(prec), float(skin), int(budget_bytes), int(max_slots),
                                        int(chunk_steps), ctypes.byref(h)))
        self.h, self.ctx, self.params = h, ctx, params
        self._n = {}

    def check(self, rc):
        if rc != OK:
            raise TersoffError(rc, tersoff_server_last_error(self.h).decode())
        return rc

    def submit(self, pos, vel, types, box, dt, nsteps):
        n = int(np.shape(pos)[0])
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(n, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3)
        types = np.ascontiguousarray(types, dtype=np.int32).reshape(n)
        job = tersoff_job(n, pos.ctypes.data, vel.ctypes.data, types.ctypes.data,
                          (ctypes.c_double * 3)(*[float(b) for b in _box(box)]), float(dt), int(nsteps))
        jid = _U64()
        self.check(tersoff_server_submit(self.h, ctypes.byref(job), ctypes.byref(jid)))
        self._n[jid.value] = n
        return jid.value

    def poll(self, jid):
        d = _I()
        self.check(tersoff_server_poll(self.h, jid, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, jid, timeout=60.0):
        """True when the job finished, False on timeout; raises if the job failed."""
        rc = tersoff_server_wait(self.h, jid, float(timeout))
        if rc == ERR_TIMEOUT:
            return False
        self.check(rc)
        return True

    def result(self, jid):
        """(pos, vel, (epot, ekin), (queued_s, run_s, total_s)); releases the job."""
        n = self._n[jid]
        p, v, e, t = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(2), np.zeros(3)
        self.check(tersoff_server_result(self.h, jid, ptr(p), ptr(v), ptr(e), ptr(t)))
        del self._n[jid]
        return p, v, (e[0], e[1]), tuple(t)

    def stats(self):
        st = tersoff_server_stats()
        self.check(tersoff_server_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            tersoff_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
