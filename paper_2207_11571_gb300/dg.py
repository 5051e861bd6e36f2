"""Thin Python binding of libdgnn.so (C ABI in include/dgnn.h).

Functions keep the C names and only marshal arguments: tensors become device
pointers, Python numbers become C scalars, a non-zero status raises
``DGError`` with the library's message.  Every computation runs in the CUDA
library; there is no fallback: if ``libdgnn.so`` is missing, loading raises.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdgnn.so")

DG_OK = 0
DG_ERR_INVALID_ARG = -1
DG_ERR_CUDA = -2
DG_ERR_NONFINITE = -3
DG_ERR_TIMEOUT = -4
DG_ERR_IO = -5
DG_ERR_UNSUPPORTED = -6
DG_ERR_EXCHANGE = -7

DG_PREC_FP64 = 0
DG_PREC_FP32 = 1


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libdgnn status {status}: {msg}")
        self.status = status


class dg_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int),
                ("gamma", ctypes.c_double), ("Cs", ctypes.c_double), ("Prt", ctypes.c_double),
                ("les_delta", ctypes.c_double), ("elems_per_block", ctypes.c_int), ("block_shape", ctypes.c_int),
                ("volume_flux", ctypes.c_int)]


class dg_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("energy", ctypes.c_double),
                ("ke", ctypes.c_double), ("dke_dt", ctypes.c_double), ("e_inf", ctypes.c_double * 3),
                ("max_wave", ctypes.c_double), ("nonfinite", ctypes.c_int64)]

    def as_dict(self):
        return {"mass": self.mass, "momentum": list(self.momentum), "energy": self.energy, "ke": self.ke,
                "dke_dt": self.dke_dt, "e_inf": list(self.e_inf), "max_wave": self.max_wave,
                "nonfinite": int(self.nonfinite)}


class dg_instance_desc(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("P", ctypes.c_int), ("Re", ctypes.c_double), ("Mach", ctypes.c_double),
                ("Pr", ctypes.c_double), ("closure", ctypes.c_int)]


DG_BATCH_MAX = 16
DG_BATCH_NO_GRAPH = 1
DG_BATCH_PERSISTENT = 2

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# int (*)(void* user, int what, const void* send_lo, const void* send_hi, void* recv_lo,
#         void* recv_hi, size_t bytes, void* stream)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, _P, _I, _P, _P, _P, _P, ctypes.c_size_t, _P)

# name -> argument types (all return int)
_SIGS = {
    "dg_opts_default": [ctypes.POINTER(dg_opts)],
    "dg_create": [_I, _I, _D, _D, _D, _I, ctypes.POINTER(dg_opts), ctypes.POINTER(_P)],
    "dg_destroy": [_P],
    "dg_basis_1d": [_I, _P, _P, _P],
    "dg_sizes": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "dg_init_tgv": [_P, _P, _P, _P],
    "dg_rhs": [_P, _P, _P, _P, _P],
    "dg_rk3_step": [_P, _P, _D, _I, _P, _P],
    "dg_advance_host": [_P, _P, _D, _I, _P, ctypes.POINTER(dg_diag), _P],
    "dg_advance_host_async": [_P, _P, _D, _I, _P, _I, _P],
    "dg_advance_host_wait": [_P, ctypes.POINTER(dg_diag), _P],
    "dg_project": [_P, _P, _P, _P, _P],
    "dg_prolong": [_P, _P, _P, _P, _P],
    "dg_diagnostics": [_P, _P, _P, _P, ctypes.POINTER(dg_diag), _P],
    "dg_stable_dt": [_P, _P, _D, ctypes.POINTER(_D), _P],
    "dg_make_pairs": [_P, _P, _P, _P, _D, _I, _I, _P, _P, _P],
    "dg_check_conversions": [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P],
    "dg_autotune": [_P, _P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P],
    "dg_blocking": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "dg_set_forcing_mode": [_P, _I],
    "dg_check_bounded_waits": [ctypes.POINTER(_D), _P],
    "dg_rhs_noalloc": [_I, _I, _D, _D, _D, _I, _I, _P, _P, _P],
    "dg_create_batch": [ctypes.POINTER(dg_instance_desc), _I, ctypes.POINTER(dg_opts), ctypes.POINTER(_P)],
    "dg_batch_destroy": [_P],
    "dg_batch_size": [_P, ctypes.POINTER(_I)],
    "dg_batch_member": [_P, _I, ctypes.POINTER(_P)],
    "dg_batch_rk3_step": [_P, ctypes.POINTER(_P), ctypes.POINTER(_D), _I, _I, _P],
    "dg_batch_autotune": [_P, ctypes.POINTER(_P), ctypes.POINTER(_D), _P],
    "dg_create_part": [_I, _I, _D, _D, _D, _I, ctypes.POINTER(dg_opts), _I, _I, ctypes.POINTER(_P)],
    "dg_part_layout": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_int64)],
    "dg_part_set_exchange": [_P, EXCHANGE_FN, _P],
    "dg_part_trace_bytes": [_P, _I, ctypes.POINTER(ctypes.c_size_t)],
    "dg_group_rk3_step": [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), _D, _I, _P],
    "dg_group_rhs": [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "dg_group_diagnostics": [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(dg_diag), _P],
    "dg_diag_combine": [ctypes.POINTER(dg_diag), _I, ctypes.POINTER(dg_diag)],
    "dg_profile_rk3": [_P, _P, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I),
                       ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D), _P],
}

_lib = None


def lib():
    """Loads libdgnn.so once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2207_11571_gb300.build` "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.dg_last_error.argtypes = []
        L.dg_last_error.restype = ctypes.c_char_p
        _register_nn(L)
        _lib = L
    return _lib


def _register_nn(L):
    from . import nn as _nn
    _nn._register(L)


def check(status):
    if status != DG_OK:
        raise DGError(status, lib().dg_last_error().decode(errors="replace"))
    return status


def ptr(t):
    """Device (or host numpy) pointer of a contiguous array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(t)}")


def stream_ptr(stream=None):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_state(ctx, t, name, dtype="float64"):
    n = dg_sizes(ctx)[0]
    if t.numel() != 5 * n:
        raise ValueError(f"{name} must hold 5 * {n} values, got {t.numel()}")
    if str(t.dtype).split(".")[-1] != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if hasattr(t, "is_cuda") and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def _check_host_state(ctx, a, name):
    n = dg_sizes(ctx)[0]
    size = a.numel() if hasattr(a, "numel") else a.size
    if size != 5 * n:
        raise ValueError(f"{name} must hold 5 * {n} values, got {size}")
    if str(a.dtype).split(".")[-1] != "float64":
        raise TypeError(f"{name} must be float64")
    if hasattr(a, "is_cuda") and a.is_cuda:
        raise ValueError(f"{name} must be a host array")


# ----------------------------------------------------------------------------- entry points

def dg_opts_default():
    o = dg_opts()
    check(lib().dg_opts_default(ctypes.byref(o)))
    return o


def dg_create(K, P, Re, Mach, Pr=0.71, closure=0, opts=None, **kw):
    """Returns an opaque context handle (int).  ``kw`` overrides fields of dg_opts."""
    o = opts if opts is not None else dg_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    check(lib().dg_create(int(K), int(P), float(Re), float(Mach), float(Pr), int(closure), ctypes.byref(o),
                          ctypes.byref(h)))
    return h.value


def dg_destroy(ctx):
    check(lib().dg_destroy(ctypes.c_void_p(ctx)))


def dg_basis_1d(P):
    import numpy as np
    n = P + 1
    xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    check(lib().dg_basis_1d(int(P), ptr(xi), ptr(w), ptr(D)))
    return xi, w, D


def dg_sizes(ctx):
    n, e = ctypes.c_int64(), ctypes.c_int64()
    check(lib().dg_sizes(ctypes.c_void_p(ctx), ctypes.byref(n), ctypes.byref(e)))
    return n.value, e.value


def _net(net):
    return None if net is None else ctypes.c_void_p(net if isinstance(net, int) else net.handle)


def dg_init_tgv(ctx, q, perturbation=None, stream=None):
    _check_state(ctx, q, "q")
    if perturbation is not None:
        _check_state(ctx, perturbation, "perturbation")
    check(lib().dg_init_tgv(ctypes.c_void_p(ctx), ptr(q), ptr(perturbation), stream_ptr(stream)))


def dg_rhs(ctx, q, dqdt, forcing=None, stream=None):
    _check_state(ctx, q, "q")
    _check_state(ctx, dqdt, "dqdt")
    check(lib().dg_rhs(ctypes.c_void_p(ctx), ptr(q), ptr(dqdt), _net(forcing), stream_ptr(stream)))


def dg_rk3_step(ctx, q, dt, nsteps=1, forcing=None, stream=None):
    _check_state(ctx, q, "q")
    check(lib().dg_rk3_step(ctypes.c_void_p(ctx), ptr(q), float(dt), int(nsteps), _net(forcing),
                            stream_ptr(stream)))


def dg_advance_host(ctx, q_host, dt, nsteps=1, forcing=None, stream=None, want_diag=True):
    """q_host: numpy float64 or CPU torch tensor (pinned or pageable), updated in place."""
    d = dg_diag()
    check(lib().dg_advance_host(ctypes.c_void_p(ctx), ptr(q_host), float(dt), int(nsteps), _net(forcing),
                                ctypes.byref(d) if want_diag else None, stream_ptr(stream)))
    return d.as_dict() if want_diag else None


def dg_advance_host_async(ctx, q_host, dt, nsteps=1, forcing=None, stream=None, want_diag=True):
    """Enqueues dg_advance_host on stream without waiting; q_host (pinned CPU tensor or
    numpy float64) must stay untouched until the matching dg_advance_host_wait returns.
    Up to two calls may be pending per context (on one stream)."""
    _check_host_state(ctx, q_host, "q_host")
    check(lib().dg_advance_host_async(ctypes.c_void_p(ctx), ptr(q_host), float(dt), int(nsteps), _net(forcing),
                                      int(bool(want_diag)), stream_ptr(stream)))


def dg_advance_host_wait(ctx, stream=None, want_diag=True):
    """Waits for the oldest pending dg_advance_host_async call (for that call only: a
    second pending call keeps running); returns its diagnostics."""
    d = dg_diag()
    check(lib().dg_advance_host_wait(ctypes.c_void_p(ctx), ctypes.byref(d) if want_diag else None,
                                     stream_ptr(stream)))
    return d.as_dict() if want_diag else None


def dg_project(hi, lo, q_hi, q_lo, stream=None):
    _check_state(hi, q_hi, "q_hi")
    _check_state(lo, q_lo, "q_lo")
    check(lib().dg_project(ctypes.c_void_p(hi), ctypes.c_void_p(lo), ptr(q_hi), ptr(q_lo), stream_ptr(stream)))


def dg_prolong(lo, hi, q_lo, q_hi, stream=None):
    """q_hi = the order-P_lo solution of lo evaluated at hi's nodes (same K)."""
    _check_state(lo, q_lo, "q_lo")
    _check_state(hi, q_hi, "q_hi")
    check(lib().dg_prolong(ctypes.c_void_p(lo), ctypes.c_void_p(hi), ptr(q_lo), ptr(q_hi), stream_ptr(stream)))


def dg_diagnostics(ctx, q, q_ref=None, forcing=None, stream=None, raise_nonfinite=True):
    _check_state(ctx, q, "q")
    d = dg_diag()
    st = lib().dg_diagnostics(ctypes.c_void_p(ctx), ptr(q), ptr(q_ref), _net(forcing), ctypes.byref(d),
                              stream_ptr(stream))
    if st != DG_ERR_NONFINITE or raise_nonfinite:
        check(st)
    return d.as_dict()


def dg_stable_dt(ctx, q, cfl, stream=None):
    _check_state(ctx, q, "q")
    dt = ctypes.c_double()
    check(lib().dg_stable_dt(ctypes.c_void_p(ctx), ptr(q), float(cfl), ctypes.byref(dt), stream_ptr(stream)))
    return dt.value


def dg_make_pairs(lo, q_bar_n, q_nn_np1, q_bar_np1, dt, first_var, n_vars, X, Y, stream=None):
    for t, nm in ((q_bar_n, "q_bar_n"), (q_nn_np1, "q_nn_np1"), (q_bar_np1, "q_bar_np1")):
        _check_state(lo, t, nm)
    nodes, _ = dg_sizes(lo)
    for t, nm in ((X, "X"), (Y, "Y")):
        if t.numel() != nodes * n_vars or str(t.dtype) != "torch.float32":
            raise ValueError(f"{nm} must be float32 with {nodes * n_vars} values")
    check(lib().dg_make_pairs(ctypes.c_void_p(lo), ptr(q_bar_n), ptr(q_nn_np1), ptr(q_bar_np1), float(dt),
                              int(first_var), int(n_vars), ptr(X), ptr(Y), stream_ptr(stream)))


def dg_profile_rk3(ctx, q, dt, nsteps=1, stream=None):
    """Per-kernel device times of nsteps RK3 steps (CUDA events inside the library)."""
    _check_state(ctx, q, "q")
    tg, tf, fb, gb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lg, lf = ctypes.c_int(), ctypes.c_int()
    check(lib().dg_profile_rk3(ctypes.c_void_p(ctx), ptr(q), float(dt), int(nsteps), ctypes.byref(tg),
                               ctypes.byref(tf), ctypes.byref(lg), ctypes.byref(lf), ctypes.byref(fb),
                               ctypes.byref(gb), stream_ptr(stream)))
    return {"ms_gradient": tg.value, "ms_flux": tf.value, "launches_gradient": lg.value,
            "launches_flux": lf.value, "flux_bytes_per_launch": fb.value, "gradient_bytes_per_launch": gb.value}


def dg_autotune(ctx, q, dt, stream=None):
    """Picks the fastest elements-per-block for the context; returns (E, ms per RK3 step)."""
    _check_state(ctx, q, "q")
    E, ms = ctypes.c_int(), ctypes.c_double()
    check(lib().dg_autotune(ctypes.c_void_p(ctx), ptr(q), float(dt), ctypes.byref(E), ctypes.byref(ms),
                            stream_ptr(stream)))
    return E.value, ms.value


def dg_check_bounded_waits(stream=None):
    """Runs the bounded-wait self-check; returns the seconds the two expiring waits took."""
    sec = ctypes.c_double()
    check(lib().dg_check_bounded_waits(ctypes.byref(sec), stream_ptr(stream)))
    return sec.value


DG_FORCING_STAGE, DG_FORCING_POST = 0, 1


def dg_set_forcing_mode(ctx, mode):
    """Where dg_rk3_step applies a network forcing: DG_FORCING_STAGE (s in every RK
    stage, Eq. 4) or DG_FORCING_POST (Algorithm 1: uncorrected step, then q += dt s(q^n))."""
    check(lib().dg_set_forcing_mode(ctypes.c_void_p(ctx), int(mode)))


def dg_blocking(ctx):
    """(elements per block, block shape) the context's kernels use; shape 0 = rows of
    consecutive elements, 1 = 2 x 2 x 2 cubes."""
    E, shape = ctypes.c_int(), ctypes.c_int()
    check(lib().dg_blocking(ctypes.c_void_p(ctx), ctypes.byref(E), ctypes.byref(shape)))
    return E.value, shape.value


def dg_rhs_noalloc(K, P, Re, Mach, Pr, closure, precision, q, dqdt, stream=None):
    """dqdt = p(q) without device allocation (for callers that may not allocate, such as
    an in-situ hook with a fixed memory budget); at most 32768 nodes; calls share one
    scratch array, so overlapping calls must be serialised."""
    nodes = K ** 3 * (P + 1) ** 3
    for t, nm in ((q, "q"), (dqdt, "dqdt")):
        if t.numel() != 5 * nodes or str(t.dtype) != "torch.float64" or not t.is_cuda:
            raise ValueError(f"{nm} must be a CUDA float64 tensor of 5 * {nodes} values")
    check(lib().dg_rhs_noalloc(int(K), int(P), float(Re), float(Mach), float(Pr), int(closure), int(precision),
                               ptr(q), ptr(dqdt), stream_ptr(stream)))


def dg_create_batch(members, opts=None, **kw):
    """members: sequence of (K, P, Re, Mach, Pr, closure).  Returns an opaque batch handle."""
    n = len(members)
    arr = (dg_instance_desc * max(n, 1))(*[dg_instance_desc(int(K), int(P), float(Re), float(M), float(Pr), int(c))
                                           for K, P, Re, M, Pr, c in members])
    o = opts if opts is not None else dg_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    check(lib().dg_create_batch(arr, n, ctypes.byref(o), ctypes.byref(h)))
    return h.value


def dg_batch_destroy(batch):
    check(lib().dg_batch_destroy(ctypes.c_void_p(batch)))


def dg_batch_size(batch):
    n = ctypes.c_int()
    check(lib().dg_batch_size(ctypes.c_void_p(batch), ctypes.byref(n)))
    return n.value


def dg_batch_member(batch, i):
    """Borrowed context of member i (owned by the batch)."""
    h = ctypes.c_void_p()
    check(lib().dg_batch_member(ctypes.c_void_p(batch), int(i), ctypes.byref(h)))
    return h.value


def _batch_arrays(batch, qs, dts):
    n = dg_batch_size(batch)
    if len(qs) != n or len(dts) != n:
        raise ValueError(f"need {n} states and {n} step sizes")
    for i, q in enumerate(qs):
        _check_state(dg_batch_member(batch, i), q, f"q[{i}]")
    return (ctypes.c_void_p * n)(*[q.data_ptr() for q in qs]), (ctypes.c_double * n)(*[float(d) for d in dts])


def dg_batch_rk3_step(batch, qs, dts, nsteps=1, flags=0, stream=None):
    qa, da = _batch_arrays(batch, qs, dts)
    check(lib().dg_batch_rk3_step(ctypes.c_void_p(batch), qa, da, int(nsteps), int(flags), stream_ptr(stream)))


def dg_batch_autotune(batch, qs, dts, stream=None):
    qa, da = _batch_arrays(batch, qs, dts)
    check(lib().dg_batch_autotune(ctypes.c_void_p(batch), qa, da, stream_ptr(stream)))


def dg_check_conversions(x, stream=None):
    """(mismatches of the FP64->FP32 conversion, of the FP32->FP64 widening) on device array x."""
    mm = (ctypes.c_int64 * 2)()
    check(lib().dg_check_conversions(ptr(x), int(x.numel()), mm, stream_ptr(stream)))
    return int(mm[0]), int(mm[1])


# ----------------------------------------------------------------------------- slabs

def dg_create_part(K, P, Re, Mach, Pr=0.71, closure=0, z_begin=0, z_count=None, opts=None, **kw):
    """Context of the slab of element layers [z_begin, z_begin + z_count) with one ghost
    layer on each side (local arrays of z_count + 2 layers)."""
    o = opts if opts is not None else dg_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    check(lib().dg_create_part(int(K), int(P), float(Re), float(Mach), float(Pr), int(closure), ctypes.byref(o),
                               int(z_begin), int(K if z_count is None else z_count), ctypes.byref(h)))
    return h.value


def dg_part_layout(ctx):
    """(z_begin, z_count, first owned node, owned nodes) of a slab's local arrays."""
    zb, zc, f, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().dg_part_layout(ctypes.c_void_p(ctx), ctypes.byref(zb), ctypes.byref(zc), ctypes.byref(f),
                               ctypes.byref(n)))
    return zb.value, zc.value, f.value, n.value


def dg_part_set_exchange(ctx, fn):
    """fn: an EXCHANGE_FN instance (the caller keeps it alive) or None."""
    check(lib().dg_part_set_exchange(ctypes.c_void_p(ctx), fn if fn is not None else EXCHANGE_FN(), None))


def dg_part_trace_bytes(ctx, what):
    b = ctypes.c_size_t()
    check(lib().dg_part_trace_bytes(ctypes.c_void_p(ctx), int(what), ctypes.byref(b)))
    return b.value


def _group_arrays(parts, qs, name="q"):
    n = len(parts)
    if len(qs) != n:
        raise ValueError(f"need {n} states")
    for i, (c, q) in enumerate(zip(parts, qs)):
        _check_state(c, q, f"{name}[{i}]")
    return n, (ctypes.c_void_p * n)(*parts), (ctypes.c_void_p * n)(*[q.data_ptr() for q in qs])


def dg_group_rk3_step(parts, qs, dt, nsteps=1, stream=None):
    n, pa, qa = _group_arrays(parts, qs)
    check(lib().dg_group_rk3_step(pa, n, qa, float(dt), int(nsteps), stream_ptr(stream)))


def dg_group_rhs(parts, qs, dqdts, stream=None):
    n, pa, qa = _group_arrays(parts, qs)
    _, _, da = _group_arrays(parts, dqdts, "dqdt")
    check(lib().dg_group_rhs(pa, n, qa, da, stream_ptr(stream)))


def dg_group_diagnostics(parts, qs, stream=None, raise_nonfinite=True):
    n, pa, qa = _group_arrays(parts, qs)
    d = dg_diag()
    st = lib().dg_group_diagnostics(pa, n, qa, ctypes.byref(d), stream_ptr(stream))
    if st != DG_ERR_NONFINITE or raise_nonfinite:
        check(st)
    return d.as_dict()


def dg_diag_combine(diags, raise_nonfinite=True):
    """Combines the slabs' diagnostics (dicts as returned by dg_diagnostics), in order."""
    n = len(diags)
    arr = (dg_diag * n)()
    for a, d in zip(arr, diags):
        a.mass, a.energy, a.ke, a.dke_dt, a.max_wave = d["mass"], d["energy"], d["ke"], d["dke_dt"], d["max_wave"]
        a.nonfinite = int(d["nonfinite"])
        for k in range(3):
            a.momentum[k] = d["momentum"][k]
            a.e_inf[k] = d["e_inf"][k]
    out = dg_diag()
    st = lib().dg_diag_combine(arr, n, ctypes.byref(out))
    if st != DG_ERR_NONFINITE or raise_nonfinite:
        check(st)
    return out.as_dict()
