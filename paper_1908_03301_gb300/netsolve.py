"""Python binding of the C ABI in ``include/netsolve.h`` (ctypes).

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libnetsolve.so``.  There is no CPU fallback: if the library is not
built, :func:`lib` raises.  Bond planes may be numpy arrays (host) or torch
CUDA tensors (device; the current torch stream is used for the work).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NET_OK, NET_EINVAL, NET_ENOMEM, NET_EBUDGET, NET_ENOTCONVERGED, NET_ETIMEOUT, NET_ECUDA, \
    NET_ECANCELLED, NET_EBUSY = range(9)
NET_F64, NET_F32 = 0, 1
NET_MIXED, NET_FP64 = 0, 1
NET_REFINE_RELIABLE, NET_REFINE_RESTART = 0, 1
STATUS_NAMES = ["NET_OK", "NET_EINVAL", "NET_ENOMEM", "NET_EBUDGET", "NET_ENOTCONVERGED",
                "NET_ETIMEOUT", "NET_ECUDA", "NET_ECANCELLED", "NET_EBUSY"]


class net_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int64 * 3), ("flow_axis", C.c_int),
                ("periodic_mask", C.c_uint), ("p_in", C.c_double), ("p_out", C.c_double),
                ("bond_dtype", C.c_int), ("on_device", C.c_int), ("stream", C.c_void_p)]


class net_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol_rel", C.c_double), ("tol_inner", C.c_double),
                ("max_outer", C.c_int), ("max_inner", C.c_int64), ("check_every", C.c_int),
                ("x0", C.c_void_p), ("x0_on_device", C.c_int), ("stream", C.c_void_p),
                ("tol_geff", C.c_double), ("refine", C.c_int), ("update_delta", C.c_double)]


class net_result(C.Structure):
    _fields_ = [("g_eff", C.c_double), ("k_eff", C.c_double), ("q_in", C.c_double),
                ("q_out", C.c_double), ("rel_residual", C.c_double),
                ("max_imbalance", C.c_double), ("energy_g", C.c_double),
                ("n_active", C.c_int64), ("outer_iters", C.c_int), ("inner_iters", C.c_int64),
                ("fp64_fallback", C.c_int), ("ms", C.c_float), ("inner_ms", C.c_float),
                ("inner_launches", C.c_int64), ("status", C.c_int), ("g_eff_err", C.c_double),
                ("n_solved", C.c_int64), ("queue_ms", C.c_double), ("co_running", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class net_tune(C.Structure):
    _fields_ = [("col_block", C.c_int), ("row_band", C.c_int), ("seg_per_sm", C.c_int),
                ("size_class", C.c_int), ("candidates", C.c_int), ("us_per_sweep", C.c_double),
                ("us_default", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class net_fbm_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int64 * 3), ("hurst", C.c_double),
                ("beta", C.c_double * 3), ("fft_f32", C.c_int), ("stream", C.c_void_p)]


EXPORTS = ["net_opts_default", "net_create", "net_solve", "net_flux", "net_get_pressure",
           "net_get_labels", "net_destroy", "net_solve_batch", "netq_create", "netq_submit",
           "netq_poll", "netq_wait", "netq_cancel", "netq_stats", "netq_destroy",
           "net_last_error", "net_labels_noalloc", "net_autotune", "net_tune_clear",
           "net_get_backbone", "net_close_smallest", "net_fbm_field", "net_fbm_bonds"]

_lib = None


def lib(build_if_missing: bool = False):
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    P = C.POINTER
    vp = C.c_void_p
    L.net_opts_default.argtypes = [P(net_opts)]
    L.net_opts_default.restype = None
    L.net_create.argtypes = [P(net_desc), P(vp), P(vp)]
    L.net_create.restype = C.c_int
    L.net_solve.argtypes = [vp, P(net_opts), P(net_result)]
    L.net_solve.restype = C.c_int
    L.net_flux.argtypes = [vp, P(C.c_double), P(C.c_double), P(C.c_double)]
    L.net_flux.restype = C.c_int
    L.net_get_pressure.argtypes = [vp, vp, C.c_int64, C.c_int]
    L.net_get_pressure.restype = C.c_int
    L.net_get_labels.argtypes = [vp, vp, vp, C.c_int64]
    L.net_get_labels.restype = C.c_int
    L.net_get_backbone.argtypes = [vp, vp, C.c_int64]
    L.net_get_backbone.restype = C.c_int
    L.net_destroy.argtypes = [vp]
    L.net_destroy.restype = C.c_int
    L.net_last_error.argtypes = []
    L.net_last_error.restype = C.c_char_p
    L.net_labels_noalloc.argtypes = [P(net_desc), P(vp), vp, vp]
    L.net_labels_noalloc.restype = C.c_int
    L.net_close_smallest.argtypes = [P(net_desc), P(vp), C.c_double]
    L.net_close_smallest.restype = C.c_int
    L.net_fbm_field.argtypes = [P(net_fbm_desc), vp, vp]
    L.net_fbm_field.restype = C.c_int
    L.net_fbm_bonds.argtypes = [P(net_desc), vp, C.c_double, P(vp)]
    L.net_fbm_bonds.restype = C.c_int
    L.net_autotune.argtypes = [P(vp), C.c_int, P(net_opts), P(net_tune)]
    L.net_autotune.restype = C.c_int
    L.net_tune_clear.argtypes = []
    L.net_tune_clear.restype = None
    L.net_solve_batch.argtypes = [P(vp), C.c_int, P(net_opts), P(net_result)]
    L.net_solve_batch.restype = C.c_int
    L.netq_create.argtypes = [C.c_size_t, C.c_int, P(net_opts), P(vp)]
    L.netq_create.restype = C.c_int
    L.netq_submit.argtypes = [vp, P(net_desc), P(vp), P(C.c_uint64)]
    L.netq_submit.restype = C.c_int
    L.netq_poll.argtypes = [vp, C.c_uint64, P(net_result)]
    L.netq_poll.restype = C.c_int
    L.netq_wait.argtypes = [vp, C.c_uint64, C.c_int, P(net_result)]
    L.netq_wait.restype = C.c_int
    L.netq_cancel.argtypes = [vp, C.c_uint64]
    L.netq_cancel.restype = C.c_int
    L.netq_stats.argtypes = [vp, P(C.c_double), P(C.c_double), P(C.c_uint64)]
    L.netq_stats.restype = C.c_int
    L.netq_destroy.argtypes = [vp]
    L.netq_destroy.restype = C.c_int
    _lib = L
    return L


class NetError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = lib().net_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


def _check(st, where):
    if st != NET_OK:
        raise NetError(st, where)


def opts_default() -> net_opts:
    o = net_opts()
    lib().net_opts_default(C.byref(o))
    return o


def make_opts(precision=NET_MIXED, tol_rel=None, tol_inner=None, max_outer=None,
              max_inner=None, check_every=None, stream=None, tol_geff=None, refine=None,
              update_delta=None) -> net_opts:
    o = opts_default()
    if refine is not None:
        o.refine = refine
    if update_delta is not None:
        o.update_delta = update_delta
    if tol_geff is not None:
        o.tol_geff = tol_geff
    o.precision = precision
    if tol_rel is not None:
        o.tol_rel = tol_rel
    if tol_inner is not None:
        o.tol_inner = tol_inner
    if max_outer is not None:
        o.max_outer = max_outer
    if max_inner is not None:
        o.max_inner = max_inner
    if check_every is not None:
        o.check_every = check_every
    if stream is not None:
        o.stream = stream
    return o


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def periodic_mask(periodic):
    """Axes (iterable of 0/1/2) -> net_desc.periodic_mask."""
    m = 0
    for a in periodic:
        m |= 1 << int(a)
    return m


def plane_elems(dims, d, periodic=()):
    """Number of bonds in plane d (the last layer wraps along a periodic axis)."""
    n = [int(v) for v in dims]
    if d not in periodic:
        n[d] -= 1
    return int(np.prod(n))


def make_desc(dims, flow_axis=0, p_in=1.0, p_out=0.0, bond_dtype=NET_F64, on_device=0,
              stream=None, periodic=()) -> net_desc:
    n = list(int(v) for v in dims) + [1] * (3 - len(dims))
    return net_desc(len(dims), (C.c_int64 * 3)(*n), int(flow_axis), periodic_mask(periodic),
                    float(p_in), float(p_out), int(bond_dtype), int(on_device), stream)


def marshal_planes(planes, ndim):
    """-> (keepalive list, void* [3], bond_dtype, on_device, stream)."""
    keep = []
    ptrs = (C.c_void_p * 3)()
    dev = _is_torch(planes[0]) and planes[0].is_cuda
    f32 = None
    stream = None
    for d in range(ndim):
        a = planes[d]
        if dev:
            import torch
            a = a.contiguous()
            if a.dtype not in (torch.float32, torch.float64):
                raise TypeError("bond planes must be float32 or float64")
            this32 = a.dtype == torch.float32
            ptrs[d] = a.data_ptr() if a.numel() else None
            stream = torch.cuda.current_stream(a.device).cuda_stream
        else:
            a = np.ascontiguousarray(a)
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
            this32 = a.dtype == np.float32
            ptrs[d] = a.ctypes.data if a.size else None
        if f32 is None:
            f32 = this32
        elif f32 != this32:
            raise TypeError("all bond planes must share one dtype")
        keep.append(a)
    return keep, ptrs, (NET_F32 if f32 else NET_F64), int(dev), stream


@dataclass
class Result:
    g_eff: float
    k_eff: float
    q_in: float
    q_out: float
    rel_residual: float
    max_imbalance: float
    energy_g: float
    n_active: int
    outer_iters: int
    inner_iters: int
    fp64_fallback: int
    ms: float
    inner_ms: float
    inner_launches: int
    status: int
    g_eff_err: float
    n_solved: int
    queue_ms: float = 0.0  # queue: submit -> admission onto the device
    co_running: int = 0    # queue: requests running when this one was admitted
    error: str = ""  # message of a non-OK status

    @classmethod
    def from_c(cls, r: net_result):
        return cls(**r.as_dict())


class Network:
    """One resident network (net_create ... net_destroy)."""

    def __init__(self, dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, periodic=()):
        L = lib()
        self.dims = tuple(int(v) for v in dims)
        self.N = int(np.prod(self.dims))
        for d in range(len(self.dims)):
            size = planes[d].numel() if _is_torch(planes[d]) else np.size(planes[d])
            if size != plane_elems(self.dims, d, periodic):
                raise ValueError(f"bond plane {d} has {size} entries, expected "
                                 f"{plane_elems(self.dims, d, periodic)}")
        keep, ptrs, bdt, dev, stream = marshal_planes(planes, len(dims))
        desc = make_desc(dims, flow_axis, p_in, p_out, bdt, dev, stream, periodic)
        h = C.c_void_p()
        _check(L.net_create(C.byref(desc), ptrs, C.byref(h)), "net_create")
        self.h = h
        self.shape = tuple(reversed(self.dims))

    def solve(self, opts: net_opts | None = None, x0=None, check=True) -> Result:
        L = lib()
        o = opts if opts is not None else opts_default()
        keep = None
        if x0 is not None:
            if _is_torch(x0):
                keep = x0.contiguous().to(dtype=__import__("torch").float64)
                o.x0 = keep.data_ptr()
                o.x0_on_device = int(keep.is_cuda)
            else:
                keep = np.ascontiguousarray(x0, dtype=np.float64)
                o.x0 = keep.ctypes.data
                o.x0_on_device = 0
        r = net_result()
        st = L.net_solve(self.h, C.byref(o), C.byref(r))
        if check and st not in (NET_OK, NET_ENOTCONVERGED):
            raise NetError(st, "net_solve")
        return Result.from_c(r)

    def flux(self):
        qi, qo, g = C.c_double(), C.c_double(), C.c_double()
        _check(lib().net_flux(self.h, C.byref(qi), C.byref(qo), C.byref(g)), "net_flux")
        return qi.value, qo.value, g.value

    def pressure(self, out=None):
        """FP64 node pressures: numpy (host) or into a torch CUDA tensor."""
        if out is not None and _is_torch(out):
            _check(lib().net_get_pressure(self.h, out.data_ptr(), out.numel(), int(out.is_cuda)),
                   "net_get_pressure")
            return out
        P = np.empty(self.N, np.float64)
        _check(lib().net_get_pressure(self.h, P.ctypes.data, self.N, 0), "net_get_pressure")
        return P.reshape(self.shape)

    def labels(self):
        lab = np.empty(self.N, np.int32)
        cls = np.empty(self.N, np.uint8)
        _check(lib().net_get_labels(self.h, lab.ctypes.data, cls.ctypes.data, self.N),
               "net_get_labels")
        return lab.reshape(self.shape), cls.reshape(self.shape)

    def backbone(self):
        """bool mask of the backbone (spanning nodes left in the system)."""
        b = np.empty(self.N, np.uint8)
        _check(lib().net_get_backbone(self.h, b.ctypes.data, self.N), "net_get_backbone")
        return b.reshape(self.shape).astype(bool)

    def close(self):
        if getattr(self, "h", None):
            lib().net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def close_smallest(dims, planes, q, periodic=(), flow_axis=0):
    """net_close_smallest: close the floor(q M) weakest bonds of torch CUDA
    planes in place (Sec. VI.B sorted removal); returns the planes."""
    if not (_is_torch(planes[0]) and planes[0].is_cuda):
        raise TypeError("close_smallest takes torch CUDA bond planes")
    for d in range(len(dims)):
        if not planes[d].is_contiguous():
            raise ValueError("bond planes must be contiguous (they are modified in place)")
        if planes[d].numel() != plane_elems(dims, d, periodic):
            raise ValueError(f"bond plane {d} has {planes[d].numel()} entries")
    keep, ptrs, bdt, dev, stream = marshal_planes(planes, len(dims))
    desc = make_desc(dims, flow_axis, 1.0, 0.0, bdt, 1, stream, periodic)
    _check(lib().net_close_smallest(C.byref(desc), ptrs, float(q)), "net_close_smallest")
    return planes


def fbm_field(dims, noise, hurst, beta=None, out=None):
    """net_fbm_field: FBM field (Eq. 1 / Eq. 2) from complex noise, a torch
    complex128 (FP64 transform) or complex64 (FP32 transform) CUDA tensor of
    node shape (it is overwritten).  Returns a float64 CUDA tensor of node
    shape (``out`` if given)."""
    import torch

    if not (_is_torch(noise) and noise.is_cuda and noise.dtype in (torch.complex128, torch.complex64)
            and noise.is_contiguous()):
        raise TypeError("noise must be a contiguous complex128 or complex64 CUDA tensor")
    f32 = int(noise.dtype == torch.complex64)
    N = int(np.prod(dims))
    if noise.numel() != N:
        raise ValueError(f"noise has {noise.numel()} values, expected {N}")
    if out is None:
        out = torch.empty(tuple(reversed([int(v) for v in dims])), dtype=torch.float64, device=noise.device)
    if not (out.dtype == torch.float64 and out.is_cuda and out.is_contiguous() and out.numel() == N):
        raise ValueError("out must be a contiguous float64 CUDA tensor with one value per node")
    n = list(int(v) for v in dims) + [1] * (3 - len(dims))
    b = list(beta) if beta is not None else [1.0] * len(dims)
    b = [float(v) for v in b] + [1.0] * (3 - len(b))
    stream = torch.cuda.current_stream(noise.device).cuda_stream
    d = net_fbm_desc(len(dims), (C.c_int64 * 3)(*n), float(hurst), (C.c_double * 3)(*b), f32, stream)
    _check(lib().net_fbm_field(C.byref(d), noise.data_ptr(), out.data_ptr()), "net_fbm_field")
    return out


def fbm_bonds(dims, field, sigma, dtype=None, periodic=(), flow_axis=0):
    """net_fbm_bonds: conductance planes exp(sigma (B_i + B_j)/2) from a
    float64 CUDA field; returns torch CUDA planes of ``dtype`` (float64)."""
    import torch

    dtype = dtype or torch.float64
    if not (_is_torch(field) and field.is_cuda and field.dtype == torch.float64 and field.is_contiguous()):
        raise TypeError("field must be a contiguous float64 CUDA tensor")
    planes = []
    for d in range(len(dims)):
        n = [int(v) for v in dims]
        if d not in periodic:
            n[d] -= 1
        planes.append(torch.empty(tuple(reversed(n)), dtype=dtype, device=field.device))
    keep, ptrs, bdt, dev, stream = marshal_planes(planes, len(dims))
    desc = make_desc(dims, flow_axis, 1.0, 0.0, bdt, 1, stream, periodic)
    _check(lib().net_fbm_bonds(C.byref(desc), field.data_ptr(), float(sigma), ptrs), "net_fbm_bonds")
    return planes


def last_error() -> str:
    """Message of the last failing call on this thread (net_last_error)."""
    return lib().net_last_error().decode(errors="replace")


def solve_batch(networks, opts: net_opts | None = None, check=True):
    """net_solve_batch over a list of Network objects; returns [Result]."""
    L = lib()
    n = len(networks)
    hs = (C.c_void_p * n)(*[net.h for net in networks])
    res = (net_result * n)()
    st = L.net_solve_batch(hs, n, C.byref(opts) if opts is not None else None, res)
    if check and st not in (NET_OK, NET_ENOTCONVERGED):
        raise NetError(st, "net_solve_batch")
    return [Result.from_c(res[i]) for i in range(n)]


def autotune(networks, opts: net_opts | None = None) -> dict:
    """net_autotune over a list of Network objects (all 2D or all 3D); returns
    the chosen tile shape and its time per sweep as a dict."""
    n = len(networks)
    hs = (C.c_void_p * n)(*[net.h for net in networks])
    out = net_tune()
    _check(lib().net_autotune(hs, n, C.byref(opts) if opts is not None else None, C.byref(out)),
           "net_autotune")
    return out.as_dict()


def tune_clear():
    """net_tune_clear: forget every tuned tile shape."""
    lib().net_tune_clear()


class Queue:
    """netq_*: continuous-batching request queue on the current device."""

    def __init__(self, mem_budget_bytes, max_slots, opts: net_opts | None = None):
        L = lib()
        h = C.c_void_p()
        _check(L.netq_create(int(mem_budget_bytes), int(max_slots),
                             C.byref(opts) if opts is not None else None, C.byref(h)),
               "netq_create")
        self.h = h

    def submit(self, dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, periodic=()):
        keep, ptrs, bdt, dev, _ = marshal_planes(planes, len(dims))
        if dev:
            raise TypeError("queue requests take host (numpy) bond planes")
        desc = make_desc(dims, flow_axis, p_in, p_out, bdt, 0, None, periodic)
        t = C.c_uint64()
        _check(lib().netq_submit(self.h, C.byref(desc), ptrs, C.byref(t)), "netq_submit")
        return t.value

    def poll(self, ticket):
        r = net_result()
        st = lib().netq_poll(self.h, C.c_uint64(ticket), C.byref(r))
        return st, (self._result(st, r) if st != NET_EBUSY else None)

    def wait(self, ticket, timeout_ms=-1):
        r = net_result()
        st = lib().netq_wait(self.h, C.c_uint64(ticket), int(timeout_ms), C.byref(r))
        return st, (self._result(st, r) if st != NET_ETIMEOUT else None)

    @staticmethod
    def _result(st, r):
        res = Result.from_c(r)
        if st != NET_OK:
            res.error = lib().net_last_error().decode(errors="replace")
        return res

    def cancel(self, ticket):
        return lib().netq_cancel(self.h, C.c_uint64(ticket))

    def stats(self):
        p50, p99, n = C.c_double(), C.c_double(), C.c_uint64()
        _check(lib().netq_stats(self.h, C.byref(p50), C.byref(p99), C.byref(n)), "netq_stats")
        return p50.value, p99.value, n.value

    def close(self):
        if getattr(self, "h", None):
            lib().netq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve(dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, precision=NET_MIXED, **kw):
    """net_create + net_solve + read-back in one call; returns (Result, P)."""
    with Network(dims, planes, flow_axis, p_in, p_out) as net:
        r = net.solve(make_opts(precision=precision, **kw))
        return r, net.pressure()
