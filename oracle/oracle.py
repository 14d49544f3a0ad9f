"""ctypes front end of the plain-C FP64 oracle (``netoracle.c``), plus the
numpy oracles of the input-side steps: sorted-removal percolation and the FBM
generator (Eq. 1, Eq. 2) with its conductance map.

Test infrastructure: the CUDA solver never imports this module.

Input conventions match the rest of the project: ``dims = (nx, ny[, nz])``,
bond planes as numpy arrays of shape node-shape with the extent along their own
direction reduced by one (x fastest, numpy order (z, y, x)).  Planes of any
float dtype are widened to float64 exactly before the call.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "netoracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

CLS_ISOLATED, CLS_INLET, CLS_OUTLET, CLS_SPANNING, CLS_FACE_IN, CLS_FACE_OUT = range(6)


class _Desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int64 * 3), ("flow_axis", C.c_int),
                ("p_in", C.c_double), ("p_out", C.c_double), ("periodic", C.c_uint)]


class _Res(C.Structure):
    _fields_ = [("g_eff", C.c_double), ("k_eff", C.c_double), ("q_in", C.c_double),
                ("q_out", C.c_double), ("rel_residual", C.c_double),
                ("max_imbalance", C.c_double), ("energy_g", C.c_double),
                ("n_active", C.c_int64), ("iters", C.c_int64), ("status", C.c_int)]


@dataclass
class OracleResult:
    g_eff: float
    k_eff: float
    q_in: float
    q_out: float
    rel_residual: float
    max_imbalance: float
    energy_g: float
    n_active: int
    iters: int
    status: int
    P: np.ndarray
    label: np.ndarray
    cls: np.ndarray


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp3 = C.POINTER(C.c_double) * 3
        lib.or_labels.argtypes = [C.POINTER(_Desc), dp3, C.c_void_p, C.c_void_p]
        lib.or_labels.restype = C.c_int
        lib.or_backbone.argtypes = [C.POINTER(_Desc), dp3, C.c_void_p]
        lib.or_backbone.restype = C.c_int
        lib.or_backbone_blocks.argtypes = [C.POINTER(_Desc), dp3, C.c_void_p]
        lib.or_backbone_blocks.restype = C.c_int
        lib.or_residual.argtypes = [C.POINTER(_Desc), dp3, C.c_void_p, C.c_void_p]
        lib.or_residual.restype = C.c_int
        lib.or_solve.argtypes = [C.POINTER(_Desc), dp3, C.c_double, C.c_int64, C.c_int,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Res)]
        lib.or_solve.restype = C.c_int
        lib.or_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def _mask(periodic):
    """Axes (iterable of 0/1/2) -> bit mask."""
    m = 0
    for a in periodic:
        m |= 1 << int(a)
    return m


def _prep(dims, planes, flow_axis, p_in, p_out, periodic=()):
    ndim = len(dims)
    n = list(int(v) for v in dims) + [1] * (3 - ndim)
    mask = _mask(periodic)
    desc = _Desc(ndim, (C.c_int64 * 3)(*n), int(flow_axis), float(p_in), float(p_out), mask)
    arrs = []
    for d in range(ndim):
        want = list(n)
        if not (mask >> d) & 1:
            want[d] -= 1
        a = np.ascontiguousarray(planes[d], dtype=np.float64)
        if a.size != int(np.prod(want)):
            raise ValueError(f"bond plane {d} has {a.size} entries, expected {int(np.prod(want))}")
        arrs.append(a)
    while len(arrs) < 3:
        arrs.append(np.zeros(1))
    ptrs = (C.POINTER(C.c_double) * 3)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
    N = int(np.prod(n))
    shape = tuple(reversed(n[:ndim]))
    return desc, ptrs, arrs, N, shape


def labels(dims, planes, flow_axis=0, periodic=()):
    """Canonical cluster labels (int32) and classes (uint8), node-shaped.
    ``periodic``: transverse axes with periodic boundaries (their bond planes
    have the full node extent along that axis)."""
    lib = _load()
    desc, ptrs, keep, N, shape = _prep(dims, planes, flow_axis, 1.0, 0.0, periodic)
    lab = np.empty(N, np.int32)
    cls = np.empty(N, np.uint8)
    if lib.or_labels(C.byref(desc), ptrs, lab.ctypes.data, cls.ctypes.data) != 0:
        raise ValueError("invalid network")
    return lab.reshape(shape), cls.reshape(shape)


def backbone(dims, planes, flow_axis=0, periodic=()):
    """Spanning-cluster nodes left after stripping dead-end trees (bool,
    node-shaped); every other node is False."""
    lib = _load()
    desc, ptrs, keep, N, shape = _prep(dims, planes, flow_axis, 1.0, 0.0, periodic)
    out = np.empty(N, np.uint8)
    if lib.or_backbone(C.byref(desc), ptrs, out.ctypes.data) != 0:
        raise ValueError("invalid network")
    return out.reshape(shape).astype(bool)


def backbone_blocks(dims, planes, flow_axis=0, periodic=()):
    """Current-carrying backbone (bool, node-shaped): the interior nodes of
    the biconnected component that holds the extra edge between the two faces
    (each face taken as one vertex) -- the nodes on a path from the inlet face
    to the outlet face that visits no node twice.  Dead-end trees and dead-end
    loops are both left out."""
    lib = _load()
    desc, ptrs, keep, N, shape = _prep(dims, planes, flow_axis, 1.0, 0.0, periodic)
    out = np.empty(N, np.uint8)
    if lib.or_backbone_blocks(C.byref(desc), ptrs, out.ctypes.data) != 0:
        raise ValueError("invalid network")
    return out.reshape(shape).astype(bool)


def residual(dims, planes, P, flow_axis=0, periodic=()):
    """Nodal imbalance sum_j g_ij (P_j - P_i) at interior nodes (0 on faces)."""
    lib = _load()
    desc, ptrs, keep, N, shape = _prep(dims, planes, flow_axis, 1.0, 0.0, periodic)
    Pc = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
    out = np.empty(N, np.float64)
    if lib.or_residual(C.byref(desc), ptrs, Pc.ctypes.data, out.ctypes.data) != 0:
        raise ValueError("invalid network")
    return out.reshape(shape)


def solve(dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, tol=1e-13, max_iter=10**7,
          nthreads=0, periodic=()) -> OracleResult:
    """FP64 Jacobi-PCG solve of Eq. 3 plus the flows of Eq. 4."""
    lib = _load()
    desc, ptrs, keep, N, shape = _prep(dims, planes, flow_axis, p_in, p_out, periodic)
    P = np.empty(N, np.float64)
    lab = np.empty(N, np.int32)
    cls = np.empty(N, np.uint8)
    res = _Res()
    lib.or_solve(C.byref(desc), ptrs, float(tol), int(max_iter), int(nthreads),
                 P.ctypes.data, lab.ctypes.data, cls.ctypes.data, C.byref(res))
    if res.status < 0:
        raise ValueError("invalid network")
    return OracleResult(res.g_eff, res.k_eff, res.q_in, res.q_out, res.rel_residual,
                        res.max_imbalance, res.energy_g, int(res.n_active), int(res.iters),
                        int(res.status), P.reshape(shape), lab.reshape(shape),
                        cls.reshape(shape))


def max_threads() -> int:
    return int(_load().or_max_threads())


def close_smallest(planes, q):
    """Correlated percolation by sorted removal (Sec. VI.B): of all M bonds
    (the planes concatenated in plane order, each in its own x-fastest
    order), close (set to 0) the floor(q M) with the smallest conductance;
    equal conductances are taken in that position order.  A stable sort is
    the whole method here.  Returns new planes of the input dtype."""
    if not (0.0 <= q <= 1.0):
        raise ValueError("q must lie in [0, 1]")
    flat = np.concatenate([np.asarray(g).reshape(-1) for g in planes]).astype(np.float64)
    if not np.all(np.isfinite(flat)) or np.any(flat < 0):
        raise ValueError("conductances must be finite and non-negative")
    k = int(np.floor(q * flat.size))
    order = np.argsort(flat, kind="stable")
    closed = np.zeros(flat.size, bool)
    closed[order[:k]] = True
    out, o = [], 0
    for g in planes:
        g = np.asarray(g)
        c = closed[o:o + g.size].reshape(g.shape)
        out.append(np.where(c, g.dtype.type(0), g))
        o += g.size
    return out


def fbm_field(noise, hurst, beta=None):
    """Fractional Brownian motion by spectral filtering (Eq. 1, Eq. 2).

    ``noise``: complex white noise, node-shaped (numpy order (z, y, x)); the
    random draws are an input.  Each Fourier mode is weighted by the square
    root of the spectral density, S ~ (sum_a beta_a w_a^2)^-(H + d/2) with
    w_a the discrete frequencies (cycles per node, numpy's fftfreq) and d the
    dimension (Eq. 1: d = 2 and beta = 1 give (w_x^2 + w_y^2)^-(H+1); Eq. 2:
    the anisotropic betas); the zero mode is dropped.  The field is the real
    part of the inverse transform, shifted and scaled to zero mean and unit
    variance (population).  ``beta`` is per lattice axis (x, y[, z]), default 1.
    """
    noise = np.asarray(noise, dtype=np.complex128)
    shape = noise.shape
    d = len(shape)
    if beta is None:
        beta = (1.0,) * d
    k2 = np.zeros(shape)
    for ax in range(d):
        lattice_axis = d - 1 - ax           # numpy axis ax is lattice axis d-1-ax
        w = np.fft.fftfreq(shape[ax])
        sh = [1] * d
        sh[ax] = shape[ax]
        k2 = k2 + float(beta[lattice_axis]) * (w * w).reshape(sh)
    k2.flat[0] = 1.0
    amp = k2 ** (-(2.0 * hurst + d) / 4.0)
    amp.flat[0] = 0.0
    field = np.fft.ifftn(noise * amp).real
    field = field - field.mean()
    sd = np.sqrt(np.mean(field * field))
    return field / sd if sd > 0 else field


def fbm_bonds(field, sigma):
    """Conductances g = exp(sigma * B_b), B_b the mean of the bond's two end
    nodes of the field (the workloads' map); planes in the project's layout."""
    field = np.asarray(field, dtype=np.float64)
    nd = field.ndim
    out = []
    for d in range(nd):
        ax = nd - 1 - d
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        out.append(np.exp(sigma * 0.5 * (field[tuple(lo)] + field[tuple(hi)])))
    return out
