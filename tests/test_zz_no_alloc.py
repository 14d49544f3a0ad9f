"""net_labels_noalloc: the cluster labelling entry point that allocates no
memory (for callers that cannot allocate device memory: a framework whose pool
owns all device memory, or a loop where cudaMalloc/cudaFree would block).

Its output must equal the regular path (net_create + net_get_labels) bit for
bit - the labels are integers - on two calls in a row that share the
library's fixed scratch array.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_03301_gb300 import netgen

pytestmark = pytest.mark.gpu


def _noalloc_labels(ns, dims, planes, flow_axis=0):
    import torch

    L = ns.lib(build_if_missing=True)
    tpl = [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in planes]
    N = int(np.prod(dims))
    lab = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    cls = torch.full((N,), 99, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    bdt = ns.NET_F32 if planes[0].dtype == np.float32 else ns.NET_F64
    desc = ns.make_desc(dims, flow_axis, 1.0, 0.0, bdt, 1, stream.cuda_stream)
    ptrs = (ctypes.c_void_p * 3)(*([t.data_ptr() for t in tpl] + [None] * (3 - len(tpl))))
    st = L.net_labels_noalloc(ctypes.byref(desc), ptrs, lab.data_ptr(), cls.data_ptr())
    assert st == ns.NET_OK, L.net_last_error()
    shape = tuple(reversed(dims))
    return lab.cpu().numpy().reshape(shape), cls.cpu().numpy().reshape(shape)


def _regular_labels(ns, dims, planes, flow_axis=0):
    with ns.Network(dims, planes, flow_axis) as net:
        return net.labels()


def test_noalloc_labels_match_regular_path_twice():
    from paper_1908_03301_gb300 import netsolve as ns

    cases = [netgen.workload_perc3d(n=64, p=0.26, seed=31) + (0,),
             (lambda d, pl: (d, pl, 1))(*netgen.batch_instance(2, smin=700, smax=1000))]
    for dims, planes, f in cases:  # two calls in a row on the shared scratch
        got_l, got_c = _noalloc_labels(ns, dims, planes, f)
        ref_l, ref_c = _regular_labels(ns, dims, planes, f)
        np.testing.assert_array_equal(got_l, ref_l)
        np.testing.assert_array_equal(got_c, ref_c)


def test_noalloc_rejects_oversize_request():
    import torch

    from paper_1908_03301_gb300 import netsolve as ns

    L = ns.lib(build_if_missing=True)
    dims = (1100, 1000)  # 1.1e6 nodes > 2^20
    desc = ns.make_desc(dims, 0, 1.0, 0.0, ns.NET_F64, 1, None)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * 3)(buf.data_ptr(), buf.data_ptr(), None)
    st = L.net_labels_noalloc(ctypes.byref(desc), ptrs, buf.data_ptr(), buf.data_ptr())
    assert st == ns.NET_EINVAL
    assert b"scratch" in L.net_last_error()
