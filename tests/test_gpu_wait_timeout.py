"""Failure detection on the device: the grid-barrier waits of the two
cooperative inner-solve kernels (the persistent 2D kernel and the compacted
solve) are bounded in time, and a wait that runs out ends the solve with
NET_ETIMEOUT instead of hanging the GPU.

The failure is made without faulting anything: NETSOLVE_WITHHOLD_ARRIVAL
tells one CTA to skip its first grid-barrier arrival (a flag that nothing
else will set), and NETSOLVE_WAIT_NS shortens the limit to 20 ms.  Every
other CTA's wait then runs out, sets the error word and returns; the host
reports the status, and the next solve of the same network on the same
device converges to the oracle's answer.
"""
import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen

pytestmark = pytest.mark.gpu
G_TOL = 1e-8


@pytest.fixture(scope="module")
def ns():
    import torch

    assert torch.cuda.is_available()
    from paper_1908_03301_gb300 import netsolve

    netsolve.lib(build_if_missing=True)
    return netsolve


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("kernel,dims,p", [("persist", (300, 260), 1.0), ("compact", (40, 36, 30), 0.33),
                                           ("compact", (200, 150), 0.62)])
def test_withheld_arrival_times_out_then_recovers(ns, monkeypatch, kernel, dims, p):
    import time

    gen = netgen.rng(8800 + len(dims))
    planes = netgen.lognormal_iid(dims, gen, 1.0)
    if p < 1.0:
        planes = netgen.percolate(planes, p, gen)
    ref = oracle.solve(dims, planes, tol=1e-13)
    monkeypatch.setenv("NETSOLVE_KERNEL", kernel)
    with ns.Network(dims, planes) as net:
        monkeypatch.setenv("NETSOLVE_WAIT_NS", "20000000")
        monkeypatch.setenv("NETSOLVE_WITHHOLD_ARRIVAL", "0")
        t = time.perf_counter()
        r = net.solve(check=False)
        dt = time.perf_counter() - t
        assert r.status == ns.NET_ETIMEOUT, r
        assert "bounded device wait" in ns.last_error()
        assert dt < 10.0  # gave up after the short limit, no hang
        monkeypatch.delenv("NETSOLVE_WITHHOLD_ARRIVAL")
        monkeypatch.delenv("NETSOLVE_WAIT_NS")
        r2 = net.solve()
        P = net.pressure()
    assert r2.status == ns.NET_OK, r2
    assert rel(r2.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7
    # and a fresh network on the same device still solves
    with ns.Network(dims, planes) as net:
        r3 = net.solve()
    assert r3.status == ns.NET_OK and rel(r3.g_eff, ref.g_eff) <= G_TOL
