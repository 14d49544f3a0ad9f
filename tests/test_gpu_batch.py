"""Batched solves (net_solve_batch) and the continuous-batching queue.

Each network's result in a batch or in the queue must equal its stand-alone
net_solve within the solver's accuracy target (1e-8 relative effective
conductance) and match the FP64 oracle to the same tolerance.
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


def mixed_nets(count, seed0=0, with3d=True):
    nets = []
    for i in range(count):
        if with3d and i % 4 == 3:
            gen = netgen.rng(5000 + seed0 + i)
            s = int(gen.integers(8, 28))
            dims = (s, s + 3, s + 1)
            planes = netgen.lognormal_iid(dims, gen, 1.0)
            if i % 8 == 7:
                planes = netgen.percolate(planes, 0.4, gen)
            nets.append((dims, planes))
        else:
            nets.append(netgen.batch_instance(seed0 + i, smin=24, smax=180))
    return nets


def solo(ns, dims, planes, precision=0):
    with ns.Network(dims, planes) as net:
        return net.solve(ns.make_opts(precision=precision))


def test_batch_matches_solo_and_oracle(ns):
    specs = mixed_nets(14, seed0=0)
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets)
    for (dims, planes), net, r in zip(specs, nets, res):
        assert r.status == ns.NET_OK, r
        s = solo(ns, dims, planes)
        if s.g_eff == 0.0:
            assert r.g_eff == 0.0
            continue
        assert rel(r.g_eff, s.g_eff) <= G_TOL
        ref = oracle.solve(dims, planes, tol=1e-13)
        assert rel(r.g_eff, ref.g_eff) <= G_TOL
        P = net.pressure()
        assert np.max(np.abs(P - ref.P)) <= 1e-7
    for net in nets:
        net.close()


def test_batch_fp64_and_determinism(ns):
    specs = mixed_nets(8, seed0=40)
    nets = [ns.Network(d, p) for d, p in specs]
    r1 = ns.solve_batch(nets, ns.make_opts(precision=ns.NET_FP64))
    r2 = ns.solve_batch(nets, ns.make_opts(precision=ns.NET_FP64))
    for (dims, planes), a, b in zip(specs, r1, r2):
        assert a.status == ns.NET_OK and b.status == ns.NET_OK
        assert a.g_eff == b.g_eff and a.inner_iters == b.inner_iters
        ref = oracle.solve(dims, planes, tol=1e-13)
        if ref.g_eff > 0:
            assert rel(a.g_eff, ref.g_eff) <= G_TOL
    m1 = ns.solve_batch(nets)
    m2 = ns.solve_batch(nets)
    assert [x.g_eff for x in m1] == [x.g_eff for x in m2]
    for net in nets:
        net.close()


def test_batch_degenerate_members(ns):
    dims = (20, 12)
    gen = netgen.rng(9)
    cut = netgen.lognormal_iid(dims, gen)
    cut[0][:, 7] = 0.0  # no spanning cluster
    uni = netgen.uniform((33, 17), 2.0)
    specs = [(dims, cut), ((33, 17), uni)] + mixed_nets(3, seed0=70, with3d=False)
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets)
    assert res[0].g_eff == 0.0 and res[0].n_active == 0
    assert rel(res[1].g_eff, 2.0 * 17 / 32) <= 1e-12
    for net in nets:
        net.close()
    assert ns.solve_batch([]) == []


def test_queue_results_match_solo_and_oracle(ns):
    """Requests finish at different steps and their networks are released at
    once while others keep running (30 requests, 6 slots, 2D and 3D); every
    result equals the stand-alone solve and the oracle."""
    specs = mixed_nets(30, seed0=100)
    with ns.Queue(mem_budget_bytes=96 << 20, max_slots=6) as q:
        tickets = [q.submit(d, p) for d, p in specs]
        results = [q.wait(t, timeout_ms=120000) for t in tickets]
        p50, p99, n = q.stats()
    assert n == len(specs) and 0 < p50 <= p99
    for (dims, planes), (st, r) in zip(specs, results):
        assert st == ns.NET_OK, (st, r)
        s = solo(ns, dims, planes)
        ref = oracle.solve(dims, planes, tol=1e-13)
        if s.g_eff == 0.0:
            assert r.g_eff == 0.0 and ref.g_eff == 0.0
        else:
            assert rel(r.g_eff, s.g_eff) <= G_TOL
            assert rel(r.g_eff, ref.g_eff) <= G_TOL


def test_queue_admits_requests_while_others_run(ns):
    """Continuous batching: a slow request (a 2048^2 network near the 2D
    percolation threshold) is admitted first; small requests that arrive
    while it runs are admitted onto the device beside it (co_running >= 1,
    with a measured wait), and every result matches the oracle (the slow one
    its stand-alone solve)."""
    import time

    gen = netgen.rng(6200)
    big_dims = (2048, 2048)
    big = (big_dims, netgen.percolate(netgen.lognormal_iid(big_dims, gen, 1.0), 0.53, gen))
    smalls = [netgen.batch_instance(400 + i, smin=40, smax=120) for i in range(6)]
    with ns.Queue(mem_budget_bytes=8 << 30, max_slots=8) as q:
        tb = q.submit(*big)
        time.sleep(0.1)
        ts = []
        for d, p in smalls:
            ts.append(q.submit(d, p))
            time.sleep(0.01)
        small_res = [q.wait(t, timeout_ms=120000) for t in ts]
        big_res = q.wait(tb, timeout_ms=300000)
    assert big_res[0] == ns.NET_OK, big_res
    assert big_res[1].co_running == 0
    beside = [r.co_running for _, r in small_res]
    assert max(beside) >= 1, beside  # admitted while the slow one was on the device
    for (dims, planes), (st, r) in zip(smalls, small_res):
        assert st == ns.NET_OK, (st, r)
        assert r.queue_ms >= 0.0
        ref = oracle.solve(dims, planes, tol=1e-13)
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
        else:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL
    a = solo(ns, *big)
    assert rel(big_res[1].g_eff, a.g_eff) <= G_TOL


def test_batch_wide_members_match_oracle(ns):
    """Members as wide as the 512-network workload's widest (1024, 760 and
    540 columns: sweep stages of only two or three rows) beside small ones,
    lognormal and percolated: every member's G_eff and pressures against the
    oracle."""
    shapes = [(1024, 48), (760, 40), (540, 64), (96, 80), (33, 150), (1024, 9)]
    specs = []
    for i, dims in enumerate(shapes):
        gen = netgen.rng(6100 + i)
        planes = netgen.lognormal_iid(dims, gen, 1.0)
        if i % 2:
            planes = netgen.percolate(planes, 0.6, gen)
        specs.append((dims, planes))
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets)
    for (dims, planes), net, r in zip(specs, nets, res):
        assert r.status == ns.NET_OK, (dims, r)
        ref = oracle.solve(dims, planes, tol=1e-13)
        P = net.pressure()
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
        else:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL, (dims, r.g_eff, ref.g_eff)
        assert np.max(np.abs(P - ref.P)) <= 1e-7, dims
    for net in nets:
        net.close()


def test_queue_budget_cancel_and_errors(ns):
    with ns.Queue(mem_budget_bytes=8 << 20, max_slots=1) as q:
        big = netgen.uniform((1024, 1024))
        with pytest.raises(ns.NetError) as ei:
            q.submit((1024, 1024), big)
        assert ei.value.status == ns.NET_EBUDGET
        bad = netgen.uniform((30, 30))
        bad[0][3, 4] = -2.0
        tb = q.submit((30, 30), bad)
        specs = mixed_nets(6, seed0=200, with3d=False)
        ts = [q.submit(d, p) for d, p in specs]
        c = q.cancel(ts[-1])
        assert c in (ns.NET_OK, ns.NET_EBUSY)
        st, r = q.wait(tb, timeout_ms=60000)
        assert st == ns.NET_EINVAL
        assert "negative" in r.error and f"request {tb}" in r.error
        for t in ts[:-1]:
            st, r = q.wait(t, timeout_ms=60000)
            assert st == ns.NET_OK and r.error == ""
        st, r = q.wait(ts[-1], timeout_ms=60000)
        assert st == (ns.NET_ECANCELLED if c == ns.NET_OK else ns.NET_OK)
        if c == ns.NET_OK:
            assert "cancelled" in r.error
        # a read ticket is gone
        st, _ = q.poll(ts[0])
        assert st == ns.NET_EINVAL


def test_queue_reports_not_converged(ns):
    """A request that cannot meet its tolerance within max_outer refinement
    steps ends NET_ENOTCONVERGED, and its message reaches the caller."""
    opts = ns.make_opts(tol_rel=1e-15, tol_geff=1e-15, max_outer=1)
    dims, planes = netgen.batch_instance(3, smin=64, smax=96)
    with ns.Queue(mem_budget_bytes=64 << 20, max_slots=2, opts=opts) as q:
        t = q.submit(dims, planes)
        st, r = q.wait(t, timeout_ms=60000)
    assert st == ns.NET_ENOTCONVERGED
    assert r.outer_iters == 1 and "not converged" in r.error


def test_near_critical_3d_converges_alone_and_in_batch(ns):
    """A 110^3 near-critical percolation network (p = 0.26, lognormal
    conductances) whose FP64 inner solves plateau for hundreds of iterations:
    it must converge in a few refinement steps both alone and in a batch."""
    dims, planes = netgen.request_instance(7)
    assert dims == (110, 110, 110)
    a = solo(ns, dims, planes)
    assert a.status == ns.NET_OK and a.outer_iters <= 20, a
    others = mixed_nets(5, seed0=300, with3d=False)
    nets = [ns.Network(dims, planes)] + [ns.Network(d, p) for d, p in others]
    res = ns.solve_batch(nets)
    for net in nets:
        net.close()
    assert all(r.status == ns.NET_OK for r in res)
    assert res[0].outer_iters <= 20
    assert rel(res[0].g_eff, a.g_eff) <= G_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_on_lists_matches_oracle(ns, monkeypatch, precision):
    """Every member of a mixed 2D/3D batch forced onto the batched compacted
    path (phase launches over list segments, one last-arriver reduction per
    network), in both precisions: G_eff and pressures against the oracle."""
    monkeypatch.setenv("NETSOLVE_BATCH_COMPACT_BELOW", "1.01")
    specs = mixed_nets(10, seed0=500)
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets, ns.make_opts(precision=precision))
    for (dims, planes), net, r in zip(specs, nets, res):
        assert r.status == ns.NET_OK, r
        ref = oracle.solve(dims, planes, tol=1e-13)
        P = net.pressure()
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
        else:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert np.max(np.abs(P - ref.P)) <= 1e-7
    for net in nets:
        net.close()
