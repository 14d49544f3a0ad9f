"""Dead-end stripping on the GPU: the backbone mask is bit-exact against the
oracle's, the linear system shrinks to it (n_solved), and G_eff and every
node's pressure (the stripped ones included) still match the FP64 oracle,
which solves the whole spanning cluster."""
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


CASES = [((40, 33), 0, 0.6, 1), ((29, 41), 1, 0.58, 2), ((23, 19, 17), 0, 0.36, 3),
         ((18, 21, 20), 2, 0.34, 4), ((64, 64, 64), 1, 0.28, 5), ((300, 257), 0, 0.55, 6)]


@pytest.mark.parametrize("dims,f,p,seed", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_backbone_and_solution_match_oracle(ns, dims, f, p, seed, precision):
    gen = netgen.rng(9500 + seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), p, gen)
    ref = oracle.solve(dims, planes, flow_axis=f, tol=1e-13)
    bb_ref = oracle.backbone(dims, planes, flow_axis=f)
    with ns.Network(dims, planes, flow_axis=f) as net:
        bb = net.backbone()
        r = net.solve(ns.make_opts(precision=precision))
        P = net.pressure()
        lab, cls = net.labels()
    np.testing.assert_array_equal(bb, bb_ref)
    np.testing.assert_array_equal(cls, ref.cls)
    np.testing.assert_array_equal(lab, ref.label)
    assert r.n_active == ref.n_active and r.n_solved == int(bb_ref.sum())
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
        return
    assert r.status == ns.NET_OK
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7


def test_stripping_off_gives_the_same_answer(ns, monkeypatch):
    gen = netgen.rng(9600)
    dims = (48, 44, 40)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.3, gen)
    with ns.Network(dims, planes) as net:
        a = net.solve()
        Pa = net.pressure()
    monkeypatch.setenv("NETSOLVE_PRUNE", "0")
    with ns.Network(dims, planes) as net:
        b = net.solve()
        Pb = net.pressure()
        assert not (net.backbone() != (net.labels()[1] == 3)).any()
    assert b.n_solved == b.n_active and a.n_solved < a.n_active
    assert rel(a.g_eff, b.g_eff) <= G_TOL
    assert np.max(np.abs(Pa - Pb)) <= 1e-7


def test_unpercolated_network_keeps_every_node(ns):
    dims, planes, _ = netgen.workload_small("random")
    with ns.Network(dims, planes) as net:
        r = net.solve()
        assert net.backbone().sum() == r.n_active == r.n_solved


def test_backbone_in_batch_and_queue(ns):
    specs = []
    for i in range(6):
        gen = netgen.rng(9700 + i)
        dims = (30 + 7 * i, 26 + 5 * i) if i % 2 else (14 + i, 13, 12 + i)
        planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.62 if i % 2 else 0.38, gen)
        specs.append((dims, planes))
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets)
    for n in nets:
        n.close()
    with ns.Queue(mem_budget_bytes=64 << 20, max_slots=3) as q:
        qres = [q.wait(q.submit(d, p), timeout_ms=60000) for d, p in specs]
    for (dims, planes), r, (st, rq) in zip(specs, res, qres):
        ref = oracle.solve(dims, planes, tol=1e-13)
        assert st == ns.NET_OK and r.status == ns.NET_OK
        assert r.n_solved == rq.n_solved == int(oracle.backbone(dims, planes).sum())
        if ref.g_eff > 0:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL and rel(rq.g_eff, ref.g_eff) <= G_TOL
