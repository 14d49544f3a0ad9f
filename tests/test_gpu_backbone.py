"""Dead-end stripping on the GPU: the backbone mask is bit-exact against the
oracle's, the linear system shrinks to it (n_solved), and G_eff and every
node's pressure (the stripped ones included) still match the FP64 oracle,
which solves the whole spanning cluster.

Two levels: the default removes dead-end trees and then dead-end loops (the
current-carrying backbone: the block of the extra inlet-outlet edge, checked
against oracle.backbone_blocks); NETSOLVE_PRUNE=trees removes the trees only
(checked against oracle.backbone)."""
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


CASES = [((40, 33), 0, 0.6, 1, ()), ((29, 41), 1, 0.58, 2, ()), ((23, 19, 17), 0, 0.36, 3, ()),
         ((18, 21, 20), 2, 0.34, 4, ()), ((64, 64, 64), 1, 0.28, 5, ()), ((300, 257), 0, 0.55, 6, ()),
         ((45, 38), 0, 0.58, 7, (1,)), ((21, 19, 18), 0, 0.33, 8, (1, 2)), ((3, 40, 37), 0, 0.6, 9, ()),
         ((130, 5, 4), 0, 0.5, 10, ())]


def oracle_backbone(level, dims, planes, f, per):
    if level == "trees":
        return oracle.backbone(dims, planes, flow_axis=f, periodic=per)
    return oracle.backbone_blocks(dims, planes, flow_axis=f, periodic=per)


@pytest.mark.parametrize("dims,f,p,seed,per", CASES)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("level", ["blocks", "trees"])
def test_backbone_and_solution_match_oracle(ns, monkeypatch, dims, f, p, seed, per, precision, level):
    if level == "trees":
        monkeypatch.setenv("NETSOLVE_PRUNE", "trees")
    gen = netgen.rng(9500 + seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, periodic=per), p, gen)
    ref = oracle.solve(dims, planes, flow_axis=f, tol=1e-13, periodic=per)
    bb_ref = oracle_backbone(level, dims, planes, f, per)
    with ns.Network(dims, planes, flow_axis=f, periodic=per) as net:
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
        assert r.n_solved == rq.n_solved == int(oracle.backbone_blocks(dims, planes).sum())
        if ref.g_eff > 0:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL and rel(rq.g_eff, ref.g_eff) <= G_TOL


def test_loops_stripped_beyond_trees(ns, monkeypatch):
    """At near-threshold disorder the block backbone is strictly smaller than
    the tree-stripped set, and both give the same G and pressures."""
    gen = netgen.rng(9800)
    dims = (40, 36, 34)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.3, gen)
    with ns.Network(dims, planes) as net:
        a = net.solve()
        Pa = net.pressure()
    monkeypatch.setenv("NETSOLVE_PRUNE", "trees")
    with ns.Network(dims, planes) as net:
        b = net.solve()
        Pb = net.pressure()
    assert a.n_solved < b.n_solved < b.n_active == a.n_active
    assert a.n_solved == int(oracle.backbone_blocks(dims, planes).sum())
    assert rel(a.g_eff, b.g_eff) <= G_TOL
    assert np.max(np.abs(Pa - Pb)) <= 1e-7


def test_hand_made_dead_end_loop(ns):
    """The oracle's hand-made 9 x 7 network: two parallel paths, a dead-end
    loop and a dead-end tree on stems, a branch into the outlet face."""
    dims = (9, 7)
    gx = np.zeros((7, 8))
    gy = np.zeros((6, 9))
    gx[3, :] = 1.0
    gx[6, :] = 1.5
    gy[2, 4] = 2.0
    gx[2, 4] = gy[1, 5] = gx[1, 4] = gy[1, 4] = 2.0
    gy[2, 2] = gy[1, 2] = gy[0, 2] = 3.0
    gy[2, 7] = gx[2, 7] = 0.5
    gy[5, 3] = 2.5
    gx[5, 3] = gy[4, 4] = gx[4, 3] = gy[4, 3] = 2.5
    want = np.zeros((7, 9), bool)
    want[3, 1:8] = True
    want[6, 1:8] = True
    want[2, 7] = True
    ref = oracle.solve(dims, [gx, gy], tol=1e-14)
    with ns.Network(dims, [gx, gy]) as net:
        bb = net.backbone()
        r = net.solve()
        P = net.pressure()
    np.testing.assert_array_equal(bb, want)
    assert r.n_solved == int(want.sum())
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7


def _edge_cases():
    out = []
    gen = netgen.rng(9900)
    # n_f = 3: every interior node touches both faces
    out.append(((3, 17), 0, (), netgen.percolate(netgen.lognormal_iid((3, 17), gen), 0.6, gen)))
    # a chain (ny = 1): one closed bond cuts it, otherwise one path
    g = netgen.lognormal_iid((12, 1), gen)
    out.append(((12, 1), 0, (), g))
    g2 = [x.copy() for x in g]
    g2[0][0, 5] = 0.0
    out.append(((12, 1), 0, (), g2))
    # tiny 3D and periodic extent 3
    out.append(((3, 3, 3), 0, (), netgen.percolate(netgen.lognormal_iid((3, 3, 3), gen), 0.7, gen)))
    out.append(((6, 3, 4), 0, (1,), netgen.percolate(netgen.lognormal_iid((6, 3, 4), gen, periodic=(1,)), 0.6, gen)))
    # fully open but one bond: everything carries current
    g3 = netgen.lognormal_iid((20, 15), gen)
    g3[1][7, 9] = 0.0
    out.append(((20, 15), 0, (), g3))
    # two spanning paths joined only through the faces, with a loop on one
    gx = np.zeros((6, 9))
    gy = np.zeros((5, 10))
    gx[1, :] = 1.0
    gx[4, :] = 2.0
    gy[1, 4] = gy[2, 4] = 1.0   # stem (4,1)-(4,2)-(4,3), dead end
    gx[3, 4] = gy[2, 5] = 1.0   # (4,3)-(5,3)-(5,2)... a loop hanging from the stem
    gx[2, 4] = 1.0
    out.append(((10, 6), 0, (), [gx, gy]))
    # FP32 raw conductances, flow along y
    g4 = [x.astype(np.float32) for x in netgen.percolate(netgen.lognormal_iid((30, 40), gen), 0.58, gen)]
    out.append(((30, 40), 1, (), g4))
    return out


@pytest.mark.parametrize("case", range(8))
def test_backbone_edge_cases(ns, case):
    dims, f, per, planes = _edge_cases()[case]
    want = oracle.backbone_blocks(dims, planes, flow_axis=f, periodic=per)
    ref = oracle.solve(dims, planes, flow_axis=f, tol=1e-13, periodic=per)
    with ns.Network(dims, planes, flow_axis=f, periodic=per) as net:
        bb = net.backbone()
        r = net.solve()
        P = net.pressure()
    np.testing.assert_array_equal(bb, want)
    assert r.n_solved == int(want.sum())
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
    else:
        assert r.status == ns.NET_OK
        assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert np.max(np.abs(P - ref.P)) <= 1e-7
