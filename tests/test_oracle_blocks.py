"""Pins of the oracle's current-carrying backbone (``oracle.backbone_blocks``:
Sec. V and VI.B say that near the percolation threshold most of the spanning
cluster carries no flow).

Definition pinned: with every inlet-face node taken as one vertex A and every
outlet-face node as one vertex B, a node carries current (for generic
conductances) exactly when it lies on a path from A to B that visits no vertex
twice.  The oracle computes it as the biconnected component of the extra edge
A-B (a Hopcroft-Tarjan search); these tests check it against
* that definition by brute force over all such paths on tiny networks,
* networkx's biconnected components in two formulations (the extra edge A-B;
  and both faces merged into one vertex S, where the current-carrying nodes
  are the spanning-cluster nodes of the blocks that contain S -- on spanning
  clusters the two agree),
* a hand-made network with a dead-end loop, a dead-end tree, a parallel path
  and a branch into the outlet face,
* exactness: closing every bond of the removed nodes leaves G unchanged and
  no current flows through them in the full solve.
"""
import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen
from tests import _independent as ind


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _random_small(seed):
    gen = netgen.rng(7700 + seed)
    if gen.random() < 0.5:
        dims = (int(gen.integers(3, 8)), int(gen.integers(1, 6)))
    else:
        dims = (int(gen.integers(3, 5)), int(gen.integers(1, 4)), int(gen.integers(1, 4)))
    f = int(gen.integers(0, len(dims)))
    if dims[f] < 3:
        f = 0
        dims = (max(3, dims[0]),) + dims[1:]
    per = ()
    if len(dims) == 3 and gen.random() < 0.3:
        cand = [a for a in (1, 2) if a != f and dims[a] >= 3]
        per = tuple(cand[:1])
    p = float(gen.uniform(0.35, 0.8))
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, periodic=per), p, gen)
    return dims, planes, f, per


@pytest.mark.parametrize("seed", range(60))
def test_blocks_bruteforce_simple_paths(seed):
    dims, planes, f, per = _random_small(seed)
    on = ind.simple_path_nodes(dims, planes, f, per)
    want = np.zeros(int(np.prod(dims)), bool)
    want[sorted(on)] = True
    got = oracle.backbone_blocks(dims, planes, f, per).reshape(-1)
    np.testing.assert_array_equal(got, want)


def _nx_blocks(dims, planes, f, periodic, merged):
    nx = pytest.importorskip("networkx")
    adj = ind.contracted_graph(dims, planes, f, periodic)
    G = nx.Graph()
    for u, vs in adj.items():
        for v in vs:
            if merged:
                u2 = "S" if isinstance(u, str) else u
                v2 = "S" if isinstance(v, str) else v
                G.add_edge(u2, v2)
            else:
                G.add_edge(u, v)
    N = int(np.prod(dims))
    out = np.zeros(N, bool)
    if merged:
        _, cls = oracle.labels(dims, planes, f, periodic)
        span = cls.reshape(-1) == oracle.CLS_SPANNING
        if "S" not in G:
            return out
        for comp in nx.biconnected_components(G):
            if "S" in comp and len(comp) > 2:
                for v in comp:
                    if not isinstance(v, str) and span[v]:
                        out[v] = True
        return out
    G.add_edge("A", "B")
    for comp in nx.biconnected_component_edges(G):
        if ("A", "B") in comp or ("B", "A") in comp:
            for e in comp:
                for v in e:
                    if not isinstance(v, str):
                        out[v] = True
    return out


@pytest.mark.parametrize("merged", [False, True])
@pytest.mark.parametrize("dims,f,per,p,seed", [((30, 30), 0, (), 0.55, 1), ((25, 34), 1, (), 0.58, 2),
                                               ((12, 11, 10), 0, (), 0.33, 3), ((10, 12, 9), 2, (), 0.3, 4),
                                               ((14, 13, 12), 0, (1, 2), 0.3, 5),
                                               ((24, 20), 0, (1,), 0.56, 6)])
def test_blocks_equal_networkx(dims, f, per, p, seed, merged):
    gen = netgen.rng(7800 + seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, periodic=per), p, gen)
    got = oracle.backbone_blocks(dims, planes, f, per).reshape(-1)
    np.testing.assert_array_equal(got, _nx_blocks(dims, planes, f, per, merged))
    assert got.any()


def test_blocks_hand_made():
    """9 x 7 network, flow along x.  Row 3 and row 6 are open paths from the
    inlet to the outlet (two parallel paths: both carry current).  Hanging
    from row 3: a loop of four nodes on a one-bond stem (a dead-end loop,
    kept by dead-end tree stripping, removed here) and a three-node tree; a
    branch from (7,3) down to the outlet face (a second way into the outlet:
    it carries current).  Hanging from row 6: another dead-end loop on a
    one-bond stem."""
    dims = (9, 7)
    gx = np.zeros((7, 8))
    gy = np.zeros((6, 9))
    gx[3, :] = 1.0                      # row 3: path x = 0..8
    gx[6, :] = 1.5                      # row 6: parallel path
    gy[2, 4] = 2.0                      # stem (4,2)-(4,3)
    gx[2, 4] = gy[1, 5] = gx[1, 4] = gy[1, 4] = 2.0   # loop (4,2)-(5,2)-(5,1)-(4,1)-(4,2)
    gy[2, 2] = gy[1, 2] = gy[0, 2] = 3.0             # tree (2,3)-(2,2)-(2,1)-(2,0)
    gy[2, 7] = gx[2, 7] = 0.5           # (7,3)-(7,2)-(8,2): into the outlet face
    gy[5, 3] = 2.5                      # stem (3,5)-(3,6)
    gx[5, 3] = gy[4, 4] = gx[4, 3] = gy[4, 3] = 2.5  # loop (3,5)-(4,5)-(4,4)-(3,4)-(3,5)
    want = np.zeros((7, 9), bool)
    want[3, 1:8] = True
    want[6, 1:8] = True
    want[2, 7] = True
    got = oracle.backbone_blocks(dims, [gx, gy])
    np.testing.assert_array_equal(got, want)
    # dead-end tree stripping keeps both loops and drops only the tree
    trees = oracle.backbone(dims, [gx, gy])
    loops = np.zeros((7, 9), bool)
    loops[1:3, 4:6] = True
    loops[4:6, 3:5] = True
    np.testing.assert_array_equal(trees, want | loops)


@pytest.mark.parametrize("dims,p", [((26, 24), 0.56), ((14, 13, 12), 0.31)])
def test_blocks_within_tree_backbone(dims, p):
    gen = netgen.rng(7900 + len(dims))
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), p, gen)
    blocks = oracle.backbone_blocks(dims, planes)
    trees = oracle.backbone(dims, planes)
    assert not (blocks & ~trees).any()
    assert (trees & ~blocks).any()  # some dead-end loops at this disorder
    # a network with every bond open is all backbone
    full = netgen.lognormal_iid(dims, gen)
    _, cls = oracle.labels(dims, full)
    np.testing.assert_array_equal(oracle.backbone_blocks(dims, full), cls == oracle.CLS_SPANNING)


def test_blocks_removal_is_exact():
    """Closing every bond that touches a node outside the block backbone
    leaves G unchanged, and in the full solve no open bond touching such a
    node carries a pressure drop (no current enters a dead end)."""
    gen = netgen.rng(7950)
    dims = (22, 20, 18)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.34, gen)
    full = oracle.solve(dims, planes, tol=1e-14)
    bb = oracle.backbone_blocks(dims, planes)
    span = full.cls == oracle.CLS_SPANNING
    dead = span & ~bb
    assert dead.any() and bb.any()
    assert (dead & oracle.backbone(dims, planes)).any()  # dead-end loops among them
    cut = []
    for d in range(3):
        ax = 2 - d
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        g = planes[d].copy()
        g[dead[tuple(lo)] | dead[tuple(hi)]] = 0.0
        cut.append(g)
    red = oracle.solve(dims, cut, tol=1e-14)
    assert rel(red.g_eff, full.g_eff) < 1e-10
    for d in range(3):
        ax = 2 - d
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        touch = (planes[d] > 0) & (dead[tuple(lo)] | dead[tuple(hi)])
        drop = np.abs(full.P[tuple(lo)] - full.P[tuple(hi)])[touch]
        assert drop.max() < 1e-9
    # and every backbone bond between two backbone nodes is part of a path
    # that carries current: some drop somewhere on each backbone row
    assert np.ptp(full.P[bb]) > 0.5
