"""Pins for the FP64 CPU oracle: closed forms, hand-solved fixtures, a dense
direct solve, brute-force cluster labels and the invariants of Eq. 3 / Eq. 4.

None of these re-use the oracle's code path; each would fail on a plausible
slip inside it (a dropped face bond, a sign, a transposed plane index).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen
from tests import _independent as ind

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("dims,f", [((17, 9), 0), ((9, 17), 1), ((5, 6, 7), 0),
                                     ((5, 6, 7), 1), ((5, 6, 7), 2), ((3, 3), 0)])
def test_uniform_lattice_closed_form(dims, f):
    """Uniform g: P is linear along the flow axis and G = g S / R (Eq. 3, Eq. 4)."""
    g = 2.5
    r = oracle.solve(dims, netgen.uniform(dims, g), flow_axis=f, p_in=3.0, p_out=-1.0)
    R = dims[f] - 1
    S = int(np.prod(dims)) // dims[f]
    assert rel(r.g_eff, g * S / R) < 1e-12
    assert rel(r.k_eff, g) < 1e-12
    xs, ys, zs, _ = ind.node_coords(dims)
    c = [xs, ys, zs][f]
    want = 3.0 - 4.0 * c / R
    np.testing.assert_allclose(r.P.reshape(-1), want, rtol=0, atol=1e-12)


def test_stratified_along_layers_arithmetic_mean():
    """Flow along the layers: G_x = sum_y s_y / (nx - 1) (Wiener upper bound)."""
    gen = netgen.rng(11)
    dims = (23, 31)
    planes, s = netgen.stratified_layers(dims, gen, 1.0)
    r = oracle.solve(dims, planes, flow_axis=0)
    assert rel(r.g_eff, s.sum() / (dims[0] - 1)) < 1e-11


def test_stratified_across_layers_harmonic_mean():
    """Flow across the layers: G_y = nx / sum_j 1/t_j (Wiener lower bound)."""
    gen = netgen.rng(12)
    dims = (19, 29)
    planes, s = netgen.stratified_layers(dims, gen, 1.0)
    t = s[:-1]  # vertical bond between rows j and j+1 carries s_j
    r = oracle.solve(dims, planes, flow_axis=1)
    assert rel(r.g_eff, dims[0] / np.sum(1.0 / t)) < 1e-11


def test_stratified_3d_both_directions():
    """3D layers along z: arithmetic mean along x, harmonic across (z)."""
    gen = netgen.rng(13)
    dims = (7, 5, 9)
    s = np.exp(gen.standard_normal(dims[2]))
    planes = [np.broadcast_to(s[:, None, None], netgen.plane_shape(dims, 0)).copy(),
              np.broadcast_to(s[:, None, None], netgen.plane_shape(dims, 1)).copy(),
              np.broadcast_to(s[:-1, None, None], netgen.plane_shape(dims, 2)).copy()]
    rx = oracle.solve(dims, planes, flow_axis=0)
    assert rel(rx.g_eff, dims[1] * s.sum() / (dims[0] - 1)) < 1e-11
    rz = oracle.solve(dims, planes, flow_axis=2)
    assert rel(rz.g_eff, dims[0] * dims[1] / np.sum(1.0 / s[:-1])) < 1e-11


def test_series_chain():
    """A single row (ny = 1) is a chain of resistors: G = 1 / sum 1/g."""
    gen = netgen.rng(14)
    dims = (40, 1)
    gx = np.exp(gen.standard_normal((1, 39)))
    gy = np.zeros((0, 40))
    r = oracle.solve(dims, [gx, gy])
    assert rel(r.g_eff, 1.0 / np.sum(1.0 / gx)) < 1e-10


# ---------------------------------------------------------------- fixtures
@pytest.mark.parametrize("name", ["bridge_3x3.txt", "bridge_balanced_3x4.txt"])
def test_hand_solved_fixture(name):
    dims, planes, v = ind.read_golden(os.path.join(GOLD, name))
    r = oracle.solve(dims, planes, flow_axis=int(v["flow_axis"][0]))
    assert rel(r.g_eff, v["g_eff"][0]) < 1e-13
    assert rel(r.k_eff, v["k_eff"][0]) < 1e-13
    np.testing.assert_allclose(r.P, np.array(v["P"]), rtol=0, atol=1e-14)


# ---------------------------------------------------------------- dense solve
@pytest.mark.parametrize("dims,f,p", [((6, 5), 0, 1.0), ((5, 7), 1, 1.0), ((4, 3, 5), 2, 1.0),
                                       ((9, 8), 0, 0.6), ((5, 4, 4), 0, 0.55)])
def test_dense_direct_solve(dims, f, p):
    """CG result equals a dense LAPACK solve of the incidence-matrix form."""
    gen = netgen.rng(100 + len(dims) * 10 + f)
    planes = netgen.percolate(netgen.loguniform_iid(dims, gen), p, gen)
    r = oracle.solve(dims, planes, flow_axis=f, p_in=2.0, p_out=0.5)
    P, qin, qout = ind.dense_solve(dims, planes, f, 2.0, 0.5)
    np.testing.assert_allclose(r.P.reshape(-1), P, rtol=0, atol=1e-11)
    assert abs(r.q_in - qin) <= 1e-11 * max(1.0, abs(qin))
    assert abs(r.q_out - qout) <= 1e-11 * max(1.0, abs(qout))


# ---------------------------------------------------------------- labels
@pytest.mark.parametrize("dims,f,p,seed", [((7, 6), 0, 0.5, 1), ((6, 7), 1, 0.45, 2),
                                            ((5, 4, 6), 0, 0.3, 3), ((4, 5, 3), 2, 0.35, 4),
                                            ((10, 10), 0, 0.0, 5), ((10, 10), 0, 1.0, 6)])
def test_labels_bruteforce_bfs(dims, f, p, seed):
    gen = netgen.rng(seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), p, gen)
    lab, cls = oracle.labels(dims, planes, flow_axis=f)
    blab, bcls = ind.bfs_labels(dims, planes, f)
    np.testing.assert_array_equal(lab.reshape(-1), blab)
    np.testing.assert_array_equal(cls.reshape(-1), bcls)


def test_label_invariants_random():
    gen = netgen.rng(7)
    dims = (30, 20)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.5, gen)
    lab, cls = oracle.labels(dims, planes)
    lab = lab.reshape(-1)
    kind = ind.face_kind(dims, 0)
    for i, j, g in ind.bond_list(dims, planes):
        if kind[i] or kind[j]:
            continue
        if g > 0:
            assert lab[i] == lab[j]
    inner = np.where(kind == 0)[0]
    # label = smallest member
    for L in np.unique(lab[inner]):
        members = inner[lab[inner] == L]
        assert members.min() == L


# ---------------------------------------------------------------- invariants
def _rand_net(seed, dims=(24, 18), p=1.0):
    gen = netgen.rng(seed)
    planes = netgen.loguniform_iid(dims, gen)
    if p < 1.0:
        planes = netgen.percolate(planes, p, gen)
    return dims, planes


def test_conservation_and_tellegen():
    """Q_in = Q_out; zero imbalance; Q_in dP = sum_b g dP_b^2 (Tellegen)."""
    dims, planes = _rand_net(21, p=0.7)
    r = oracle.solve(dims, planes, p_in=1.0, p_out=0.0)
    assert r.g_eff > 0
    assert rel(r.q_out, r.q_in) < 1e-10
    assert rel(r.energy_g, r.g_eff) < 1e-10
    imb = oracle.residual(dims, planes, r.P)
    assert np.max(np.abs(imb)) < 1e-11 * max(1.0, np.max([np.max(g) for g in planes]))


def test_rayleigh_bounds():
    """Cutting transverse bonds lowers G, shorting them raises it."""
    dims, planes = _rand_net(22, dims=(20, 15))
    gx = planes[0]
    r = oracle.solve(dims, planes)
    g_lo = np.sum(1.0 / np.sum(1.0 / gx, axis=1))
    g_hi = 1.0 / np.sum(1.0 / np.sum(gx, axis=0))
    assert g_lo <= r.g_eff * (1 + 1e-12)
    assert r.g_eff <= g_hi * (1 + 1e-12)


def test_scaling_and_bc_affinity():
    dims, planes = _rand_net(23)
    r1 = oracle.solve(dims, planes)
    r2 = oracle.solve(dims, [3.7 * g for g in planes])
    assert rel(r2.g_eff, 3.7 * r1.g_eff) < 1e-11
    r3 = oracle.solve(dims, planes, p_in=5.0, p_out=3.0)  # P' = 2 P + 3
    assert rel(r3.g_eff, r1.g_eff) < 1e-11
    act = r1.cls == oracle.CLS_SPANNING
    np.testing.assert_allclose(r3.P[act], 2.0 * r1.P[act] + 3.0, atol=1e-10)


def test_mirror_and_transpose_symmetry():
    dims, planes = _rand_net(24, dims=(14, 11), p=0.8)
    r = oracle.solve(dims, planes)
    # mirror along x, faces swap roles: same conductance
    gm = [planes[0][:, ::-1].copy(), planes[1][:, ::-1].copy()]
    rm = oracle.solve(dims, gm)
    assert rel(rm.g_eff, r.g_eff) < 1e-10
    # transpose: x <-> y with flow along y
    gt = [planes[1].T.copy(), planes[0].T.copy()]
    rt = oracle.solve((dims[1], dims[0]), gt, flow_axis=1)
    assert rel(rt.g_eff, r.g_eff) < 1e-10


def test_percolation_no_spanning_cluster():
    """No open path between the faces: G = 0 exactly."""
    dims = (12, 9)
    gen = netgen.rng(25)
    planes = netgen.lognormal_iid(dims, gen)
    planes[0][:, 5] = 0.0  # cut every x-bond of column 5 -> 6
    r = oracle.solve(dims, planes)
    assert r.g_eff == 0.0 and r.n_active == 0
    assert r.q_in == 0.0 and r.q_out == 0.0


def test_stripping_dead_ends_keeps_g():
    """Dangling / one-sided clusters carry no current: removing them (zeroing
    their bonds) does not change G."""
    dims, planes = _rand_net(26, dims=(16, 16), p=0.6)
    r = oracle.solve(dims, planes)
    keep = (r.cls == oracle.CLS_SPANNING) | (r.cls >= oracle.CLS_FACE_IN)
    kflat = keep.reshape(-1)
    pruned = [g.copy() for g in planes]
    for d in range(2):
        m = list(dims)
        m[d] -= 1
        for y in range(m[1]):
            for x in range(m[0]):
                i = x + dims[0] * y
                j = i + (1 if d == 0 else dims[0])
                if not (kflat[i] and kflat[j]):
                    pruned[d][y, x] = 0.0
    rp = oracle.solve(dims, pruned)
    assert rel(rp.g_eff, r.g_eff) < 1e-10


def test_duality_geometric_mean_loose():
    """2D log-symmetric i.i.d. conductances: G R / S near the geometric mean
    (Keller-Dykhne duality); statistical, 10 % band."""
    gen = netgen.rng(27)
    dims = (96, 96)
    planes = netgen.lognormal_iid(dims, gen, 1.0)
    r = oracle.solve(dims, planes, tol=1e-10)
    assert 0.9 < r.k_eff < 1.1


def test_invalid_inputs_rejected():
    dims = (8, 8)
    planes = netgen.uniform(dims)
    bad = [planes[0].copy(), planes[1].copy()]
    bad[0][2, 3] = -1.0
    with pytest.raises(ValueError):
        oracle.solve(dims, bad)
    bad[0][2, 3] = np.nan
    with pytest.raises(ValueError):
        oracle.solve(dims, bad)
    with pytest.raises(ValueError):
        oracle.solve((2, 8), netgen.uniform((2, 8)))


# ---------------------------------------------------------------- backbone (dead-end stripping)
def _nx_backbone(dims, planes, flow_axis=0, periodic=()):
    """Backbone by networkx's k-core: the graph of open bonds among the
    spanning nodes and the face nodes (face-face bonds left out), every face
    node tied to a triangle so that it never drops below degree 2 while it
    keeps one interior link.  The 2-core's interior nodes are the backbone."""
    nx = pytest.importorskip("networkx")
    lab, cls = oracle.labels(dims, planes, flow_axis, periodic)
    cls = cls.reshape(-1)
    N = int(np.prod(dims))
    ndim = len(dims)
    ext = list(dims) + [1] * (3 - ndim)
    face = (cls == oracle.CLS_FACE_IN) | (cls == oracle.CLS_FACE_OUT)
    keep = (cls == oracle.CLS_SPANNING) | face
    G = nx.Graph()
    G.add_nodes_from(np.where(keep)[0].tolist())
    for d in range(ndim):
        g = planes[d].reshape(-1)
        n = list(ext)
        if d not in periodic:
            n[d] -= 1
        idx = np.arange(int(np.prod(n)))
        c = [idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])]
        i = c[0] + ext[0] * (c[1] + ext[1] * c[2])
        c[d] = (c[d] + 1) % ext[d]
        j = c[0] + ext[0] * (c[1] + ext[1] * c[2])
        ok = (g > 0) & keep[i] & keep[j] & ~(face[i] & face[j])
        G.add_edges_from(zip(i[ok].tolist(), j[ok].tolist()))
    G.add_edges_from([("S", "A"), ("A", "B"), ("B", "S")])
    G.add_edges_from(("S", int(f)) for f in np.where(face)[0])
    core = nx.k_core(G, 2)
    out = np.zeros(N, bool)
    for v in core.nodes:
        if not isinstance(v, str) and cls[v] == oracle.CLS_SPANNING:
            out[v] = True
    return out


@pytest.mark.parametrize("dims,f,p,seed", [((14, 11), 0, 0.62, 1), ((12, 15), 1, 0.58, 2),
                                           ((9, 8, 7), 0, 0.36, 3), ((8, 9, 10), 2, 0.33, 4),
                                           ((30, 30), 0, 0.55, 5), ((16, 16, 16), 1, 0.3, 6)])
def test_backbone_equals_kcore(dims, f, p, seed):
    gen = netgen.rng(9100 + seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), p, gen)
    bb = oracle.backbone(dims, planes, f).reshape(-1)
    np.testing.assert_array_equal(bb, _nx_backbone(dims, planes, f))


def test_backbone_hand_made_tree_on_a_path():
    """A single open path along row 2 of a 7x5 network plus a branch of three
    bonds hanging from it (a dead end) and a loop of four bonds beside it: the
    backbone is the path and the loop, the branch is stripped."""
    dims = (7, 5)
    gx = np.zeros((5, 6))
    gy = np.zeros((4, 7))
    gx[2, :] = 1.0           # the path x = 0..6 on row 2
    gy[2, 3] = 2.0           # branch (3,2)-(3,3)
    gx[3, 3] = 2.0           # (3,3)-(4,3)
    gy[3, 4] = 2.0           # (4,3)-(4,4)
    gy[0, 2] = gy[1, 2] = 3.0  # loop (2,0)-(2,1)-(2,2) ...
    gx[0, 2] = 3.0             # ... (2,0)-(3,0)
    gy[0, 3] = gy[1, 3] = 3.0  # (3,0)-(3,1)-(3,2)
    bb = oracle.backbone(dims, [gx, gy])
    want = np.zeros((5, 7), bool)
    want[2, 1:6] = True
    want[0, 2] = want[1, 2] = want[0, 3] = want[1, 3] = True
    np.testing.assert_array_equal(bb, want)


def test_backbone_stripping_is_exact():
    """Closing every bond that touches a stripped node leaves G unchanged, and
    each stripped node's pressure equals that of a backbone or face neighbour
    reached through stripped nodes only (no current flows into a dead end)."""
    gen = netgen.rng(9200)
    dims = (22, 20, 18)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.34, gen)
    full = oracle.solve(dims, planes, tol=1e-14)
    bb = oracle.backbone(dims, planes)
    span = full.cls == oracle.CLS_SPANNING
    dead = span & ~bb
    assert dead.any() and bb.any()
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
    # across every open bond that touches a stripped node there is no drop
    for d in range(3):
        ax = 2 - d
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        touch = (planes[d] > 0) & (dead[tuple(lo)] | dead[tuple(hi)])
        drop = np.abs(full.P[tuple(lo)] - full.P[tuple(hi)])[touch]
        assert drop.max() < 1e-9


# ---------------------------------------------------------------- periodic transverse boundaries
# Sec. II allows the transverse faces to be periodic: the last layer of bonds
# along a periodic axis joins the last node layer to the first.
def _periodic_net(dims, periodic, p, seed):
    gen = netgen.rng(9300 + seed)
    planes = netgen.lognormal_iid(dims, gen, periodic=periodic)
    return netgen.percolate(planes, p, gen)


@pytest.mark.parametrize("dims,f,per", [((9, 7), 0, (1,)), ((7, 9), 1, (0,)),
                                         ((5, 6, 7), 0, (1, 2)), ((5, 6, 7), 2, (0, 1)),
                                         ((6, 3, 4), 0, (1,))])
def test_periodic_uniform_closed_form(dims, f, per):
    """Uniform g with periodic transverse axes: the wrap bonds join nodes at
    the same pressure, so P stays linear and G = g S / R as without them."""
    g = 1.5
    r = oracle.solve(dims, netgen.uniform(dims, g, periodic=per), flow_axis=f,
                     p_in=2.0, p_out=-2.0, periodic=per)
    R = dims[f] - 1
    S = int(np.prod(dims)) // dims[f]
    assert rel(r.g_eff, g * S / R) < 1e-12
    xs, ys, zs, _ = ind.node_coords(dims)
    c = [xs, ys, zs][f]
    np.testing.assert_allclose(r.P.reshape(-1), 2.0 - 4.0 * c / R, rtol=0, atol=1e-12)


def test_periodic_wrap_only_path():
    """A 3x4 network whose only inlet-outlet path runs through a wrap bond:
    inlet (0,0) -a- (1,0) -w- (1,3) -b- (2,3) outlet, the middle bond being
    the one from row 3 back to row 0.  G is the series value 1/(1/a+1/w+1/b);
    without periodic boundaries nothing spans."""
    dims = (3, 4)
    a, w, b = 2.0, 0.5, 4.0
    gx = np.zeros((4, 2))
    gy = np.zeros((4, 3))
    gx[0, 0] = a
    gx[3, 1] = b
    gy[3, 1] = w
    r = oracle.solve(dims, [gx, gy], p_in=1.0, p_out=0.0, periodic=(1,))
    want = 1.0 / (1.0 / a + 1.0 / w + 1.0 / b)
    assert rel(r.g_eff, want) < 1e-13
    # the two interior pressures of the series chain
    assert abs(r.P[0, 1] - (1.0 - want / a)) < 1e-13
    assert abs(r.P[3, 1] - want / b) < 1e-13
    closed = oracle.solve(dims, [gx, gy[:3]], p_in=1.0, p_out=0.0)
    assert closed.g_eff == 0.0


@pytest.mark.parametrize("dims,f,per,p", [((6, 5), 0, (1,), 1.0), ((5, 7), 1, (0,), 0.7),
                                           ((4, 3, 5), 0, (1, 2), 1.0), ((4, 3, 5), 2, (0,), 0.6),
                                           ((9, 8), 0, (1,), 0.55), ((5, 4, 4), 1, (0, 2), 0.5)])
def test_periodic_dense_direct_solve(dims, f, per, p):
    """CG with wrap bonds equals a dense solve of the incidence-matrix form
    built from the bond list with the wrap bonds in it."""
    planes = _periodic_net(dims, per, p, len(dims) * 10 + f)
    r = oracle.solve(dims, planes, flow_axis=f, p_in=2.0, p_out=0.5, periodic=per)
    P, qin, qout = ind.dense_solve(dims, planes, f, 2.0, 0.5, periodic=per)
    np.testing.assert_allclose(r.P.reshape(-1), P, rtol=0, atol=1e-11)
    assert abs(r.q_in - qin) <= 1e-11 * max(1.0, abs(qin))
    assert abs(r.q_out - qout) <= 1e-11 * max(1.0, abs(qout))


@pytest.mark.parametrize("dims,f,per,p,seed", [((7, 6), 0, (1,), 0.5, 1), ((6, 7), 1, (0,), 0.45, 2),
                                                ((5, 4, 6), 0, (1, 2), 0.3, 3),
                                                ((4, 5, 3), 2, (0, 1), 0.35, 4)])
def test_periodic_labels_bruteforce_bfs(dims, f, per, p, seed):
    planes = _periodic_net(dims, per, p, 20 + seed)
    lab, cls = oracle.labels(dims, planes, flow_axis=f, periodic=per)
    blab, bcls = ind.bfs_labels(dims, planes, f, periodic=per)
    np.testing.assert_array_equal(lab.reshape(-1), blab)
    np.testing.assert_array_equal(cls.reshape(-1), bcls)


@pytest.mark.parametrize("dims,f,per,shift", [((12, 10), 0, (1,), (0, 3)),
                                               ((8, 7, 6), 2, (0, 1), (5, 2, 0)),
                                               ((7, 9, 5), 0, (1, 2), (0, 4, 2))])
def test_periodic_cyclic_shift_invariance(dims, f, per, shift):
    """Rolling a periodic network along its periodic axes (nodes and bonds
    alike) rolls P the same way and leaves G unchanged; without the wrap
    bonds this fails, so it checks that they join the right nodes."""
    planes = _periodic_net(dims, per, 0.8, 40 + f)
    axes = tuple(len(dims) - 1 - d for d in range(len(dims)))
    sh = tuple(shift[d] for d in range(len(dims)))
    rolled = [np.roll(g, sh, axis=axes) for g in planes]
    r0 = oracle.solve(dims, planes, flow_axis=f, periodic=per, tol=1e-14)
    r1 = oracle.solve(dims, rolled, flow_axis=f, periodic=per, tol=1e-14)
    assert rel(r1.g_eff, r0.g_eff) < 1e-11
    np.testing.assert_allclose(r1.P, np.roll(r0.P, sh, axis=axes), rtol=0, atol=1e-11)


@pytest.mark.parametrize("dims,f,per,p,seed", [((14, 11), 0, (1,), 0.6, 1),
                                                ((9, 8, 7), 0, (1, 2), 0.34, 2),
                                                ((8, 9, 10), 2, (0, 1), 0.33, 3)])
def test_periodic_backbone_equals_kcore(dims, f, per, p, seed):
    planes = _periodic_net(dims, per, p, 60 + seed)
    bb = oracle.backbone(dims, planes, f, periodic=per).reshape(-1)
    np.testing.assert_array_equal(bb, _nx_backbone(dims, planes, f, periodic=per))


def test_periodic_invalid_inputs_rejected():
    dims = (8, 6)
    with pytest.raises(ValueError):     # the flow axis cannot be periodic
        oracle.solve(dims, netgen.uniform(dims, periodic=(0,)), periodic=(0,))
    with pytest.raises(ValueError):     # plane with the non-periodic shape
        oracle.solve(dims, netgen.uniform(dims), periodic=(1,))
    with pytest.raises(ValueError):     # a periodic axis needs three layers
        oracle.solve((8, 2), netgen.uniform((8, 2), periodic=(1,)), periodic=(1,))
    with pytest.raises(ValueError):     # axis beyond ndim
        oracle.solve(dims, netgen.uniform(dims), periodic=(2,))


# ---------------------------------------------------------------- sorted removal (Sec. VI.B)
def _brute_close(planes, q):
    """Tiny-input brute force: rank every bond by (value, plane, index) with
    Python's sort and close the first floor(q M)."""
    items = []
    for d, g in enumerate(planes):
        for i, v in enumerate(np.asarray(g, dtype=np.float64).reshape(-1).tolist()):
            items.append((v, d, i))
    k = int(np.floor(q * len(items)))
    shut = {(d, i) for _, d, i in sorted(items)[:k]}
    out = []
    for d, g in enumerate(planes):
        f = np.asarray(g).reshape(-1).copy()
        for i in range(f.size):
            if (d, i) in shut:
                f[i] = 0
        out.append(f.reshape(np.shape(g)))
    return out


@pytest.mark.parametrize("dims,q,levels,seed", [((5, 4), 0.5, 0, 1), ((6, 5, 4), 0.3, 3, 2),
                                                 ((7, 3), 1.0, 2, 3), ((4, 4, 4), 0.0, 0, 4),
                                                 ((9, 8), 0.77, 4, 5)])
def test_close_smallest_bruteforce(dims, q, levels, seed):
    """Equal values (few levels) and zeros test the position order of ties."""
    gen = netgen.rng(9400 + seed)
    planes = netgen.lognormal_iid(dims, gen)
    if levels:
        planes = [np.floor(g * levels) / levels for g in planes]
    got = oracle.close_smallest(planes, q)
    want = _brute_close(planes, q)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


def test_close_smallest_invariants():
    gen = netgen.rng(9450)
    dims = (30, 20, 10)
    planes = [g.astype(np.float32) for g in netgen.lognormal_iid(dims, gen)]
    M = sum(g.size for g in planes)
    for q in (0.1, 0.5, 0.9):
        out = oracle.close_smallest(planes, q)
        closed = np.concatenate([(o == 0).reshape(-1) for o in out])
        vals = np.concatenate([g.reshape(-1) for g in planes])
        assert closed.sum() == int(np.floor(q * M))   # all values positive
        assert vals[closed].max() <= vals[~closed].min()
        assert all(o.dtype == np.float32 for o in out)
    with pytest.raises(ValueError):
        oracle.close_smallest(planes, 1.5)


# ---------------------------------------------------------------- FBM generator (Eq. 1, Eq. 2)
def _modes(shape, modes):
    noise = np.zeros(shape, complex)
    for idx in modes:
        noise[idx] = 1.0
    return noise


def test_fbm_single_mode_is_a_cosine():
    """One Fourier mode: the normalised field is sqrt(2) cos(2 pi k.x / n)
    (frequency convention, real part and normalisation; the weight cancels)."""
    ny, nx = 16, 24
    f = oracle.fbm_field(_modes((ny, nx), [(5, 20)]), 0.7)
    y, x = np.mgrid[0:ny, 0:nx]
    want = np.sqrt(2.0) * np.cos(2 * np.pi * (5 * y / ny + 20 * x / nx))
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,H,beta,modes", [
    ((16, 24), 0.7, (2.0, 0.5), [(0, 3), (2, 0), (5, 20)]),
    ((12, 10, 14), 0.3, (1.0, 3.0, 0.25), [(0, 0, 2), (0, 3, 0), (4, 0, 0), (11, 7, 12)])])
def test_fbm_mode_weights_follow_the_spectral_density(shape, H, beta, modes):
    """Several modes with unit noise: each mode's cosine coefficient is
    proportional to S(w)^(1/2) = (sum_a beta_a w_a^2)^-(H/2 + d/4): the ratio
    of coefficients pins the exponent, the betas and the axis order."""
    d = len(shape)
    f = oracle.fbm_field(_modes(shape, modes), H, beta)
    grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    coef, amp = [], []
    for idx in modes:
        phase = sum(2 * np.pi * idx[ax] * grids[ax] / shape[ax] for ax in range(d))
        coef.append(2.0 * np.mean(f * np.cos(phase)))
        k2 = 0.0
        for ax in range(d):
            w = idx[ax] / shape[ax]
            w = w - 1.0 if w > 0.5 else w
            k2 += beta[d - 1 - ax] * w * w
        amp.append(k2 ** (-(2 * H + d) / 4))
    for i in range(1, len(modes)):
        assert abs(coef[i] / coef[0] - amp[i] / amp[0]) <= 1e-10 * amp[i] / amp[0]


def test_fbm_spectrum_slope_eq1():
    """Isotropic 2D field from white noise: the radially averaged power
    spectrum falls as |w|^-(2H+2) (Eq. 1)."""
    gen = netgen.rng(9500)
    n, H = 512, 0.7
    noise = gen.standard_normal((n, n)) + 1j * gen.standard_normal((n, n))
    f = oracle.fbm_field(noise, H)
    P = np.abs(np.fft.fft2(f)) ** 2
    w = np.sqrt(np.add.outer(np.fft.fftfreq(n) ** 2, np.fft.fftfreq(n) ** 2))
    bins = np.geomspace(4.0 / n, 0.4, 12)
    lw, lp = [], []
    for a, b in zip(bins[:-1], bins[1:]):
        m = (w >= a) & (w < b)
        lw.append(np.log(w[m].mean()))
        lp.append(np.log(P[m].mean()))
    slope = np.polyfit(lw, lp, 1)[0]
    assert abs(slope + (2 * H + 2)) < 0.1


def test_fbm_anisotropy_layers_parallel_to_x():
    """beta_x / beta_y > 1 damps modes that vary along x: the field is
    smoother along x than along y (layers parallel to x, Eq. 2)."""
    gen = netgen.rng(9501)
    noise = gen.standard_normal((256, 256)) + 1j * gen.standard_normal((256, 256))
    f = oracle.fbm_field(noise, 0.5, beta=(5.0, 1.0))
    dx = np.mean(np.diff(f, axis=1) ** 2)
    dy = np.mean(np.diff(f, axis=0) ** 2)
    assert dx < 0.5 * dy
    g = oracle.fbm_field(noise, 0.5, beta=(1.0, 1.0))
    np.testing.assert_allclose(g, oracle.fbm_field(noise, 0.5), rtol=0, atol=1e-13)
    assert abs(f.mean()) < 1e-12 and abs(np.mean(f * f) - 1.0) < 1e-12


def test_fbm_bonds_hand_values():
    B = np.array([[0.0, 1.0, -1.0], [2.0, 0.5, 0.0]])  # (ny, nx) = (2, 3)
    gx, gy = oracle.fbm_bonds(B, 2.0)
    np.testing.assert_allclose(gx, np.exp(2.0 * np.array([[0.5, 0.0], [1.25, 0.25]])), rtol=1e-15)
    np.testing.assert_allclose(gy, np.exp(2.0 * np.array([[1.0, 0.75, -0.5]])), rtol=1e-15)
