"""Periodic transverse boundaries (Sec. II: a pressure drop along one axis,
periodic boundaries on the others).  The wrap bonds live in the last layer of
each periodic bond plane; the set-up kernels, the FP64 residual pass and the
compacted solve's neighbour table follow them.  Labels and backbone must be
the oracle's bit for bit, G_eff and P within the solver's tolerance."""
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


def periodic_net(dims, per, p, seed, sigma=1.0):
    gen = netgen.rng(9700 + seed)
    planes = netgen.lognormal_iid(dims, gen, sigma=sigma, periodic=per)
    return netgen.percolate(planes, p, gen) if p < 1.0 else planes


CASES = [((64, 50), 0, (1,), 0.58, 1), ((41, 37), 0, (1,), 1.0, 2),
         ((40, 36, 30), 0, (1, 2), 0.34, 3), ((28, 33, 36), 2, (1,), 0.3, 4),
         ((36, 31, 29), 1, (2,), 0.6, 5), ((96, 80), 0, (1,), 0.52, 6)]


@pytest.mark.parametrize("dims,f,per,p,seed", CASES)
@pytest.mark.parametrize("precision,refine,kernel", [(0, 0, ""), (1, 0, ""), (0, 1, ""),
                                                     (0, 0, "compact"), (0, 1, "compact")])
def test_periodic_matches_oracle(ns, monkeypatch, dims, f, per, p, seed, precision, refine, kernel):
    """Dense 2D periodic networks take the persistent kernel (wrap rows in its
    halo exchange) unless the compacted solve is forced; 3D ones, FP64 and
    sparse ones take the compacted solve."""
    if kernel:
        monkeypatch.setenv("NETSOLVE_KERNEL", kernel)
    planes = periodic_net(dims, per, p, seed)
    ref = oracle.solve(dims, planes, flow_axis=f, tol=1e-13, periodic=per)
    lab_o, cls_o = oracle.labels(dims, planes, flow_axis=f, periodic=per)
    bb_o = oracle.backbone_blocks(dims, planes, f, periodic=per)
    with ns.Network(dims, planes, flow_axis=f, periodic=per) as net:
        r = net.solve(ns.make_opts(precision=precision, refine=refine))
        P = net.pressure()
        lab, cls = net.labels()
        bb = net.backbone()
    np.testing.assert_array_equal(lab, lab_o)
    np.testing.assert_array_equal(cls, cls_o)
    np.testing.assert_array_equal(bb, bb_o)
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
        return
    assert r.status == ns.NET_OK, r
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7


def test_periodic_differs_from_no_flow(ns):
    """The same bulk conductances with and without the wrap bonds: both
    solves agree with their own oracle, and the wrap bonds change G."""
    dims, per = (48, 40), (1,)
    planes = periodic_net(dims, per, 0.55, 20)
    closed = [planes[0], planes[1][:-1]]
    with ns.Network(dims, planes, periodic=per) as a, ns.Network(dims, closed) as b:
        ra, rb = a.solve(), b.solve()
    oa = oracle.solve(dims, planes, periodic=per, tol=1e-13)
    ob = oracle.solve(dims, closed, tol=1e-13)
    assert rel(ra.g_eff, oa.g_eff) <= G_TOL and rel(rb.g_eff, ob.g_eff) <= G_TOL
    assert rel(oa.g_eff, ob.g_eff) > 1e-4


@pytest.mark.parametrize("dims,per", [((33, 17), (1,)), ((12, 9, 7), (1, 2))])
def test_periodic_uniform_closed_form(ns, dims, per):
    g = 0.75
    with ns.Network(dims, netgen.uniform(dims, g, periodic=per), p_in=2.0, p_out=-1.0,
                    periodic=per) as net:
        r = net.solve()
        P = net.pressure()
    R = dims[0] - 1
    S = int(np.prod(dims)) // dims[0]
    assert rel(r.g_eff, g * S / R) <= 1e-10
    xs = np.arange(dims[0])
    np.testing.assert_allclose(P, np.broadcast_to(2.0 - 3.0 * xs / R, P.shape), rtol=0, atol=1e-9)


def test_periodic_wrap_only_path(ns):
    """The only inlet-outlet path runs through one wrap bond: G is the
    series value of its three bonds."""
    dims = (3, 4)
    a, w, b = 2.0, 0.5, 4.0
    gx = np.zeros((4, 2))
    gy = np.zeros((4, 3))
    gx[0, 0], gx[3, 1], gy[3, 1] = a, b, w
    with ns.Network(dims, [gx, gy], periodic=(1,)) as net:
        r = net.solve()
    assert rel(r.g_eff, 1.0 / (1.0 / a + 1.0 / w + 1.0 / b)) <= 1e-10


def test_periodic_networks_in_batch_and_queue(ns):
    """Periodic members (solved on their list of unknowns, whose table holds
    the wrap bonds) beside no-flow ones in one batch and in the queue, 2D and
    3D, dense and percolated: every result against the periodic oracle."""
    specs = [((48, 40), 0, (1,), 1.0, 40), ((64, 50), 0, (1,), 0.58, 41), ((30, 28, 26), 0, (1, 2), 0.34, 42),
             ((26, 24, 22), 2, (1,), 0.5, 43), ((40, 36), 1, (), 0.6, 44), ((20, 21, 19), 0, (), 0.4, 45)]
    nets, refs, inputs = [], [], []
    for dims, f, per, p, seed in specs:
        planes = periodic_net(dims, per, p, seed)
        inputs.append((dims, planes, f, per))
        refs.append(oracle.solve(dims, planes, flow_axis=f, tol=1e-13, periodic=per))
        nets.append(ns.Network(dims, planes, flow_axis=f, periodic=per))
    res = ns.solve_batch(nets)
    for net, r, ref in zip(nets, res, refs):
        P = net.pressure()
        assert r.status == ns.NET_OK, r
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
        else:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert np.max(np.abs(P - ref.P)) <= 1e-7
    for net in nets:
        net.close()
    with ns.Queue(mem_budget_bytes=1 << 30, max_slots=4) as q:
        tickets = [q.submit(d, pl, flow_axis=f, periodic=per) for d, pl, f, per in inputs]
        qres = [q.wait(t, timeout_ms=120000) for t in tickets]
    for (st, r), ref in zip(qres, refs):
        assert st == ns.NET_OK, (st, r)
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
        else:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL


def test_periodic_rejected_by_autotune(ns):
    dims, per = (16, 12), (1,)
    planes = periodic_net(dims, per, 1.0, 30)
    with ns.Network(dims, planes, periodic=per) as net:
        with pytest.raises(ns.NetError) as e:
            ns.autotune([net])
        assert e.value.status == ns.NET_EINVAL


def test_periodic_fbm_network_matches_oracle(ns):
    """A correlated (FBM, H = 0.7, sigma = 1.5) 192^2 network with periodic y,
    the headline workload's medium at a size the oracle solves in seconds."""
    from paper_1908_03301_gb300 import netgen as ng

    dims, planes = ng.workload_fbm2d(n=192, seed=4242, periodic=(1,))
    ref = oracle.solve(dims, planes, tol=1e-13, periodic=(1,))
    with ns.Network(dims, planes, periodic=(1,)) as net:
        r = net.solve()
        P = net.pressure()
    assert r.status == ns.NET_OK, r
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7
