"""The compacted inner solve (unknowns listed in lattice order, ELL rows, one
cooperative launch per inner solve): every combination of dimension, inner
precision and refinement scheme must give the oracle's G_eff and pressures,
and the same answer as the lattice kernels."""
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


CASES = [((45, 38), 0, 0.56, 1), ((33, 52), 1, 0.6, 2), ((26, 21, 19), 0, 0.33, 3),
         ((20, 24, 27), 2, 0.32, 4), ((70, 66, 64), 1, 0.27, 5), ((17, 15, 16), 0, 1.0, 6)]


@pytest.mark.parametrize("dims,f,p,seed", CASES)
@pytest.mark.parametrize("precision,refine", [(0, 0), (1, 0), (0, 1)])
def test_compact_matches_oracle(ns, monkeypatch, dims, f, p, seed, precision, refine):
    monkeypatch.setenv("NETSOLVE_KERNEL", "compact")
    gen = netgen.rng(9800 + seed)
    planes = netgen.lognormal_iid(dims, gen)
    if p < 1.0:
        planes = netgen.percolate(planes, p, gen)
    ref = oracle.solve(dims, planes, flow_axis=f, tol=1e-13)
    with ns.Network(dims, planes, flow_axis=f) as net:
        r = net.solve(ns.make_opts(precision=precision, refine=refine))
        P = net.pressure()
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
        return
    assert r.status == ns.NET_OK, r
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7


def test_compact_is_chosen_for_sparse_networks_and_agrees_with_sweep(ns, monkeypatch):
    """A near-critical 3D network (few unknowns after stripping) takes the
    compacted solve by default; forcing the lattice sweep gives the same G."""
    gen = netgen.rng(9900)
    dims = (60, 58, 56)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.27, gen)
    with ns.Network(dims, planes) as net:
        a = net.solve()
    assert a.n_solved * 100 < 35 * np.prod(dims)
    assert a.inner_launches <= 2 * a.outer_iters + 2  # one launch per inner solve
    monkeypatch.setenv("NETSOLVE_KERNEL", "sweep")
    with ns.Network(dims, planes) as net:
        b = net.solve()
    assert b.inner_launches > 10 * a.inner_launches
    assert rel(a.g_eff, b.g_eff) <= G_TOL


def test_compact_repeat_is_bit_identical(ns, monkeypatch):
    monkeypatch.setenv("NETSOLVE_KERNEL", "compact")
    gen = netgen.rng(9901)
    dims = (40, 40, 40)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.3, gen)
    with ns.Network(dims, planes) as net:
        a = net.solve()
        b = net.solve()
    assert a.g_eff == b.g_eff and a.inner_iters == b.inner_iters


@pytest.mark.parametrize("dims,planes_fn", [
    ((3, 1), lambda d: netgen.uniform(d, 2.0)),                       # one unknown
    ((4, 1), lambda d: netgen.uniform(d, 1.0)),                       # a chain of two
    ((5, 4), lambda d: netgen.lognormal_iid(d, netgen.rng(1))),
    ((3, 3, 3), lambda d: netgen.lognormal_iid(d, netgen.rng(2))),
    ((9, 7), lambda d: netgen.percolate(netgen.lognormal_iid(d, netgen.rng(3)), 0.6, netgen.rng(4))),
])
def test_compact_tiny_networks(ns, monkeypatch, dims, planes_fn):
    """Far fewer unknowns than threads in the cooperative grid (down to one)."""
    monkeypatch.setenv("NETSOLVE_KERNEL", "compact")
    planes = planes_fn(dims)
    ref = oracle.solve(dims, planes, tol=1e-13)
    for precision in (0, 1):
        with ns.Network(dims, planes) as net:
            r = net.solve(ns.make_opts(precision=precision))
            P = net.pressure()
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0
            continue
        assert r.status == ns.NET_OK, r
        assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert np.max(np.abs(P - ref.P)) <= 1e-7


def test_compact_capped_solve_resumes(ns, monkeypatch):
    """A solve stopped by max_outer leaves consistent pressures; the next
    solve, started from them, converges to the oracle."""
    monkeypatch.setenv("NETSOLVE_KERNEL", "compact")
    gen = netgen.rng(9910)
    dims = (30, 28, 26)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen), 0.33, gen)
    ref = oracle.solve(dims, planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        a = net.solve(ns.make_opts(max_outer=1), check=False)
        P1 = net.pressure()
        b = net.solve(x0=P1)
    assert a.outer_iters == 1
    assert b.status == ns.NET_OK and rel(b.g_eff, ref.g_eff) <= G_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_compact_beyond_shared_table_matches_persistent(ns, monkeypatch, precision):
    """A list longer than the table rows each CTA keeps in shared memory (a
    1400 x 1200 network: 1.68 M unknowns, eleven 1024-row chunks per CTA of
    which ten fit in FP32 and four in FP64): the later chunks read their rows
    from global memory.  G_eff and pressures equal those of the FP64 solve on
    the lattice (the sweep kernel, itself pinned against the oracle)."""
    dims = (1400, 1200)
    gen = netgen.rng(9911)
    planes = netgen.lognormal_iid(dims, gen)
    with ns.Network(dims, planes) as net:
        r_ref = net.solve(ns.make_opts(precision=ns.NET_FP64))
        P_ref = net.pressure()
    monkeypatch.setenv("NETSOLVE_KERNEL", "compact")
    with ns.Network(dims, planes) as net:
        r = net.solve(ns.make_opts(precision=precision))
        P = net.pressure()
    assert r.status == ns.NET_OK and r_ref.status == ns.NET_OK
    assert rel(r.g_eff, r_ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - P_ref)) <= 1e-7
    assert rel(r.energy_g, r.g_eff) <= 1e-8
