"""The sweep kernel's tile-shape autotuner (net_autotune) and every shape it
may pick: each must give the oracle's effective conductance within the
accuracy target, and solves after tuning stay bit-for-bit repeatable."""
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


def net3d(seed=11, dims=(37, 29, 23), p=0.7):
    gen = netgen.rng(8000 + seed)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, 1.0), p, gen)
    return dims, planes


def test_autotune_picks_a_shape_and_solves_repeat_exactly(ns):
    ns.tune_clear()
    dims, planes = net3d()
    ref = oracle.solve(dims, planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        t = ns.autotune([net])
        assert t["candidates"] >= 4
        assert 0 < t["us_per_sweep"] <= t["us_default"]
        assert t["col_block"] % 4 == 0 and 1 <= t["row_band"] <= 32
        assert t["col_block"] * t["row_band"] <= 1024
        r1 = net.solve()
        r2 = net.solve()
    assert r1.status == ns.NET_OK
    assert r1.g_eff == r2.g_eff and r1.inner_iters == r2.inner_iters
    assert rel(r1.g_eff, ref.g_eff) <= G_TOL


def test_autotune_rejects_bad_sets(ns):
    a = ns.Network((12, 10), netgen.uniform((12, 10)))
    b = ns.Network((6, 5, 4), netgen.uniform((6, 5, 4)))
    with pytest.raises(ns.NetError) as ei:
        ns.autotune([a, b])
    assert ei.value.status == ns.NET_EINVAL
    a.close()
    b.close()


@pytest.mark.parametrize("shape", ["256,4,1", "128,8,2", "64,16,4", "32,32,1", "16,0,3", "0,0,2"])
@pytest.mark.parametrize("precision", [0, 1])
def test_every_3d_shape_matches_oracle(ns, monkeypatch, shape, precision):
    monkeypatch.setenv("NETSOLVE_SWEEP_SHAPE", shape)
    dims, planes = net3d(seed=3, dims=(41, 27, 19))
    ref = oracle.solve(dims, planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        r = net.solve(ns.make_opts(precision=precision))
        P = net.pressure()
    assert r.status == ns.NET_OK
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
    assert np.max(np.abs(P - ref.P)) <= 1e-7


@pytest.mark.parametrize("shape", ["1024,0,1", "512,0,2", "256,0,4", "64,0,3"])
def test_every_2d_shape_matches_oracle_batched(ns, monkeypatch, shape):
    """2D FP32 inner loops of a batch and 2D FP64 inner loops run the sweep
    kernel under the forced shape."""
    monkeypatch.setenv("NETSOLVE_SWEEP_SHAPE", shape)
    specs = [netgen.batch_instance(i, smin=40, smax=300) for i in range(4)]
    nets = [ns.Network(d, p) for d, p in specs]
    res = ns.solve_batch(nets)
    res64 = [n.solve(ns.make_opts(precision=ns.NET_FP64)) for n in nets]
    for n in nets:
        n.close()
    for (dims, planes), r, r64 in zip(specs, res, res64):
        ref = oracle.solve(dims, planes, tol=1e-13)
        assert r.status == ns.NET_OK and r64.status == ns.NET_OK
        if ref.g_eff == 0.0:
            assert r.g_eff == 0.0 and r64.g_eff == 0.0
            continue
        assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert rel(r64.g_eff, ref.g_eff) <= G_TOL


def test_batch_tunes_by_itself_and_reuses_the_entry(ns, monkeypatch):
    """A batch of an untuned size class tunes once (its networks are re-armed
    afterwards); a second batch of that class reuses the shape, so the two
    batches agree bit for bit."""
    ns.tune_clear()
    specs = [net3d(seed=20 + i, dims=(20 + i, 18, 16)) for i in range(5)]
    nets = [ns.Network(d, p) for d, p in specs]
    r1 = ns.solve_batch(nets)
    r2 = ns.solve_batch(nets)
    for n in nets:
        n.close()
    assert [x.g_eff for x in r1] == [x.g_eff for x in r2]
    for (dims, planes), r in zip(specs, r1):
        ref = oracle.solve(dims, planes, tol=1e-13)
        if ref.g_eff > 0:
            assert rel(r.g_eff, ref.g_eff) <= G_TOL


def test_tuning_off_uses_default_shape(ns, monkeypatch):
    monkeypatch.setenv("NETSOLVE_AUTOTUNE", "0")
    ns.tune_clear()
    dims, planes = net3d(seed=5)
    ref = oracle.solve(dims, planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        r = net.solve()
    assert rel(r.g_eff, ref.g_eff) <= G_TOL
