"""Full-size parity: the 2048^2 correlated networks (bench workload) against
the oracle's stored full-size results and against exact closed forms, and
the 256^3 near-threshold percolation network's labels, bit for bit.

The stored values come from tests/golden/make_oracle_reference.py (oracle
only, tol 1e-13)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen

pytestmark = pytest.mark.gpu
G_TOL = 1e-8
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_full_size.json")


@pytest.fixture(scope="module")
def ns():
    import torch

    assert torch.cuda.is_available()
    from paper_1908_03301_gb300 import netsolve

    netsolve.lib(build_if_missing=True)
    return netsolve


def stored(name):
    d = json.load(open(GOLD))
    if name not in d:
        pytest.skip(f"no stored oracle result for {name}")
    return d[name]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("name,variant,f", [("fbm2048_iso_x", "isotropic", 0),
                                              ("fbm2048_strat_x", "stratified", 0),
                                              ("fbm2048_strat_y", "stratified", 1)])
@pytest.mark.parametrize("precision", [0, 1])
def test_fbm2048_against_stored_oracle(ns, name, variant, f, precision):
    ref = stored(name)
    dims, planes = netgen.workload_fbm2d(variant=variant)
    with ns.Network(dims, planes, flow_axis=f) as net:
        r = net.solve(ns.make_opts(precision=precision))
    assert r.status == ns.NET_OK
    assert r.n_active == ref["n_active"]
    assert rel(r.g_eff, ref["g_eff"]) <= G_TOL
    assert rel(r.q_out, r.q_in) <= 1e-8
    assert rel(r.energy_g, r.g_eff) <= 1e-8


def test_fbm2048_pressures_against_stored_oracle(ns):
    """Pressures of the 2048^2 headline network (persistent kernel over all
    152 SMs, L2 set-aside) at 64 x 64 sampled nodes, element by element
    against the oracle's stored values."""
    ref = stored("fbm2048_iso_x")
    if "P_sample" not in ref:
        pytest.skip("no stored oracle pressures")
    smp = ref["P_sample"]
    dims, planes = netgen.workload_fbm2d(variant="isotropic")
    with ns.Network(dims, planes) as net:
        r = net.solve()
        P = net.pressure()
    assert r.status == ns.NET_OK
    got = P[np.ix_(smp["rows"], smp["cols"])]
    assert np.max(np.abs(got - np.array(smp["values"]))) <= 1e-7


def test_fbm2048_layered_closed_forms(ns):
    """Noise-free layers: arithmetic mean along, harmonic mean across."""
    dims, planes = netgen.workload_fbm2d(variant="stratified_exact")
    gx, gy = planes
    nx, ny = dims
    g_along = gx[:, 0].sum() / (nx - 1)          # each row is a uniform chain
    g_across = nx / np.sum(1.0 / gy[:, 0])       # each column is a chain of t_j
    with ns.Network(dims, planes, flow_axis=0) as net:
        rx = net.solve()
    with ns.Network(dims, planes, flow_axis=1) as net:
        ry = net.solve()
    assert rel(rx.g_eff, g_along) <= G_TOL
    assert rel(ry.g_eff, g_across) <= G_TOL


def test_perc256_labels_bit_exact(ns):
    dims, planes = netgen.workload_perc3d()
    lab_ref, cls_ref = oracle.labels(dims, planes)
    with ns.Network(dims, planes) as net:
        lab, cls = net.labels()
    np.testing.assert_array_equal(cls, cls_ref)
    np.testing.assert_array_equal(lab, lab_ref)


def test_perc256_backbone_bit_exact(ns):
    """The current-carrying backbone of the 256^3 network (dead-end trees and
    loops removed), bit for bit against the oracle's Hopcroft-Tarjan blocks."""
    dims, planes = netgen.workload_perc3d()
    want = oracle.backbone_blocks(dims, planes)
    with ns.Network(dims, planes) as net:
        bb = net.backbone()
    np.testing.assert_array_equal(bb, want)


def test_perc256_solve(ns):
    dims, planes = netgen.workload_perc3d()
    with ns.Network(dims, planes) as net:
        rm = net.solve()
        rd = net.solve(ns.make_opts(precision=ns.NET_FP64))
    assert rm.status == ns.NET_OK and rd.status == ns.NET_OK
    assert rm.n_active > 0
    assert rel(rm.g_eff, rd.g_eff) <= G_TOL
    assert rel(rm.q_out, rm.q_in) <= 1e-8
    assert rel(rm.energy_g, rm.g_eff) <= 1e-8
    d = json.load(open(GOLD))
    if "perc256_x" in d:
        assert rel(rm.g_eff, d["perc256_x"]["g_eff"]) <= G_TOL
        assert rm.n_active == d["perc256_x"]["n_active"]
