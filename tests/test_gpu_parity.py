"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: effective conductance within 1e-8 relative (the accuracy target
of the solver); node pressures within 1e-7 of the pressure drop (the outer
tolerance 1e-11 on the relative residual times the condition numbers of
these small networks); cluster labels and classes bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen

pytestmark = pytest.mark.gpu

G_TOL = 1e-8
P_TOL = 1e-7


@pytest.fixture(scope="module")
def ns():
    import torch

    assert torch.cuda.is_available()
    from paper_1908_03301_gb300 import netsolve

    netsolve.lib(build_if_missing=True)
    return netsolve


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_against_oracle(ns, dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, precision=0,
                         g_tol=G_TOL, p_tol=P_TOL):
    ref = oracle.solve(dims, planes, flow_axis=flow_axis, p_in=p_in, p_out=p_out, tol=1e-13)
    with ns.Network(dims, planes, flow_axis, p_in, p_out) as net:
        r = net.solve(ns.make_opts(precision=precision))
        P = net.pressure()
        lab, cls = net.labels()
    assert r.status == ns.NET_OK, r
    assert r.n_active == ref.n_active
    np.testing.assert_array_equal(lab, ref.label)
    np.testing.assert_array_equal(cls, ref.cls)
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
    else:
        assert rel(r.g_eff, ref.g_eff) <= g_tol, (r.g_eff, ref.g_eff)
        assert rel(r.q_out, ref.q_out) <= 1e-7
    dp = abs(p_in - p_out)
    assert np.max(np.abs(P - ref.P)) <= p_tol * dp
    return r, ref


# ------------------------------------------------------------ small workload
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", ["random", "uniform", "stratified"])
def test_small_64x64_variants(ns, variant, precision):
    dims, planes, s = netgen.workload_small(variant)
    r, ref = check_against_oracle(ns, dims, planes, precision=precision)
    if variant == "uniform":
        assert rel(r.g_eff, 64.0 / 63.0) <= 1e-12
    if variant == "stratified":
        assert rel(r.g_eff, s.sum() / 63.0) <= G_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_small_stratified_across_layers(ns, precision):
    dims, planes, s = netgen.workload_small("stratified")
    r, ref = check_against_oracle(ns, dims, planes, flow_axis=1, precision=precision)
    assert rel(r.g_eff, 64.0 / np.sum(1.0 / s[:-1])) <= G_TOL


# ------------------------------------------------------------ ragged and 3D
@pytest.mark.parametrize("dims,f,p", [((67, 45), 0, 1.0), ((45, 67), 1, 0.62),
                                       ((257, 19), 0, 0.8), ((3, 50), 0, 1.0),
                                       ((50, 3), 1, 1.0), ((300, 1), 0, 1.0),
                                       ((33, 17, 21), 0, 1.0), ((17, 21, 33), 2, 0.45),
                                       ((21, 33, 17), 1, 0.35), ((70, 9, 11), 0, 0.6)])
@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_shapes(ns, dims, f, p, precision):
    gen = netgen.rng(1000 + sum(dims) + f)
    planes = netgen.lognormal_iid(dims, gen, 1.0)
    if p < 1.0:
        planes = netgen.percolate(planes, p, gen)
    check_against_oracle(ns, dims, planes, flow_axis=f, precision=precision, p_in=2.5,
                         p_out=-0.5)


@pytest.mark.parametrize("precision", [0, 1])
def test_float32_bonds_3d_percolation(ns, precision):
    """FP32 conductances (the 3D percolation workload's dtype), p = 0.3."""
    dims, planes = netgen.workload_perc3d(n=40, p=0.3, seed=7)
    assert planes[0].dtype == np.float32
    r, ref = check_against_oracle(ns, dims, planes, precision=precision)
    assert r.n_active > 0


def test_labels_3d_near_threshold(ns):
    dims, planes = netgen.workload_perc3d(n=64, p=0.26, seed=11)
    lab_ref, cls_ref = oracle.labels(dims, planes)
    with ns.Network(dims, planes) as net:
        lab, cls = net.labels()
    np.testing.assert_array_equal(lab, lab_ref)
    np.testing.assert_array_equal(cls, cls_ref)


# ------------------------------------------------------------ degenerate cases
def test_no_spanning_cluster(ns):
    dims = (20, 12)
    gen = netgen.rng(5)
    planes = netgen.lognormal_iid(dims, gen)
    planes[0][:, 9] = 0.0
    with ns.Network(dims, planes) as net:
        r = net.solve()
        P = net.pressure()
        lab, cls = net.labels()
    assert r.status == ns.NET_OK and r.g_eff == 0.0 and r.n_active == 0
    ref = oracle.solve(dims, planes)
    np.testing.assert_array_equal(P, ref.P)
    np.testing.assert_array_equal(cls, ref.cls)


def test_all_bonds_closed(ns):
    dims = (9, 9)
    planes = [np.zeros(netgen.plane_shape(dims, d)) for d in range(2)]
    with ns.Network(dims, planes) as net:
        r = net.solve()
    assert r.g_eff == 0.0 and r.n_active == 0


def test_minimum_length_three(ns):
    dims = (3, 6)
    gen = netgen.rng(8)
    planes = netgen.loguniform_iid(dims, gen)
    check_against_oracle(ns, dims, planes)


def test_invalid_conductances(ns):
    dims = (10, 10)
    for bad in (-1.0, np.nan, np.inf):
        planes = netgen.uniform(dims)
        planes[1][3, 4] = bad
        with pytest.raises(ns.NetError) as ei:
            ns.Network(dims, planes)
        assert ei.value.status == ns.NET_EINVAL


# ------------------------------------------------------------ API behaviour
def test_device_input_equals_host_input(ns):
    import torch

    dims = (130, 70)
    gen = netgen.rng(21)
    planes = netgen.percolate(netgen.loguniform_iid(dims, gen), 0.7, gen)
    r1, P1 = ns.solve(dims, planes)
    tplanes = [torch.from_numpy(g).cuda() for g in planes]
    with ns.Network(dims, tplanes) as net:
        r2 = net.solve()
        P2 = net.pressure(torch.empty(dims[0] * dims[1], dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert r1.g_eff == r2.g_eff
    np.testing.assert_array_equal(P1.reshape(-1), P2.cpu().numpy())


def test_repeat_solve_is_bit_identical(ns):
    dims = (96, 80)
    gen = netgen.rng(22)
    planes = netgen.lognormal_iid(dims, gen, 1.0)
    with ns.Network(dims, planes) as net:
        a = net.solve()
        Pa = net.pressure()
        b = net.solve()
        Pb = net.pressure()
    assert a.g_eff == b.g_eff and a.inner_iters == b.inner_iters
    np.testing.assert_array_equal(Pa, Pb)


def test_resume_from_interrupted_solve(ns):
    """Checkpoint/resume: a capped solve's pressures are a valid restart."""
    dims = (128, 128)
    gen = netgen.rng(23)
    planes = netgen.fbm_bonds(dims, 0.7, 1.5, gen)
    with ns.Network(dims, planes) as net:
        full = net.solve()
        part = net.solve(ns.make_opts(max_outer=1, tol_inner=1e-2), check=False)
        assert part.status == ns.NET_ENOTCONVERGED
        x_ck = net.pressure()
        resumed = net.solve(x0=x_ck)
    assert resumed.status == ns.NET_OK
    assert rel(resumed.g_eff, full.g_eff) <= G_TOL


def test_mixed_matches_fp64(ns):
    dims = (256, 256)
    gen = netgen.rng(24)
    planes = netgen.fbm_bonds(dims, 0.7, 1.5, gen)
    rm, _ = ns.solve(dims, planes, precision=ns.NET_MIXED)
    rd, _ = ns.solve(dims, planes, precision=ns.NET_FP64)
    ref = oracle.solve(dims, planes, tol=1e-13)
    assert rel(rm.g_eff, ref.g_eff) <= G_TOL
    assert rel(rd.g_eff, ref.g_eff) <= G_TOL
    assert rm.fp64_fallback == 0


@pytest.mark.parametrize("dims,p,per,kernel", [((200, 150), 0.65, (), ""), ((200, 150), 0.65, (), "compact"),
                                               ((40, 36, 30), 0.33, (1,), ""), ((48, 40, 36), 0.3, (), "")])
def test_invariants_after_solve(ns, monkeypatch, dims, p, per, kernel):
    """Flux balance, Tellegen (energy = G) and the reported largest nodal
    imbalance against the oracle's residual of the returned pressures: for
    the lattice kernels and for the list path, whose refinement pass sums
    over the listed unknowns only (3D sparse networks take it by default)."""
    if kernel:
        monkeypatch.setenv("NETSOLVE_KERNEL", kernel)
    gen = netgen.rng(25 + len(dims))
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, periodic=per), p, gen)
    with ns.Network(dims, planes, periodic=per) as net:
        r = net.solve()
        P = net.pressure()
    assert r.status == ns.NET_OK and r.g_eff > 0.0
    assert rel(r.q_out, r.q_in) <= 1e-8
    assert rel(r.energy_g, r.g_eff) <= 1e-8
    imb = oracle.residual(dims, planes, P, periodic=per)
    assert np.max(np.abs(imb)) <= 1e-8 * max(np.max(g) for g in planes)
    assert abs(np.max(np.abs(imb)) - r.max_imbalance) <= 1e-12 + 1e-6 * r.max_imbalance


@pytest.mark.parametrize("tol_rel", [1e-6, 1e-8])
def test_geff_error_estimate_tracks_actual_error(ns, tol_rel):
    """The reported g_eff_err (first-order adjoint estimate) matches the
    actual relative error against the oracle when the solve stops early."""
    dims = (160, 120)
    gen = netgen.rng(31)
    planes = netgen.percolate(netgen.lognormal_iid(dims, gen, 1.5), 0.7, gen)
    ref = oracle.solve(dims, planes, tol=1e-14)
    with ns.Network(dims, planes) as net:
        r = net.solve(ns.make_opts(precision=ns.NET_FP64, tol_rel=tol_rel, tol_geff=1.0))
    actual = rel(r.g_eff, ref.g_eff)
    assert actual > 1e-13  # the early stop left a measurable error
    assert 0.8 <= r.g_eff_err / actual <= 1.25, (r.g_eff_err, actual)


# ------------------------------------------------- refinement modes, kernels
@pytest.fixture
def kernel_env():
    import os

    old = os.environ.get("NETSOLVE_KERNEL")
    yield os.environ
    if old is None:
        os.environ.pop("NETSOLVE_KERNEL", None)
    else:
        os.environ["NETSOLVE_KERNEL"] = old


def _ill_conditioned(dims, seed):
    gen = netgen.rng(seed)
    return netgen.percolate(netgen.lognormal_iid(dims, gen, 1.5), 0.62, gen)


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("kernel,dims", [("persist", (150, 131)), ("sweep", (150, 131)),
                                         ("compact", (150, 131)), ("sweep", (23, 30, 27)),
                                         ("compact", (23, 30, 27))])
def test_refine_modes_every_kernel(ns, kernel_env, kernel, dims, refine):
    """Reliable updates (the recursion kept across refinement passes, with
    the true residual put in place of the recursive one) and classical
    restarted refinement reach the oracle's G_eff and pressures through each
    inner-loop kernel: the persistent in-place kernel, the double-buffered
    sweep kernel and the compacted solve."""
    kernel_env["NETSOLVE_KERNEL"] = kernel
    planes = _ill_conditioned(dims, 40 + len(dims))
    ref = oracle.solve(dims, planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        r = net.solve(ns.make_opts(refine=refine))
        P = net.pressure()
    assert r.status == ns.NET_OK, r
    assert rel(r.g_eff, ref.g_eff) <= G_TOL, (r.g_eff, ref.g_eff)
    assert np.max(np.abs(P - ref.P)) <= P_TOL
    if refine == ns.NET_REFINE_RELIABLE:
        assert r.outer_iters >= 2  # the recursion was carried across passes


def test_reliable_updates_save_iterations(ns):
    """On an ill-conditioned network the FP32 inner loop with reliable
    updates needs no more CG iterations than restarted refinement."""
    dims = (256, 256)
    planes = _ill_conditioned(dims, 77)
    with ns.Network(dims, planes) as net:
        a = net.solve(ns.make_opts(refine=ns.NET_REFINE_RELIABLE))
        b = net.solve(ns.make_opts(refine=ns.NET_REFINE_RESTART))
    assert a.status == ns.NET_OK and b.status == ns.NET_OK
    assert rel(a.g_eff, b.g_eff) <= G_TOL
    assert a.inner_iters <= 1.1 * b.inner_iters, (a.inner_iters, b.inner_iters)


def test_refine_options_are_checked(ns):
    dims = (20, 20)
    with ns.Network(dims, netgen.uniform(dims)) as net:
        for kw in ({"refine": 7}, {"update_delta": 1.5}, {"update_delta": -0.1}):
            r = net.solve(ns.make_opts(**kw), check=False)
            assert r.status == ns.NET_EINVAL, kw
        r = net.solve(ns.make_opts(update_delta=0.01))
        assert r.status == ns.NET_OK and rel(r.g_eff, 20 / 19) <= 1e-12
