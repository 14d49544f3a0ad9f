"""Correlated percolation by sorted removal (Sec. VI.B) on the device: the
closed set must be the oracle's bit for bit (a stable sort of all bonds by
conductance), with many equal conductances, zeros and -0, both dtypes, 2D,
3D and periodic planes, and sizes that span many chunks of the tie ranking."""
import numpy as np
import pytest

import oracle
from paper_1908_03301_gb300 import netgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ns():
    import torch

    assert torch.cuda.is_available()
    from paper_1908_03301_gb300 import netsolve

    netsolve.lib(build_if_missing=True)
    return netsolve


def _run(ns, dims, planes, q, periodic=()):
    import torch

    t = [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in planes]
    ns.close_smallest(dims, t, q, periodic=periodic)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in t]


def _check(got, want):
    for a, b in zip(got, want):
        assert a.dtype == b.dtype
        np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8))


CASES = [((37, 29), np.float64, 0, 0.5, (), 1), ((37, 29), np.float32, 0, 0.013, (), 2),
         ((21, 18, 15), np.float32, 3, 0.37, (), 3), ((21, 18, 15), np.float64, 2, 0.999, (), 4),
         ((16, 12, 10), np.float32, 5, 0.6, (1, 2), 5), ((64, 48), np.float64, 1, 0.25, (1,), 6),
         ((9, 7), np.float64, 0, 1.0, (), 7), ((9, 7), np.float32, 0, 0.0, (), 8),
         ((128, 128, 128), np.float32, 7, 0.41, (), 9), ((700, 650), np.float64, 3, 0.52, (1,), 10)]


@pytest.mark.parametrize("dims,dtype,levels,q,per,seed", CASES)
def test_close_smallest_matches_oracle(ns, dims, dtype, levels, q, per, seed):
    gen = netgen.rng(9600 + seed)
    planes = netgen.lognormal_iid(dims, gen, periodic=per)
    if levels:  # few distinct values: ties straddle the cut
        planes = [np.floor(g * levels) / levels for g in planes]
    planes = [g.astype(dtype) for g in planes]
    if seed % 2:  # some negative zeros, which order like 0
        planes[0].reshape(-1)[::97] = -0.0
    want = oracle.close_smallest(planes, q)
    got = _run(ns, dims, planes, q, per)
    _check(got, want)


def test_close_smallest_rejects_bad_input(ns):
    import torch

    dims = (10, 8)
    planes = [torch.ones(netgen.plane_shape(dims, d), dtype=torch.float64, device="cuda") for d in range(2)]
    planes[1][3, 4] = -1.0
    with pytest.raises(ns.NetError) as e:
        ns.close_smallest(dims, planes, 0.5)
    assert e.value.status == ns.NET_EINVAL
    assert int((planes[0] == 0).sum()) == 0 and int((planes[1] == 0).sum()) == 0  # untouched
    planes[1][3, 4] = 1.0
    with pytest.raises(ns.NetError):
        ns.close_smallest(dims, planes, 1.5)


def test_sorted_removal_network_solves_like_oracle(ns):
    """Sec. VI.B workload in small: an FBM network (H = 0.7, sigma = 1) with
    the weakest 45 % of bonds closed on the device, then solved; the oracle
    closes the same bonds and solves in FP64."""
    import torch

    gen = netgen.rng(9650)
    dims = (96, 96)
    planes = netgen.fbm_bonds(dims, 0.7, 1.0, gen)
    t = [torch.from_numpy(g).cuda() for g in planes]
    ns.close_smallest(dims, t, 0.45)
    ref_planes = oracle.close_smallest(planes, 0.45)
    _check([x.cpu().numpy() for x in t], ref_planes)
    ref = oracle.solve(dims, ref_planes, tol=1e-13)
    with ns.Network(dims, t) as net:
        r = net.solve()
    if ref.g_eff == 0.0:
        assert r.g_eff == 0.0
    else:
        assert abs(r.g_eff - ref.g_eff) <= 1e-8 * ref.g_eff
