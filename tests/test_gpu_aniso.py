"""Permeability anisotropy workload (Sec. VI.B, Fig. 10): both flow axes of
anisotropic FBM networks (Eq. 2) solved in one batch must match the FP64
oracle along each axis, and K_x of a field must equal K_y of its transpose."""
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


@pytest.mark.parametrize("hi,ri", [(0, 4), (1, 0), (1, 2)])
def test_both_axes_batched_match_oracle(ns, hi, ri):
    specs = [netgen.aniso_instance(hi, ri, r, n=72) for r in range(2)]
    nets = [ns.Network(d, p, flow_axis=ax) for d, p in specs for ax in (0, 1)]
    res = ns.solve_batch(nets)
    for n in nets:
        n.close()
    for k, (d, p) in enumerate(specs):
        for ax in (0, 1):
            r = res[2 * k + ax]
            ref = oracle.solve(d, p, flow_axis=ax, tol=1e-13)
            assert r.status == ns.NET_OK
            assert rel(r.g_eff, ref.g_eff) <= G_TOL
            assert rel(r.k_eff, ref.k_eff) <= G_TOL


def test_kx_equals_ky_of_the_transposed_field(ns):
    dims, (gx, gy) = netgen.aniso_instance(1, 4, 0, n=80)
    # transpose: the y bonds become x bonds and vice versa
    tdims = (dims[1], dims[0])
    tplanes = [np.ascontiguousarray(gy.T), np.ascontiguousarray(gx.T)]
    with ns.Network(dims, [gx, gy], flow_axis=0) as a, ns.Network(tdims, tplanes, flow_axis=1) as b:
        ra, rb = a.solve(), b.solve()
    assert rel(ra.k_eff, rb.k_eff) <= G_TOL


@pytest.mark.parametrize("hi,ri", [(0, 3), (1, 1)])
def test_periodic_both_axes_batched_match_oracle(ns, hi, ri):
    """The paper's boundaries (periodic transverse faces): K_x from the field
    with periodic y, K_y from its transpose with periodic y, all in one batch
    (the periodic members take the batched compacted path), against the
    periodic oracle."""
    pairs = [netgen.aniso_pair_periodic(hi, ri, r, n=64) for r in range(2)]
    specs = [spec for pair in pairs for spec in pair]
    nets = [ns.Network(d, p, periodic=(1,)) for d, p in specs]
    res = ns.solve_batch(nets)
    for n in nets:
        n.close()
    for (d, p), r in zip(specs, res):
        ref = oracle.solve(d, p, tol=1e-13, periodic=(1,))
        assert r.status == ns.NET_OK, r
        assert rel(r.g_eff, ref.g_eff) <= G_TOL
        assert rel(r.k_eff, ref.k_eff) <= G_TOL
