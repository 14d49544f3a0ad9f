"""The FBM generator on the device (Eq. 1, Eq. 2) against the oracle's
spectral filtering of the same noise, the conductance map, and the whole
chain noise -> field -> bonds -> solve against the oracle's chain."""
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


def _noise(shape, seed):
    gen = netgen.rng(9900 + seed)
    return gen.standard_normal(shape) + 1j * gen.standard_normal(shape)


def _gpu_field(ns, dims, noise, H, beta=None, f32=False):
    import torch

    t = torch.from_numpy(noise.astype(np.complex64) if f32 else noise.copy()).cuda()
    f = ns.fbm_field(dims, t, H, beta)
    return f.cpu().numpy()


CASES = [((64, 48), 0.7, None, 1), ((256, 256), 0.3, None, 2), ((333, 200), 0.75, (5.0, 1.0), 3),
         ((101, 77), 0.35, (0.2, 1.0), 4), ((32, 24, 20), 0.3, None, 5), ((17, 30, 9), 0.6, (1.0, 2.0, 0.5), 6)]


@pytest.mark.parametrize("dims,H,beta,seed", CASES)
def test_fbm_field_matches_oracle(ns, dims, H, beta, seed):
    shape = tuple(reversed(dims))
    noise = _noise(shape, seed)
    want = oracle.fbm_field(noise, H, beta)
    got = _gpu_field(ns, dims, noise, H, beta)
    # FP64 FFTs of two libraries: rounding differences only (unit variance field)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11)
    assert abs(got.mean()) < 1e-12 and abs(np.mean(got * got) - 1.0) < 1e-12


@pytest.mark.parametrize("dims,H,beta,seed", CASES)
def test_fbm_field_fp32_transform(ns, dims, H, beta, seed):
    """The FP32 transform: the oracle's field (FP64, from the same noise
    rounded to FP32) to FP32 accuracy."""
    shape = tuple(reversed(dims))
    noise = _noise(shape, seed).astype(np.complex64)
    want = oracle.fbm_field(noise.astype(np.complex128), H, beta)
    got = _gpu_field(ns, dims, noise, H, beta, f32=True)
    assert np.max(np.abs(got - want)) < 1e-4
    assert np.sqrt(np.mean((got - want) ** 2)) < 1e-5
    # mean and variance are formed in FP32 per thread: FP32-level normalisation
    assert abs(got.mean()) < 1e-6 and abs(np.mean(got * got) - 1.0) < 1e-5


@pytest.mark.parametrize("per", [(), (1,)])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_fbm_bonds_match_oracle(ns, per, dtype):
    import torch

    dims = (90, 70)
    field = oracle.fbm_field(_noise((70, 90), 7), 0.7)
    planes = ns.fbm_bonds(dims, torch.from_numpy(field).cuda(), 1.5, getattr(torch, dtype), periodic=per)
    want = oracle.fbm_bonds(field, 1.5)
    if per:  # the wrap bonds join the last row to row 0
        want[1] = np.exp(1.5 * 0.5 * (field + np.roll(field, -1, axis=0)))
    for g, w in zip(planes, want):
        got = g.cpu().numpy()
        assert got.shape == w.shape
        # FP32 planes: the argument formed in FP32 (|arg| < 8 here)
        rt = 1e-14 if dtype == "float64" else 2e-6
        np.testing.assert_allclose(got, w.astype(got.dtype), rtol=rt)


def test_fbm_bonds_3d_periodic(ns):
    """3D planes with periodic y and z: the wrap layers join the last and
    first node layers of the field."""
    import torch

    dims, per = (20, 17, 13), (1, 2)
    field = oracle.fbm_field(_noise((13, 17, 20), 9), 0.4)
    planes = ns.fbm_bonds(dims, torch.from_numpy(field).cuda(), 0.8, periodic=per)
    want = [np.exp(0.4 * (field[:, :, :-1] + field[:, :, 1:])),
            np.exp(0.4 * (field + np.roll(field, -1, axis=1))),
            np.exp(0.4 * (field + np.roll(field, -1, axis=0)))]
    for g, w in zip(planes, want):
        np.testing.assert_allclose(g.cpu().numpy(), w, rtol=1e-14)


def test_fbm_network_chain_matches_oracle(ns):
    """noise -> field -> conductances -> solve on the device, against the
    oracle's field, map and solve (Sec. II's correlated network)."""
    import torch

    dims, H, sigma = (160, 128), 0.7, 1.5
    noise = _noise((128, 160), 8)
    tn = torch.from_numpy(noise.copy()).cuda()
    planes = ns.fbm_bonds(dims, ns.fbm_field(dims, tn, H), sigma)
    ref_planes = oracle.fbm_bonds(oracle.fbm_field(noise, H), sigma)
    ref = oracle.solve(dims, ref_planes, tol=1e-13)
    with ns.Network(dims, planes) as net:
        r = net.solve()
    assert r.status == ns.NET_OK
    assert abs(r.g_eff - ref.g_eff) <= 1e-8 * ref.g_eff
