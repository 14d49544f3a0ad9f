"""Input generators (no solver arithmetic): the anisotropic FBM of Eq. 2 and
correlated (sorted-removal) percolation of Sec. VI.B."""
import numpy as np

from paper_1908_03301_gb300 import netgen


def test_aniso_fbm_reduces_to_isotropic_for_equal_betas():
    a = netgen.fbm_field((64, 48), 0.7, netgen.rng(3))
    b = netgen.fbm_field_aniso((64, 48), 0.7, 1.0, 1.0, netgen.rng(3))
    assert np.array_equal(a, b)


def test_aniso_fbm_is_smoother_along_the_heavier_beta():
    """beta_x / beta_y > 1 damps the x frequencies: layers parallel to x, so
    increments along x are smaller than along y (and the reverse for < 1)."""
    for ratio, along_x_smaller in ((5.0, True), (0.2, False)):
        dx, dy = [], []
        for r in range(4):
            f = netgen.fbm_field_aniso((256, 256), 0.35, ratio, 1.0, netgen.rng(100 + r))
            dx.append(np.mean(np.diff(f, axis=1) ** 2))
            dy.append(np.mean(np.diff(f, axis=0) ** 2))
        assert (np.mean(dx) < np.mean(dy)) == along_x_smaller


def test_aniso_field_is_normalised():
    f = netgen.fbm_field_aniso((128, 96), 0.75, 2.0, 1.0, netgen.rng(7))
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12


def test_sorted_removal_closes_the_smallest_fraction():
    dims, planes = netgen.aniso_instance(1, 2, 0, n=96)
    for q in (0.0, 0.3, 0.5):
        out = netgen.percolate_sorted(planes, q)
        flat_in = np.concatenate([g.ravel() for g in planes])
        flat = np.concatenate([g.ravel() for g in out])
        closed = flat == 0.0
        assert closed.sum() == int(np.floor(q * flat.size))
        if closed.any():
            assert flat_in[closed].max() <= flat_in[~closed].min()
        assert np.array_equal(flat[~closed], flat_in[~closed])


def test_aniso_instances_are_seeded_and_distinct():
    d1, p1 = netgen.aniso_instance(0, 1, 2, n=64)
    d2, p2 = netgen.aniso_instance(0, 1, 2, n=64)
    d3, p3 = netgen.aniso_instance(0, 1, 3, n=64)
    assert d1 == (64, 64) and np.array_equal(p1[0], p2[0]) and not np.array_equal(p1[0], p3[0])


def test_periodic_plane_shapes_and_wrap_bonds():
    """Along a periodic axis a plane has one bond per node; the generators'
    wrap layer joins the last node layer to the first (mean of the two end
    nodes for the FBM map), and the other bonds equal the no-flow ones."""
    dims = (12, 9, 7)
    assert netgen.plane_shape(dims, 1, periodic=(1,)) == (7, 9, 12)
    assert netgen.plane_shape(dims, 1) == (7, 8, 12)
    assert netgen.n_bonds(dims, periodic=(1, 2)) == [11 * 9 * 7, 12 * 9 * 7, 12 * 9 * 7]
    a = netgen.fbm_bonds(dims, 0.6, 1.0, netgen.rng(5))
    b = netgen.fbm_bonds(dims, 0.6, 1.0, netgen.rng(5), periodic=(1, 2))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1][:, :-1, :])
    np.testing.assert_array_equal(a[2], b[2][:-1])
    B = netgen.fbm_field(netgen.node_shape(dims), 0.6, netgen.rng(5))
    np.testing.assert_allclose(b[1][:, -1, :], np.exp(0.5 * (B[:, -1, :] + B[:, 0, :])), rtol=1e-15)
    np.testing.assert_allclose(b[2][-1], np.exp(0.5 * (B[-1] + B[0])), rtol=1e-15)
    u = netgen.uniform(dims, 2.0, periodic=(2,))
    assert [g.shape for g in u] == [(7, 9, 11), (7, 8, 12), (7, 9, 12)]


def test_fbm_generator_matches_oracle_filtering():
    """netgen's isotropic FBM field (the workloads' inputs) is the oracle's
    spectral filtering of the same noise draw."""
    import oracle

    shape = (40, 56)
    field = netgen.fbm_field(shape, 0.7, netgen.rng(77))
    gen = netgen.rng(77)
    noise = gen.standard_normal(shape) + 1j * gen.standard_normal(shape)
    np.testing.assert_allclose(field, oracle.fbm_field(noise, 0.7), rtol=0, atol=1e-12)


def test_aniso_pair_periodic_is_the_instance_with_wrap_bonds():
    """The periodic anisotropy pair holds the same realization as the no-flow
    instance (identical bulk bonds), plus the wrap bonds, and its second
    network is the transpose of the first."""
    (d, (gx, gy)), (dt, (tx, ty)) = netgen.aniso_pair_periodic(0, 2, 0, n=32)
    d0, (ax, ay) = netgen.aniso_instance(0, 2, 0, n=32)
    assert d == dt == d0 == (32, 32)
    assert gx.shape == (32, 31) and gy.shape == (32, 32)
    np.testing.assert_allclose(gx, ax, rtol=0, atol=0)
    np.testing.assert_allclose(gy[:-1], ay, rtol=0, atol=0)
    np.testing.assert_allclose(tx, gy[:-1].T, rtol=1e-15)
    np.testing.assert_allclose(ty[:-1], gx.T, rtol=1e-15)
