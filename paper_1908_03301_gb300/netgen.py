"""Seeded synthetic bond networks (input preparation only).

This module draws conductance fields for square (2D) and cubic (3D) bond
networks.  It holds none of the solver's arithmetic: it only produces the
per-bond conductance planes that both the CUDA path and the CPU oracle take as
input.  It imports neither of them.

Layout
------
``dims`` is ``(nx, ny)`` or ``(nx, ny, nz)``; x is the fastest axis.  A node
field is a numpy array of shape ``(ny, nx)`` / ``(nz, ny, nx)``.  Bond plane
``d`` holds the bond from node ``i`` to ``i + e_d``; its shape is the node
shape with the extent along axis ``d`` reduced by one (no-flow transverse
boundaries).  ``g == 0`` marks a closed (insulating) bond.

Workloads (the paper's network families, Sec. II and Sec. V-VI)
---------------------------------------------------------------
* i.i.d. conductances (random-resistor network, Sec. II);
* fractional-Brownian-motion (FBM) correlated conductances generated by
  Fourier filtering with spectral density S(k) ~ |k|^-(2H+d) (Eq. 1 for d=2;
  the standard generalisation for d=1, 3);
* stratified (layered) media, the extreme anisotropic limit of Eq. 2;
* bond percolation: each bond is open with probability p independently of its
  conductance (Sec. V).

Seeds: workload ``k`` uses ``PCG64(SEED_BASE + k)``; instance ``i`` of a
multi-network workload ``k`` uses ``PCG64(SEED_BASE + 1000*k + i)``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20190809


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def node_shape(dims):
    return tuple(reversed(tuple(int(v) for v in dims)))


def plane_shape(dims, d, periodic=()):
    """numpy shape of bond plane ``d`` (0 = x, 1 = y, 2 = z).  Along a
    periodic axis the plane has one bond per node: the last one wraps to the
    first layer."""
    n = list(int(v) for v in dims)
    if d not in periodic:
        n[d] -= 1
    return tuple(reversed(n))


def n_bonds(dims, periodic=()):
    return [int(np.prod(plane_shape(dims, d, periodic))) for d in range(len(dims))]


def _node_to_bonds(field, dims, periodic=()):
    """Bond value = mean of the two end-node values, for each direction
    (along a periodic axis the last bond joins the last and first layers)."""
    ndim = len(dims)
    out = []
    for d in range(ndim):
        ax = ndim - 1 - d  # numpy axis of lattice direction d
        if d in periodic:
            out.append(0.5 * (field + np.roll(field, -1, axis=ax)))
            continue
        lo = [slice(None)] * ndim
        hi = [slice(None)] * ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        out.append(0.5 * (field[tuple(lo)] + field[tuple(hi)]))
    return out


# --------------------------------------------------------------------------
# elementary fields
# --------------------------------------------------------------------------
def uniform(dims, value=1.0, dtype=np.float64, periodic=()):
    return [np.full(plane_shape(dims, d, periodic), value, dtype=dtype)
            for d in range(len(dims))]


def loguniform_iid(dims, gen, lo=-1.0, hi=1.0, periodic=()):
    """g = 10**U(lo, hi), i.i.d. per bond."""
    return [10.0 ** gen.uniform(lo, hi, size=plane_shape(dims, d, periodic))
            for d in range(len(dims))]


def lognormal_iid(dims, gen, sigma=1.0, periodic=()):
    """g = exp(sigma * N(0,1)), i.i.d. per bond."""
    return [np.exp(sigma * gen.standard_normal(plane_shape(dims, d, periodic)))
            for d in range(len(dims))]


def stratified_layers(dims, gen, sigma=1.0):
    """Perfectly layered 2D medium: one value s_y = exp(sigma*N(0,1)) per row.

    Horizontal bonds in row y carry s_y; the vertical bond between rows y and
    y+1 carries s_y as well.  Returns (planes, s) with s of length ny.
    """
    nx, ny = dims
    s = np.exp(sigma * gen.standard_normal(ny))
    gx = np.repeat(s[:, None], nx - 1, axis=1)
    gy = np.repeat(s[:-1, None], nx, axis=1)
    return [gx, gy], s


def fbm_field(shape, hurst, gen):
    """Fractional Brownian motion on a grid by spectral (Fourier) filtering.

    Amplitude sqrt(S(k)) with S(k) ~ |k|^-(2H+d), d = len(shape); complex
    Gaussian white noise; k = 0 removed; real part of the inverse FFT;
    normalised to zero mean and unit variance.
    """
    d = len(shape)
    freqs = np.meshgrid(*[np.fft.fftfreq(m) for m in shape], indexing="ij", sparse=True)
    k2 = np.zeros(shape)
    for f in freqs:
        k2 = k2 + f * f
    k2.flat[0] = 1.0
    amp = k2 ** (-(2.0 * hurst + d) / 4.0)
    amp.flat[0] = 0.0
    noise = gen.standard_normal(shape) + 1j * gen.standard_normal(shape)
    field = np.fft.ifftn(noise * amp).real
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def fbm_field_aniso(shape, hurst, beta_x, beta_y, gen):
    """2D FBM with the anisotropic spectral density of Eq. 2,
    S(w) ~ (beta_x w_x^2 + beta_y w_y^2)^-(H+1), by the same spectral
    filtering as fbm_field (which it equals for beta_x = beta_y = 1).
    shape = (ny, nx).  beta_x / beta_y > 1 gives layers parallel to x."""
    ny, nx = shape
    wy = np.fft.fftfreq(ny)[:, None]
    wx = np.fft.fftfreq(nx)[None, :]
    k2 = beta_x * wx * wx + beta_y * wy * wy
    k2[0, 0] = 1.0
    amp = k2 ** (-(hurst + 1.0) / 2.0)
    amp[0, 0] = 0.0
    noise = gen.standard_normal(shape) + 1j * gen.standard_normal(shape)
    field = np.fft.ifftn(noise * amp).real
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def fbm_aniso_bonds(dims, hurst, beta_x, beta_y, sigma, gen, periodic=()):
    """Anisotropic correlated conductances g = exp(sigma * B_b), B from Eq. 2
    (spectral synthesis makes B periodic, so wrap bonds fit it)."""
    B = fbm_field_aniso(node_shape(dims), hurst, beta_x, beta_y, gen)
    return [np.exp(sigma * b) for b in _node_to_bonds(B, dims, periodic)]


def fbm_bonds(dims, hurst, sigma, gen, periodic=()):
    """Correlated conductances g = exp(sigma * B_b), B an FBM on the nodes
    (spectral synthesis makes B periodic, so wrap bonds fit it)."""
    B = fbm_field(node_shape(dims), hurst, gen)
    return [np.exp(sigma * b) for b in _node_to_bonds(B, dims, periodic)]


def fbm_stratified_bonds(dims, hurst, sigma, gen, noise=0.1):
    """Layered medium: 1D FBM along y broadcast along x, plus i.i.d. noise.

    B_b = (B_i + B_j)/2 + noise * N(0,1) per bond; g = exp(sigma * B_b).
    """
    nx, ny = dims[0], dims[1]
    b1 = fbm_field((ny,), hurst, gen)
    shp = node_shape(dims)
    B = np.broadcast_to(b1.reshape((1,) * (len(dims) - 2) + (ny, 1)), shp).astype(np.float64)
    bonds = _node_to_bonds(B, dims)
    out = []
    for b in bonds:
        if noise:
            b = b + noise * gen.standard_normal(b.shape)
        out.append(np.exp(sigma * b))
    return out


def percolate(planes, p, gen):
    """Bond percolation: keep each bond open with probability p (independent)."""
    return [np.where(gen.random(g.shape) < p, g, 0.0).astype(g.dtype) for g in planes]


def percolate_sorted(planes, q):
    """Correlated percolation (Sec. VI.B): close the fraction q of all bonds
    with the smallest conductances, so that the closed bonds keep the field's
    correlations.  Ties are broken by position (plane, then index)."""
    flat = np.concatenate([g.ravel() for g in planes])
    k = int(np.floor(q * flat.size))
    closed = np.zeros(flat.size, bool)
    if k > 0:
        closed[np.argsort(flat, kind="stable")[:k]] = True
    out, o = [], 0
    for g in planes:
        c = closed[o:o + g.size].reshape(g.shape)
        out.append(np.where(c, 0.0, g).astype(g.dtype))
        o += g.size
    return out


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def workload_small(variant="random", seed=None):
    """64x64 2D network.  variant: 'random' (g = 10^U(-1,1)), 'uniform' (g=1)
    or 'stratified' (lognormal sigma=1 layers).  Returns (dims, planes, extra)."""
    dims = (64, 64)
    gen = rng(SEED_BASE + 0 if seed is None else seed)
    if variant == "random":
        return dims, loguniform_iid(dims, gen), None
    if variant == "uniform":
        return dims, uniform(dims), None
    if variant == "stratified":
        planes, s = stratified_layers(dims, gen, 1.0)
        return dims, planes, s
    raise ValueError(variant)


def workload_fbm2d(n=2048, variant="isotropic", seed=None, hurst=0.7, sigma=1.5, periodic=()):
    """2D FBM network, H = 0.7, sigma = 1.5 (isotropic), or a stratified
    version (1D FBM along y plus 10 % i.i.d. noise), or stratified without noise.
    periodic=(1,) (isotropic only) adds the wrap bonds of a periodic y axis."""
    dims = (n, n)
    gen = rng(SEED_BASE + 1 if seed is None else seed)
    if variant == "isotropic":
        return dims, fbm_bonds(dims, hurst, sigma, gen, periodic)
    if variant == "stratified":
        return dims, fbm_stratified_bonds(dims, hurst, sigma, gen, noise=0.1)
    if variant == "stratified_exact":
        return dims, fbm_stratified_bonds(dims, hurst, sigma, gen, noise=0.0)
    raise ValueError(variant)


def workload_perc3d(n=256, p=0.26, hurst=0.3, sigma=1.0, seed=None):
    """3D cubic bond percolation, open fraction p, open g = fp32(exp(sigma*B))
    with B a 3D FBM (H = 0.3).  Conductances are float32."""
    dims = (n, n, n)
    gen = rng(SEED_BASE + 2 if seed is None else seed)
    planes = fbm_bonds(dims, hurst, sigma, gen)
    planes = percolate(planes, p, gen)
    return dims, [g.astype(np.float32) for g in planes]


def batch_instance(i, smin=64, smax=1024, p=0.55, sigma=1.0):
    """Instance i of the batched workload: square 2D network of side
    s ~ U{smin..smax}, lognormal(sigma) conductances; even i are percolated at p."""
    gen = rng(SEED_BASE + 1000 * 3 + i)
    s = int(gen.integers(smin, smax + 1))
    dims = (s, s)
    planes = lognormal_iid(dims, gen, sigma)
    if i % 2 == 0:
        planes = percolate(planes, p, gen)
    return dims, planes


def aniso_instance(h_index, ratio_index, r, n=512, sigma=1.0):
    """Realization r of the permeability-anisotropy workload (Sec. VI.B,
    Fig. 10): an n x n network with conductances exp(sigma * B), B an
    anisotropic FBM (Eq. 2) with H = ANISO_H[h_index] and
    beta_x / beta_y = ANISO_RATIOS[ratio_index] (beta_y = 1)."""
    gen = rng(SEED_BASE + 1000 * 5 + 100 * (len(ANISO_RATIOS) * h_index + ratio_index) + r)
    dims = (n, n)
    return dims, fbm_aniso_bonds(dims, ANISO_H[h_index], ANISO_RATIOS[ratio_index], 1.0, sigma, gen)


def aniso_pair_periodic(h_index, ratio_index, r, n=512, sigma=1.0):
    """The same realization as aniso_instance with the paper's boundaries
    (Sec. II: periodic transverse faces), as two networks with the flow along
    x: the field itself with periodic y (gives K_x), and its transpose with
    periodic y (the field's x: gives K_y).  Returns [(dims, planes)] * 2."""
    gen = rng(SEED_BASE + 1000 * 5 + 100 * (len(ANISO_RATIOS) * h_index + ratio_index) + r)
    dims = (n, n)
    B = fbm_field_aniso(node_shape(dims), ANISO_H[h_index], ANISO_RATIOS[ratio_index], 1.0, gen)
    out = []
    for field in (B, np.ascontiguousarray(B.T)):
        out.append((dims, [np.exp(sigma * b) for b in _node_to_bonds(field, dims, (1,))]))
    return out


ANISO_H = (0.75, 0.35)
ANISO_RATIOS = (0.2, 0.5, 1.0, 2.0, 5.0)


def batch_instance_dims(i, smin=64, smax=1024):
    """Shape of batch instance i without drawing its conductances (the first
    draw of the instance's generator, as in batch_instance)."""
    s = int(rng(SEED_BASE + 1000 * 3 + i).integers(smin, smax + 1))
    return (s, s)


def request_instance(i, p2d=0.52, p3d=0.26):
    """Request i of the served stream: 70 % 2D (side 32..1024), 30 % 3D
    (side 16..128); FBM (H in {0.3,0.5,0.7}, sigma=1) or lognormal (sigma=1),
    50/50; 20 % near-critical percolation."""
    gen = rng(SEED_BASE + 1000 * 4 + i)
    if gen.random() < 0.7:
        s = int(gen.integers(32, 1025))
        dims = (s, s)
        pc = p2d
    else:
        s = int(gen.integers(16, 129))
        dims = (s, s, s)
        pc = p3d
    if gen.random() < 0.5:
        h = float(gen.choice([0.3, 0.5, 0.7]))
        planes = fbm_bonds(dims, h, 1.0, gen)
    else:
        planes = lognormal_iid(dims, gen, 1.0)
    if gen.random() < 0.2:
        planes = percolate(planes, pc, gen)
    return dims, planes


def poisson_arrivals(n, rate_hz, seed=SEED_BASE + 4):
    """Arrival times (s) of a Poisson stream with the given mean rate."""
    gen = rng(seed)
    return np.cumsum(gen.exponential(1.0 / rate_hz, size=n))
