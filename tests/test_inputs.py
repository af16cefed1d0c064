"""Checks of the seeded input generator (geometry, boundary data, targets)."""
import math

import numpy as np
import pytest
import scipy.special

import stokes_inputs as si


def test_ellipse_perimeter_matches_elliptic_integral():
    # p = 2 superellipse is an ellipse; its perimeter is 4 a E(1 - b^2/a^2).
    a, b = 1.3, 0.6
    c = si.superellipse_curve(a, b, 256, p=2)
    L = 4 * a * scipy.special.ellipe(1 - (b / a) ** 2)
    assert abs(c.weights.sum() - L) < 1e-13 * L
    # equispaced arclength h: each chord is 2 sin(k h / 2) / k ~ h (1 - k^2 h^2 / 24)
    h = L / 256
    d = np.linalg.norm(np.diff(np.vstack([c.nodes, c.nodes[:1]]), axis=0), axis=1)
    kmax = a / b**2
    assert np.all(d <= h + 1e-15) and np.all(h - d <= h**3 * kmax**2 / 24 * 1.01)


def test_superellipse_orientation_normals_curvature():
    c = si.superellipse_curve(4.0, 1.0, 512)
    assert np.allclose(np.linalg.norm(c.normals, axis=1), 1.0, atol=1e-14)
    # on the implicit curve
    assert np.abs(si.superellipse_inside(c.nodes, 4.0, 1.0) - 1.0).max() < 1e-12
    # outward: n . x > 0 for a star-shaped convex curve centred at 0
    assert (np.einsum("ij,ij->i", c.normals, c.nodes) > 0).all()
    # counter-clockwise: positive signed area
    x, y = c.nodes[:, 0], c.nodes[:, 1]
    assert 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) > 0
    assert (c.curvature >= -1e-12).all()
    # curvature at (a, 0) of |x/a|^8 + |y/b|^8 = 1 vanishes (flat end), at (0, b) too
    assert abs(c.curvature[0]) < 1e-8
    # Gauss-Bonnet: total turning of a closed convex curve is 2 pi
    assert abs((c.curvature * c.weights).sum() - 2 * math.pi) < 1e-10


def test_circle_pore_conventions():
    c = si.circle_curve((0.5, -0.2), 0.15, 64)
    d = c.nodes - np.array([0.5, -0.2])
    assert np.allclose(np.linalg.norm(d, axis=1), 0.15)
    assert np.allclose(c.normals, -d / 0.15)          # into the pore
    x, y = d[:, 0], d[:, 1]
    assert 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) < 0   # clockwise
    assert np.allclose(c.curvature, -1 / 0.15)
    assert abs(c.weights.sum() - 2 * math.pi * 0.15) < 1e-15


def test_pipe10_shape_and_gaps(pipe10_geom):
    g = pipe10_geom
    assert g.n_nodes == 1152 and g.n_pores == 10 and g.outer_comp == 10
    assert list(np.diff(g.offsets)) == [64] * 10 + [512]
    pc, pr = g.centres[:10], g.radii[:10]
    assert (pr >= 0.1).all() and (pr <= 0.2).all()
    assert (np.abs(pc[:, 0]) < 3.2).all() and (np.abs(pc[:, 1]) < 0.6).all()
    d = np.linalg.norm(pc[:, None] - pc[None], axis=2) - pr[:, None] - pr[None]
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 0.05
    wall = g.nodes[g.comp_slice(10)]
    assert (np.linalg.norm(pc[:, None] - wall[None], axis=2) - pr[:, None]).min() >= 0.05 - 1e-3


def test_pipe_data_compatible(pipe10_geom):
    f = si.pipe_bc(pipe10_geom)
    flux = (pipe10_geom.weights[:, None] * f * pipe10_geom.normals).sum()
    assert abs(flux) < 1e-13
    assert np.all(f[: pipe10_geom.offsets[-2]] == 0)


def test_targets_clear_of_boundary(pipe10_geom):
    T = si.interior_targets(pipe10_geom, 500, min_dist=0.05, seed=3)
    assert T.shape == (500, 2)
    d = np.linalg.norm(T[:, None] - pipe10_geom.nodes[None], axis=2).min(1)
    assert d.min() >= 0.05 - 1e-9
    assert (si.superellipse_inside(T, 4.0, 1.0) < 1).all()


def test_generator_deterministic():
    a = si.pipe10_geometry(5, n_outer=128, n_pores=3, n_per_pore=16)
    b = si.pipe10_geometry(5, n_outer=128, n_pores=3, n_per_pore=16)
    assert np.array_equal(a.nodes, b.nodes)


@pytest.mark.parametrize("index", [0, 7])
def test_scaled_down_batch_geometry(index):
    """The uneven batch's geometries: pore counts in [20, 120], 64 or 128
    nodes per pore, 1024 or 2048 wall nodes, gaps >= 0.05 between pores and
    to the wall, pipe data compatible, node counts divisible by 8 (the
    two-grid coarsening of the batch benchmark)."""
    g = si.batch_small_geometry(index)
    M = g.n_pores
    assert 20 <= M <= 120 and g.outer_comp == M
    sizes = np.diff(g.offsets)
    assert len(set(sizes[:M])) == 1 and sizes[0] in (64, 128) and sizes[M] in (1024, 2048)
    assert all(n % 8 == 0 for n in sizes)
    pc, pr = g.centres[:M], g.radii[:M]
    d = np.linalg.norm(pc[:, None] - pc[None], axis=2) - pr[:, None] - pr[None]
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 0.05
    wall = g.nodes[g.comp_slice(M)]
    assert (np.linalg.norm(pc[:, None] - wall[None], axis=2) - pr[:, None]).min() >= 0.05 - 2e-3
    f = si.pipe_bc(g)
    assert abs((g.weights[:, None] * f * g.normals).sum()) < 1e-12
