"""Pins of the oracle's ESDF collision checking (voxelisation, signed Euclidean
distance transform, trilinear read) against closed forms and bounds that do
not come from the oracle itself:
  * one occupied voxel: the field is the voxel size times the Euclidean
    distance in voxel units, and -voxel inside;
  * a half-space of occupied voxels: an affine profile along its normal;
  * empty and full grids: plus / minus the grid diagonal;
  * a box whose faces lie on voxel boundaries and a sphere: the voxel sets
    follow from the geometry;
  * the trilinear read reproduces affine fields exactly and clamps outside;
  * the field of a voxelised sphere obstacle is within the discretisation
    bound of the obstacle's true signed distance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H


def test_single_occupied_voxel():
    dims = (7, 6, 5)
    occ = np.zeros((5, 6, 7), np.uint8)
    occ[2, 3, 4] = 1  # k, j, i
    h = 0.05
    f = O.esdf(occ, dims, h)
    k, j, i = np.meshgrid(np.arange(5), np.arange(6), np.arange(7), indexing="ij")
    want = h * np.sqrt((i - 4) ** 2 + (j - 3) ** 2 + (k - 2) ** 2)
    want[2, 3, 4] = -h
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)


def test_half_space():
    dims = (9, 4, 3)
    occ = np.zeros((3, 4, 9), np.uint8)
    occ[:, :, :4] = 1  # i < 4 occupied
    h = 0.1
    f = O.esdf(occ, dims, h)
    for i in range(9):
        want = (i - 4 + 1) * h if i >= 4 else -(4 - i) * h
        np.testing.assert_allclose(f[:, :, i], want, atol=1e-15)


def test_empty_and_full_grids():
    dims = (4, 5, 6)
    h = 0.2
    diag = h * np.sqrt(16 + 25 + 36)
    np.testing.assert_allclose(O.esdf(np.zeros((6, 5, 4), np.uint8), dims, h), diag)
    np.testing.assert_allclose(O.esdf(np.ones((6, 5, 4), np.uint8), dims, h), -diag)


def test_two_sites_field_is_the_minimum_of_single_site_fields():
    dims = (8, 8, 8)
    a = np.zeros((8, 8, 8), np.uint8)
    b = np.zeros((8, 8, 8), np.uint8)
    a[1, 2, 3] = 1
    b[6, 5, 1] = 1
    fa, fb, fab = O.esdf(a, dims, 1.0), O.esdf(b, dims, 1.0), O.esdf(a | b, dims, 1.0)
    free = (a | b) == 0
    np.testing.assert_array_equal(fab[free], np.minimum(fa, fb)[free])


def test_voxelize_aligned_box_and_sphere():
    h = 0.1
    origin = (-0.4, -0.4, 0.0)
    dims = (8, 8, 8)
    # box covering x in [-0.2, 0.1], y in [0.0, 0.3], z in [0.1, 0.5]: faces on voxel boundaries
    box = H.aabb([-0.05, 0.15, 0.3], [0.15, 0.15, 0.2])
    occ = O.voxelize(H.scene(boxes=[box]), origin, h, dims)
    want = np.zeros((8, 8, 8), np.uint8)
    want[1:5, 4:7, 2:5] = 1  # k in [1, 5), j in [4, 7), i in [2, 5)
    np.testing.assert_array_equal(occ, want)
    # sphere: centre (0.03, -0.02, 0.41), radius 0.17
    c, r = np.array([0.03, -0.02, 0.41]), 0.17
    occ = O.voxelize(H.scene(spheres=[[*c, r]]), origin, h, dims)
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    centres = np.stack([origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h, origin[2] + (k + 0.5) * h], -1)
    np.testing.assert_array_equal(occ, (np.linalg.norm(centres - c, axis=-1) < r).astype(np.uint8))


def test_trilinear_reproduces_affine_fields_and_clamps():
    dims = (5, 4, 6)
    h = 0.25
    origin = np.array([0.1, -0.3, 0.2])
    g = np.array([0.7, -1.3, 2.1])
    k, j, i = np.meshgrid(np.arange(6), np.arange(4), np.arange(5), indexing="ij")
    centres = np.stack([origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h, origin[2] + (k + 0.5) * h], -1)
    vals = centres @ g + 0.4
    rng = np.random.default_rng(0)
    lo = origin + 0.5 * h
    hi = origin + (np.array(dims) - 0.5) * h
    for _ in range(200):
        p = lo + rng.random(3) * (hi - lo)
        assert abs(O.esdf_query(vals, origin, h, dims, p) - (p @ g + 0.4)) < 1e-12
    # voxel centres return the stored value
    for (kk, jj, ii) in [(0, 0, 0), (5, 3, 4), (2, 1, 3)]:
        assert abs(O.esdf_query(vals, origin, h, dims, centres[kk, jj, ii]) - vals[kk, jj, ii]) < 1e-12
    # outside: clamped to the boundary centres along each axis
    p = np.array([hi[0] + 3.0, lo[1] - 2.0, 0.5 * (lo[2] + hi[2])])
    q = np.array([hi[0], lo[1], p[2]])
    assert abs(O.esdf_query(vals, origin, h, dims, p) - (q @ g + 0.4)) < 1e-12


def test_field_approximates_true_distance_of_a_sphere():
    h = 0.04
    origin = (-0.64, -0.64, -0.64)
    dims = (32, 32, 32)
    c, r = np.array([0.013, -0.021, 0.037]), 0.31
    sc = H.scene(spheres=[[*c, r]])
    occ = O.voxelize(sc, origin, h, dims)
    f = O.esdf(occ, dims, h)
    rng = np.random.default_rng(3)
    for _ in range(300):
        p = rng.uniform(-0.55, 0.55, 3)
        true = np.linalg.norm(p - c) - r
        got = O.esdf_query(f, origin, h, dims, p)
        # sites are voxel centres inside the sphere (within h*sqrt(3)/2 of its
        # surface), interpolation adds at most one voxel diagonal
        assert abs(got - true) <= 2.0 * h * np.sqrt(3), (p, got, true)


def test_clearance_uses_the_field():
    rb = H.robot([W.JOINT_PRISM_X], [0.0], bases=[[0.0, 0.0, 0.0]], lower=[-1.0], upper=[1.0],
                 spheres=[(0, (0.0, 0.0, 0.0), 0.05)], name="slider")
    dims = (16, 16, 16)
    h = 0.05
    origin = (-0.4, -0.4, -0.4)
    occ = np.zeros((16, 16, 16), np.uint8)
    occ[:, :, 12:] = 1  # occupied for x >= origin + 12 h = 0.2
    f = O.esdf(occ, dims, h)
    empty = H.empty_scene()
    for x in (-0.3, 0.0, 0.05, 0.1, 0.3):
        cl, ce, cs = O.clearance(rb, empty, [x], esdf=(f, origin, h, dims))
        want = O.esdf_query(f, origin, h, dims, [x, 0.0, 0.0]) - 0.05
        assert abs(cl - want) < 1e-12
    free, _ = O.check_states(rb, empty, np.array([[-0.2], [0.25]]), esdf=(f, origin, h, dims))
    assert free.tolist() == [True, False]
