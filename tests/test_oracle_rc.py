"""Pins of the oracle's droplet-size histogram by R_c (Fig. 5 caption).

R_c is the radius of a sphere with the cluster's volume.  Checked against a
hand-worked example, an independent cube-root binning on random sizes away
from the edges, and voxelised spheres whose R_c must land in the bin of their
radius.
"""
import math

import numpy as np

import oracle


def test_hand_worked_example():
    # R_c = k * cbrt(3 / (4 pi)) for V = k^3: 0.620, 1.241, 1.861, 6.204
    hist, rc_sum = oracle.rc_histogram([1, 8, 27, 1000], [0.5, 1.0, 2.0, 5.0, 10.0])
    assert hist.tolist() == [0, 1, 2, 0, 1, 0]
    assert math.isclose(rc_sum, 16 * (3 / (4 * math.pi)) ** (1 / 3), rel_tol=1e-12)


def test_random_sizes_match_cube_root_binning():
    rng = np.random.default_rng(9)
    sizes = rng.integers(1, 200000, size=5000)
    edges = np.array([0.8, 1.5, 2.0, 3.3, 5.0, 8.0, 13.0, 21.0, 34.0])
    rc = np.cbrt(3.0 * sizes / (4.0 * np.pi))
    keep = np.all(np.abs(rc[:, None] - edges[None, :]) > 1e-9 * edges[None, :], axis=1)
    sizes, rc = sizes[keep], rc[keep]
    want = np.bincount(np.searchsorted(edges, rc, side="right"), minlength=len(edges) + 1)
    hist, rc_sum = oracle.rc_histogram(sizes, edges)
    np.testing.assert_array_equal(hist, want)
    assert math.isclose(rc_sum, float(rc.sum()), rel_tol=1e-11)
    assert hist.sum() == len(sizes)


def test_voxel_spheres_land_in_their_radius_bin():
    radii = [3.0, 6.0, 9.0, 12.0, 6.0, 3.0]
    L = 96
    centres = np.array([[15.3, 20.1, 18.7], [48.2, 20.6, 22.4], [78.9, 24.3, 30.1],
                        [30.4, 66.2, 62.8], [72.7, 70.5, 70.9], [15.8, 80.2, 80.6]])
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    occ = np.zeros((L, L, L), dtype=bool)
    for (cx, cy, cz), r in zip(centres, radii):
        occ |= (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r
    labels, sizes, hist, n = oracle.label(np.where(occ, 1.0, -1.0).astype(np.float32), (0, 0, 0))
    assert n == len(radii)
    h, _ = oracle.rc_histogram(sizes, [1.5, 4.5, 7.5, 10.5, 13.5])
    assert h.tolist() == [0, 2, 2, 1, 1, 0]
