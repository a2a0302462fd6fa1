"""Pins of the oracle's interior/exterior identification (Sec. 6, steps 3-5).

Checked against what the paper and the definitions fix, independently of the
oracle's code: brute-force BFS components with the votes counted directly
(``brute.interior_tags``), the closed forms of ellipsoidal capsules (one
exterior cluster, one interior cluster per capsule of a directly counted
volume), and consistency with the plain labelling of the far sites.
"""
import itertools

import numpy as np
import pytest

import oracle
from brute import interior_tags
from paper_1405_1931_gb300 import fields

VALUES = np.array([-1.0, -0.7, -0.5, -0.25, 0.0, 0.25, 0.5, np.nan], dtype=np.float32)


def same_interior(got, want):
    assert got[3] == want[3]
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    np.testing.assert_array_equal(got[2], want[2])
    np.testing.assert_array_equal(got[4], want[4])


def test_random_small_fields_match_brute_force():
    rng = np.random.default_rng(17)
    pers = list(itertools.product((0, 1), repeat=3))
    for it in range(160):
        shape = tuple(int(v) for v in rng.integers(1, 6, size=3))
        # mostly far sites and two-sided near sites, some zeros, boundary values and NaN
        p = np.array([0.45, 0.05, 0.05, 0.15, 0.05, 0.15, 0.05, 0.05])
        I = VALUES[rng.choice(len(VALUES), size=shape, p=p)]
        per = pers[it % 8]
        same_interior(oracle.interior(I, per), interior_tags(I, per))


def _F(shape, centre, axes):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return ((x - centre[0]) / axes[0]) ** 2 + ((y - centre[1]) / axes[1]) ** 2 + ((z - centre[2]) / axes[2]) ** 2


@pytest.mark.parametrize("per", [(0, 0, 0), (1, 1, 1), (1, 0, 1)])
def test_single_capsule_closed_form(per):
    shape = (40, 36, 44)
    centre, axes = (21.3, 17.6, 19.2), (15.0, 9.5, 12.0)
    I = fields.capsule_index_field(shape, [(centre, axes)])
    labels, sizes, hist, n, inside = oracle.interior(I, per)
    F = _F(shape, centre, axes)
    inn = F <= 1.0
    pad = np.pad(inn, 1, mode="constant", constant_values=False)
    nb_all_in = np.ones_like(inn)
    nb_any_in = np.zeros_like(inn)
    for a in range(3):
        for d in (-1, 1):
            sh = np.roll(pad, d, axis=a)[1:-1, 1:-1, 1:-1]
            nb_all_in &= sh
            nb_any_in |= sh
    interior = int((inn & nb_all_in).sum())
    exterior = int((~inn & ~nb_any_in).sum())
    assert n == 2
    assert labels.reshape(-1)[0] == 0                     # site 0 is far outside
    assert sorted(sizes.tolist()) == sorted([interior, exterior])
    k_ext = 0                                             # the cluster of site 0 comes first
    assert sizes[k_ext] == exterior and inside[k_ext] == 0
    assert sizes[1] == interior and inside[1] == 1


def test_many_capsules_one_exterior():
    shape = (64, 72, 80)
    caps = fields.capsule_params(7, shape, seed=4)
    assert len(caps) >= 4
    I = fields.capsule_index_field(shape, caps)
    labels, sizes, hist, n, inside = oracle.interior(I, (1, 1, 1))
    assert n == len(caps) + 1
    assert int((inside == 0).sum()) == 1 and int((inside == 1).sum()) == len(caps)
    k_ext = int(np.argmax(sizes))                         # the exterior is the largest cluster
    assert inside[k_ext] == 0 and labels.reshape(-1)[0] == 0 and k_ext == 0


def test_labels_are_those_of_the_far_sites():
    rng = np.random.default_rng(3)
    I = VALUES[rng.integers(0, len(VALUES), size=(9, 11, 13))]
    for per in [(0, 0, 0), (1, 1, 1), (0, 1, 0)]:
        got = oracle.interior(I, per)
        want = oracle.label(np.where(I < -0.5, 1.0, -1.0).astype(np.float32), per)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
        np.testing.assert_array_equal(got[2], want[2])
        assert got[3] == want[3] and len(got[4]) == want[3]
