"""Pins of the oracle's per-site interior state and its incremental update (Sec. 6).

- brute force: on random small index fields the state equals the one built from BFS
  clusters and their face votes (``brute.interior_state``);
- closed form: for closed ellipsoidal membranes the state of every site is 1 exactly
  where the site lies inside an ellipsoid (F <= 1) and 0 elsewhere;
- the update (last paragraph of Sec. 6): along trajectories of capsules moving by
  under half a lattice constant per step, updating only the near sites keeps the state
  equal to that closed form (and to a full recomputation); after a jump of several
  lattice constants it does not, so the test can fail;
- the three kinds of site of the update rule, by hand.
"""
import itertools

import numpy as np
import pytest

import oracle
from brute import interior_state as brute_state
from paper_1405_1931_gb300 import fields

PERS = list(itertools.product((0, 1), repeat=3))
VALUES = np.array([-1.0, -0.5, -0.25, 0.0, 0.25, 0.5, np.nan], dtype=np.float32)


def inside_indicator(shape, caps):
    """1 where a site lies inside one of the ellipsoids (F <= 1, F summed z, y, x in float64)."""
    nz, ny, nx = shape
    z, y, x = (np.arange(n, dtype=np.float64) for n in (nz, ny, nx))
    ind = np.zeros(shape, dtype=bool)
    for (cx, cy, cz), (ax, ay, az) in caps:
        F = (((z - cz) / az) ** 2)[:, None, None] + (((y - cy) / ay) ** 2)[None, :, None] \
            + (((x - cx) / ax) ** 2)[None, None, :]
        ind |= F <= 1.0
    return ind.astype(np.int8)


def moved(caps, d):
    return [((c[0] + d[0], c[1] + d[1], c[2] + d[2]), a) for c, a in caps]


def test_state_matches_brute_force():
    rng = np.random.default_rng(31)
    for it in range(60):
        shape = tuple(int(v) for v in rng.integers(1, 7, size=3))
        I = VALUES[rng.choice(len(VALUES), size=shape, p=[0.45, 0.05, 0.2, 0.05, 0.15, 0.05, 0.05])]
        per = PERS[it % 8]
        np.testing.assert_array_equal(oracle.interior_state(I, per), brute_state(I, per))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_state_of_capsules_is_their_inside(seed):
    shape = (40, 44, 48)
    caps = fields.capsule_params(3, shape, seed=seed, a_lo=5.0, a_hi=10.0)
    I = fields.capsule_index_field(shape, caps)
    for per in [(1, 1, 1), (0, 0, 0)]:
        np.testing.assert_array_equal(oracle.interior_state(I, per), inside_indicator(shape, caps))


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_update_follows_slowly_moving_capsules(seed):
    shape = (40, 44, 48)
    caps = fields.capsule_params(3, shape, seed=seed, a_lo=5.0, a_hi=10.0)
    rng = np.random.default_rng(100 + seed)
    I = fields.capsule_index_field(shape, caps)
    state = oracle.interior_state(I)
    for _ in range(10):
        caps = moved(caps, rng.uniform(-0.25, 0.25, size=3))      # |d| < 0.44 lattice constants
        I = fields.capsule_index_field(shape, caps)
        state = oracle.interior_update(state, I)
        np.testing.assert_array_equal(state, inside_indicator(shape, caps))
    np.testing.assert_array_equal(state, oracle.interior_state(I))


def test_update_fails_after_a_jump():
    """The premise matters: after moving 2.6 lattice constants at once, sites that the
    membrane swept over without leaving them near it keep a stale state."""
    shape = (40, 44, 48)
    caps = fields.capsule_params(3, shape, seed=0, a_lo=5.0, a_hi=10.0)
    state = oracle.interior_state(fields.capsule_index_field(shape, caps))
    caps = moved(caps, (2.6, 0.0, 0.0))
    I = fields.capsule_index_field(shape, caps)
    assert (oracle.interior_update(state, I) != inside_indicator(shape, caps)).sum() > 100


def test_update_rule_by_hand():
    state = np.array([1, 0, -1, 1, 0, 1, 0], dtype=np.int8).reshape(1, 1, 7)
    index = np.array([-1.0, -1.0, -1.0, 0.25, -0.25, 0.0, np.nan], dtype=np.float32).reshape(1, 1, 7)
    # far sites keep their state (1, 0, -1); near sites take their side: +0.25 -> 0,
    # -0.25 -> 1, 0 -> 0, NaN -> 0
    assert oracle.interior_update(state, index).reshape(-1).tolist() == [1, 0, -1, 0, 1, 0, 0]


@pytest.mark.parametrize("seed", [0, 5])
def test_capsule_generator_layers_from_their_definition(seed):
    """The input generator (evaluated on bounding boxes) puts the inner layer exactly on
    the inside sites with an outside 6-neighbour and the outer layer on the outside
    sites with an inside 6-neighbour, judged on the whole grid."""
    shape = (60, 52, 70)
    caps = fields.capsule_params(6, shape, seed=seed, a_lo=4.0, a_hi=14.0)
    I = fields.capsule_index_field(shape, caps)
    ind = inside_indicator(shape, caps).astype(bool)
    pad = np.pad(ind, 1, mode="constant", constant_values=False)
    nb_out = np.zeros(shape, dtype=bool)
    nb_in = np.zeros(shape, dtype=bool)
    for axis in range(3):
        for d in (-1, 1):
            sl = [slice(1, -1)] * 3
            sl[axis] = slice(1 + d, pad.shape[axis] - 1 + d)
            nb_in |= pad[tuple(sl)]
            nb_out |= ~pad[tuple(sl)]
    want = np.full(shape, fields.INDEX_FAR, dtype=np.float32)
    want[~ind & nb_in] = fields.INDEX_OUTER
    want[ind & nb_out] = fields.INDEX_INNER
    np.testing.assert_array_equal(I, want)
