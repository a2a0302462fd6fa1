"""Parity of the interior/exterior identification (Sec. 6, steps 3-5) with the oracle.

hk_label_interior through the C ABI against oracle.interior on the same index
bytes: labels, sizes, histogram, count and the per-cluster tags must be
identical.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILES = [(8, 8), (16, 8), (16, 16), (32, 8)]
VALUES = np.array([-1.0, -0.7, -0.5, -0.25, 0.0, 0.25, 0.5, np.nan], dtype=np.float32)


@pytest.fixture(scope="module")
def labeller():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    yield lab
    lab.close()


def assert_interior_parity(lab, I, per, what=""):
    want = oracle.interior(I, per)
    d = torch.from_numpy(np.ascontiguousarray(I)).cuda()
    labels, sizes, hist, ncl, inside = lab.label_interior(d, per)
    lab.sync_status()
    n = int(ncl.item())
    assert n == want[3], f"{what}: n_clusters {n} != {want[3]}"
    np.testing.assert_array_equal(labels.cpu().numpy(), want[0], err_msg=f"{what}: labels")
    np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1], err_msg=f"{what}: sizes")
    np.testing.assert_array_equal(hist.cpu().numpy(), want[2], err_msg=f"{what}: hist")
    np.testing.assert_array_equal(inside[:n].cpu().numpy(), want[4], err_msg=f"{what}: inside")


def test_random_fields_all_periodic_sets(labeller):
    rng = np.random.default_rng(23)
    p = np.array([0.45, 0.05, 0.05, 0.15, 0.05, 0.15, 0.05, 0.05])
    for shape in [(1, 1, 1), (3, 5, 7), (17, 9, 33), (20, 40, 70), (33, 17, 65)]:
        I = VALUES[rng.choice(len(VALUES), size=shape, p=p)]
        for per in itertools.product((0, 1), repeat=3):
            assert_interior_parity(labeller, I, per, f"random {shape} {per}")


def test_capsules_every_tile_shape(labeller):
    shape = (70, 81, 97)
    caps = fields.capsule_params(9, shape, seed=8)
    I = fields.capsule_index_field(shape, caps)
    for tile in TILES:
        labeller.set_tile(*tile)
        for per in [(1, 1, 1), (0, 0, 0)]:
            assert_interior_parity(labeller, I, per, f"capsules tile {tile} {per}")
    labeller.set_tile(16, 16)


def test_capsules_256(labeller):
    shape = (256, 256, 256)
    caps = fields.capsule_params(24, shape, seed=12, a_lo=8.0, a_hi=30.0)
    I = fields.capsule_index_field(shape, caps)
    assert_interior_parity(labeller, I, (1, 1, 1), "capsules 256^3")


def test_plain_labelling_unchanged_after_interior(labeller):
    """An index-field call leaves the context's plain labelling (phi > 0) untouched."""
    rng = np.random.default_rng(2)
    phi = (rng.random((40, 48, 64)) - 0.6).astype(np.float32)
    d = torch.from_numpy(phi).cuda()
    I = VALUES[rng.integers(0, len(VALUES), size=(40, 48, 64))]
    labeller.label_interior(torch.from_numpy(I).cuda(), (1, 1, 1))
    labels, sizes, hist, ncl = labeller.label(d, (1, 0, 1))
    want = oracle.label(phi, (1, 0, 1))
    assert int(ncl.item()) == want[3]
    np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
