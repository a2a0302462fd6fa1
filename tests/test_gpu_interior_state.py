"""Parity of the per-site interior state and its incremental updates (Sec. 6) with the oracle.

hk_interior_state, hk_interior_update (dense, in place and out of place, the 16-site
vector path and the unaligned scalar path) and hk_interior_update_sites (a list of
near sites) are compared element by element with oracle.interior_state and
oracle.interior_update on the same index fields.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VALUES = np.array([-1.0, -0.5, -0.25, 0.0, 0.25, 0.5, np.nan], dtype=np.float32)


@pytest.fixture(scope="module")
def labeller():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    yield lab
    lab.close()


def moved(caps, d):
    return [((c[0] + d[0], c[1] + d[1], c[2] + d[2]), a) for c, a in caps]


def test_state_random_fields(labeller):
    rng = np.random.default_rng(8)
    for it, per in enumerate(itertools.product((0, 1), repeat=3)):
        for shape in [(7, 9, 40), (33, 17, 5), (16, 16, 64)]:
            I = VALUES[rng.choice(len(VALUES), size=shape, p=[0.55, 0.03, 0.17, 0.05, 0.12, 0.03, 0.05])]
            got = labeller.interior_state(torch.from_numpy(I).cuda(), per)
            np.testing.assert_array_equal(got.cpu().numpy(), oracle.interior_state(I, per), err_msg=f"{shape} {per}")


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_state_capsules(labeller, tile):
    shape = (70, 45, 66)
    caps = fields.capsule_params(4, shape, seed=3, a_lo=5.0, a_hi=12.0)
    I = fields.capsule_index_field(shape, caps)
    labeller.set_tile(*tile)
    try:
        for per in [(1, 1, 1), (0, 1, 0)]:
            got = labeller.interior_state(torch.from_numpy(I).cuda(), per)
            np.testing.assert_array_equal(got.cpu().numpy(), oracle.interior_state(I, per))
    finally:
        labeller.set_tile(16, 16)


def test_state_capsules_256(labeller):
    """The bench workload: 256^3, 24 capsules."""
    shape = (256, 256, 256)
    caps = fields.capsule_params(24, shape, seed=12, a_lo=8.0, a_hi=30.0)
    I = fields.capsule_index_field(shape, caps)
    got = labeller.interior_state(torch.from_numpy(I).cuda(), (1, 1, 1))
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.interior_state(I, (1, 1, 1)))


def test_updates_follow_moving_capsules(labeller):
    """Ten steps of capsules moving under half a lattice constant: the dense update in
    place, the dense update out of place on unaligned views (scalar path) and the
    sparse update from the list of near sites all equal the oracle's update chain."""
    from paper_1405_1931_gb300 import hk
    shape = (40, 44, 48)
    caps = fields.capsule_params(3, shape, seed=2, a_lo=5.0, a_hi=10.0)
    rng = np.random.default_rng(77)
    I = fields.capsule_index_field(shape, caps)
    want = oracle.interior_state(I)
    s_dense = labeller.interior_state(torch.from_numpy(I).cuda())
    s_sparse = s_dense.clone()
    n = I.size
    buf_prev = torch.empty(n + 1, dtype=torch.int8, device="cuda")
    buf_out = torch.empty(n + 1, dtype=torch.int8, device="cuda")
    buf_idx = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    s_odd = s_dense.clone().reshape(-1)
    for _ in range(10):
        caps = moved(caps, rng.uniform(-0.25, 0.25, size=3))
        I = fields.capsule_index_field(shape, caps)
        want = oracle.interior_update(want, I)
        d = torch.from_numpy(I).cuda()
        hk.interior_update(s_dense, d)                       # in place, 16-site vectors
        prev_v, out_v, idx_v = buf_prev[1:], buf_out[1:], buf_idx[1:]   # 1-byte / 4-byte offsets
        prev_v.copy_(s_odd)
        idx_v.copy_(d.reshape(-1))
        hk.interior_update(prev_v, idx_v, out=out_v)
        s_odd = out_v.clone()
        near = ~(I < -0.5)
        sites = torch.from_numpy(np.flatnonzero(near).astype(np.int32)).cuda()
        vals = torch.from_numpy(I.reshape(-1)[near.reshape(-1)]).cuda()
        hk.interior_update_sites(s_sparse, sites, vals)
        np.testing.assert_array_equal(s_dense.cpu().numpy(), want)
        np.testing.assert_array_equal(s_odd.cpu().numpy().reshape(shape), want)
        np.testing.assert_array_equal(s_sparse.cpu().numpy(), want)
    np.testing.assert_array_equal(s_dense.cpu().numpy(), oracle.interior_state(I))


def test_update_odd_lengths_and_skipped_entries(labeller):
    """Lengths that are not multiples of 16 (vector body plus scalar tail), random
    states and values; the sparse form skips far values and sites out of range."""
    from paper_1405_1931_gb300 import hk
    rng = np.random.default_rng(9)
    for n in [1, 15, 16, 17, 1000, 4099]:
        st = rng.integers(-1, 2, size=n).astype(np.int8).reshape(1, 1, n)
        I = VALUES[rng.choice(len(VALUES), size=n)].reshape(1, 1, n)
        got = hk.interior_update(torch.from_numpy(st).cuda(), torch.from_numpy(I).cuda(),
                                 out=torch.empty((1, 1, n), dtype=torch.int8, device="cuda"))
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.interior_update(st, I))
    st = torch.zeros(10, dtype=torch.int8, device="cuda")
    sites = torch.tensor([0, 3, -1, 10, 5, 7], dtype=torch.int32, device="cuda")
    vals = torch.tensor([-0.25, 0.25, -0.25, -0.25, -1.0, 0.0], dtype=torch.float32, device="cuda")
    st[3] = 1
    st[5] = -1
    hk.interior_update_sites(st, sites, vals)
    assert st.cpu().tolist() == [1, 0, 0, 0, 0, -1, 0, 0, 0, 0]
