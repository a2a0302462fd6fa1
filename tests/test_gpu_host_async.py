"""Parity of the asynchronous host-buffer entry (hk_label_host_async) with the oracle.

Fields live in page-locked host tensors; the call enqueues the copy in, the
labelling, the copies out and the device-sized copy of the sizes, and returns.
Results are compared element by element after the stream has passed the call.
"""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pinned_io(shape, cap):
    phi = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    labels = torch.empty(shape, dtype=torch.int32, pin_memory=True)
    sizes = torch.full((max(cap, 1),), -7, dtype=torch.int64, pin_memory=True)
    hist = torch.empty(32, dtype=torch.int64, pin_memory=True)
    ncl = torch.empty(1, dtype=torch.int64, pin_memory=True)
    return phi, labels, sizes, hist, ncl


@pytest.fixture(scope="module")
def labellers():
    from paper_1405_1931_gb300.hk import Labeller
    labs = [Labeller(0), Labeller(0)]
    yield labs
    for lab in labs:
        lab.close()


def test_async_matches_oracle(labellers):
    """100 x 60 x 50 (ragged tiles along x and z), p_c, periodic x and z."""
    phi_np = fields.iid_field(100, 60, 50, seed=4, occupancy=0.3116)
    want = oracle.label(phi_np, (1, 0, 1))
    n = phi_np.size
    phi, labels, sizes, hist, ncl = _pinned_io(phi_np.shape, (n + 1) // 2)
    phi.copy_(torch.from_numpy(phi_np))
    st = torch.cuda.Stream()
    labellers[0].label_host_async(phi, labels, sizes, hist, ncl, (1, 0, 1), stream=st)
    st.synchronize()
    labellers[0].sync_status()
    k = int(ncl[0])
    assert k == want[3]
    np.testing.assert_array_equal(labels.numpy(), want[0])
    np.testing.assert_array_equal(sizes[:k].numpy(), want[1])
    assert (sizes[k:].numpy() == -7).all()          # nothing written past the count
    np.testing.assert_array_equal(hist.numpy(), want[2])


def test_async_truncates_sizes_at_capacity(labellers):
    """sizes_cap below the count: the first sizes_cap sizes, no error, full labels."""
    phi_np = fields.iid_field(48, 40, 36, seed=11, occupancy=0.25)
    want = oracle.label(phi_np, (1, 1, 1))
    cap = 5
    assert want[3] > cap
    phi, labels, sizes, hist, ncl = _pinned_io(phi_np.shape, cap)
    phi.copy_(torch.from_numpy(phi_np))
    st = torch.cuda.Stream()
    labellers[0].label_host_async(phi, labels, sizes, hist, ncl, (1, 1, 1), stream=st)
    st.synchronize()
    assert int(ncl[0]) == want[3]
    np.testing.assert_array_equal(sizes.numpy(), want[1][:cap])
    np.testing.assert_array_equal(labels.numpy(), want[0])
    np.testing.assert_array_equal(hist.numpy(), want[2])


def test_async_rejects_pageable_buffers(labellers):
    """A pageable host buffer is an argument error, found before anything is enqueued."""
    from paper_1405_1931_gb300 import hk
    phi_np = np.ascontiguousarray(fields.iid_field(16, 16, 16, seed=1, occupancy=0.3))
    lab_np = np.empty(phi_np.shape, np.int32)
    phi, labels, sizes, hist, ncl = _pinned_io(phi_np.shape, 2048)
    rc = hk.hk_label_host_async(labellers[0].ctx, phi_np.ctypes.data, 16, 16, 16, (1, 1, 1), labels.data_ptr(),
                                sizes.data_ptr(), 2048, hist.data_ptr(), ncl.data_ptr(), 0)
    assert rc == hk.HK_ERR_ARG
    rc = hk.hk_label_host_async(labellers[0].ctx, phi.data_ptr(), 16, 16, 16, (1, 1, 1), lab_np.ctypes.data,
                                sizes.data_ptr(), 2048, hist.data_ptr(), ncl.data_ptr(), 0)
    assert rc == hk.HK_ERR_ARG


def test_two_contexts_pipelined(labellers):
    """Six fields of uneven shapes through two contexts on two streams, issued
    back to back (one field's copy in overlaps the other's copy out); each result
    equals the oracle's."""
    shapes = [(64, 40, 33), (97, 31, 20), (32, 32, 32), (70, 45, 33), (40, 64, 17), (33, 33, 65)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pending = []
    for i, (nx, ny, nz) in enumerate(shapes):
        phi_np = fields.iid_field(nx, ny, nz, seed=20 + i, occupancy=0.3116)
        per = ((i & 1), 1, (i >> 1) & 1)
        io = _pinned_io(phi_np.shape, (phi_np.size + 1) // 2)
        io[0].copy_(torch.from_numpy(phi_np))
        j = i % 2
        labellers[j].label_host_async(*io, per, stream=streams[j])
        pending.append((phi_np, per, io))
    for st in streams:
        st.synchronize()
    for phi_np, per, (_, labels, sizes, hist, ncl) in pending:
        want = oracle.label(phi_np, per)
        k = int(ncl[0])
        assert k == want[3]
        np.testing.assert_array_equal(labels.numpy(), want[0])
        np.testing.assert_array_equal(sizes[:k].numpy(), want[1])
        np.testing.assert_array_equal(hist.numpy(), want[2])
