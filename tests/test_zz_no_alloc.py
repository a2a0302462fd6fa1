"""The allocation-free entry point hk_label_noalloc against hk_label.

hk_label_noalloc serves callers that cannot allocate device memory: its
scratch is a fixed file-scope device array instead of a context workspace.
Its results must equal hk_label's exactly (labels, sizes, histogram and count
are integers), on two calls in a row, since the shared array keeps the
previous call's contents.  This file sorts last so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _outs(shape, cap):
    return (torch.empty(shape, dtype=torch.int32, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"),
            torch.empty(32, dtype=torch.int64, device="cuda"), torch.empty(1, dtype=torch.int64, device="cuda"))


def _call_noalloc(hk, phi, per, outs, cap):
    nz, ny, nx = phi.shape
    labels, sizes, hist, ncl = outs
    return hk.hk_label_noalloc(phi.data_ptr(), nx, ny, nz, per, labels.data_ptr(), sizes.data_ptr(), cap,
                               hist.data_ptr(), ncl.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_hk_label_on_two_calls():
    from paper_1405_1931_gb300 import hk
    lab = hk.Labeller(0)
    cases = [((100, 60, 50), 11, 0.3116, (1, 1, 0)), ((64, 64, 64), 12, 0.45, (1, 1, 1))]
    for (nx, ny, nz), seed, p, per in cases:
        phi = torch.from_numpy(fields.iid_field(nx, ny, nz, seed=seed, occupancy=p)).cuda()
        cap = (phi.numel() + 1) // 2
        ref = lab.alloc_outputs(phi.shape, phi.device)
        lab.label(phi, per, out=ref)
        got = _outs(phi.shape, cap)
        got[0].fill_(-7)
        assert _call_noalloc(hk, phi, per, got, cap) == hk.HK_OK
        torch.cuda.synchronize()
        n = int(ref[3].item())
        assert int(got[3].item()) == n
        assert torch.equal(got[0], ref[0])
        assert torch.equal(got[1][:n], ref[1][:n])
        assert torch.equal(got[2], ref[2])
    lab.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_1405_1931_gb300 import hk
    per = (ctypes.c_int * 3)(1, 1, 1)
    # a 512^3 lattice needs far more than the fixed scratch; rejected on the host, nothing is touched
    rc = hk.load().hk_label_noalloc(ctypes.c_void_p(16), 512, 512, 512, per, ctypes.c_void_p(16), None, 0,
                                    None, None, None)
    assert rc == hk.HK_ERR_TOO_LARGE
