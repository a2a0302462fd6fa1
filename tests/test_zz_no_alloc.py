"""The allocation-free entry point hk_label_noalloc against hk_label.

hk_label_noalloc serves callers that cannot allocate device memory: its
scratch is a fixed file-scope device array instead of a context workspace.
Its results must equal hk_label's exactly (labels, sizes, histogram and count
are integers), on several calls in a row, since the shared array keeps the
previous call's contents; after each call the array's status word, read with
hk_noalloc_sync_status, must be clear.  The array's documented limit is
exercised at both ends: 256^3 fits, 264^3 is rejected on the host.  This file
sorts last so a run that stops at the first failure has already run every
other test.
"""
import ctypes

import pytest

from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _outs(shape, cap):
    return (torch.empty(shape, dtype=torch.int32, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"),
            torch.empty(32, dtype=torch.int64, device="cuda"), torch.empty(1, dtype=torch.int64, device="cuda"))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call_noalloc(hk, phi, per, outs, cap):
    nz, ny, nx = phi.shape
    labels, sizes, hist, ncl = outs
    return hk.hk_label_noalloc(phi.data_ptr(), nx, ny, nz, per, labels.data_ptr(), sizes.data_ptr(), cap,
                               hist.data_ptr(), ncl.data_ptr(), _stream())


CASES = [((100, 60, 50), 11, 0.3116, (1, 1, 0)), ((64, 64, 64), 12, 0.45, (1, 1, 1)),
         ((256, 256, 256), 13, 0.3116, (1, 1, 1)), ((37, 250, 19), 14, 0.6, (0, 1, 1))]


def test_noalloc_matches_hk_label_on_consecutive_calls():
    from paper_1405_1931_gb300 import hk
    lab = hk.Labeller(0)
    for (nx, ny, nz), seed, p, per in CASES:
        phi = torch.from_numpy(fields.iid_field(nx, ny, nz, seed=seed, occupancy=p)).cuda()
        cap = (phi.numel() + 1) // 2
        ref = lab.alloc_outputs(phi.shape, phi.device)
        lab.label(phi, per, out=ref)
        lab.sync_status()
        got = _outs(phi.shape, cap)
        got[0].fill_(-7)
        assert _call_noalloc(hk, phi, per, got, cap) == hk.HK_OK
        assert hk.hk_noalloc_sync_status(_stream()) == hk.HK_OK
        n = int(ref[3].item())
        assert int(got[3].item()) == n
        assert torch.equal(got[0], ref[0])
        assert torch.equal(got[1][:n], ref[1][:n])
        assert torch.equal(got[2], ref[2])
    lab.close()


def test_noalloc_capacity_path_reads_the_status():
    """A sizes_cap below ceil(N/2) makes the call wait for the count; it then reports
    HK_ERR_CAPACITY only when the count exceeds the cap, and the status word is clear."""
    from paper_1405_1931_gb300 import hk
    phi = torch.from_numpy(fields.iid_field(48, 40, 36, seed=15, occupancy=0.3116)).cuda()
    full = _outs(phi.shape, (phi.numel() + 1) // 2)
    assert _call_noalloc(hk, phi, (1, 1, 1), full, (phi.numel() + 1) // 2) == hk.HK_OK
    n = int(full[3].item())
    exact = _outs(phi.shape, n)
    assert _call_noalloc(hk, phi, (1, 1, 1), exact, n) == hk.HK_OK
    assert torch.equal(exact[1][:n], full[1][:n])
    short = _outs(phi.shape, n - 1)
    assert _call_noalloc(hk, phi, (1, 1, 1), short, n - 1) == hk.HK_ERR_CAPACITY
    assert int(short[3].item()) == n and torch.equal(short[0], full[0])
    assert hk.hk_noalloc_sync_status(_stream()) == hk.HK_OK


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_1405_1931_gb300 import hk
    per = (ctypes.c_int * 3)(1, 1, 1)
    # 264^3 and 512^3 need more than the fixed scratch; rejected on the host, nothing is touched
    for L in (264, 512):
        rc = hk.load().hk_label_noalloc(ctypes.c_void_p(16), L, L, L, per, ctypes.c_void_p(16), None, 0,
                                        None, None, None)
        assert rc == hk.HK_ERR_TOO_LARGE, L
