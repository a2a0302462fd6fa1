"""Failure detection on the GPU without a GPU fault.

Every device loop whose length depends on other threads is capped (the
shared-memory union retries, the global finds, unions and compression of the
piece merge); a loop that reaches its cap sets a flag in the context's device
status word and stops, and hk_sync_status turns the flag into HK_ERR_TIMEOUT.
hk_set_loop_cap lowers those caps so that ordinary inputs make the loops give
up: the call then returns wrong labels, but every access stays in range (a
capped find stops at a valid id, a capped union stops without linking), the
status is reported, the context and the GPU stay usable, and the next call at
the natural caps is exact again.  The waits on TMA copies keep their bound.
"""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rod_z(nx, ny, nz):
    """A one-site rod along z through every tile plane: one piece per tile, chained
    from tile to tile, so the piece merge builds a chain of nz / 16 pieces."""
    phi = np.full((nz, ny, nx), -1.0, np.float32)
    phi[:, ny // 3, nx // 5] = 1.0
    return phi


def _label(lab, phi_np, per):
    phi = torch.from_numpy(np.ascontiguousarray(phi_np)).cuda()
    labels, sizes, hist, ncl = lab.label(phi, per)
    torch.cuda.synchronize()
    n = int(ncl.item())
    return labels.cpu().numpy(), sizes[:n].cpu().numpy(), hist.cpu().numpy(), n


def _status(lab):
    from paper_1405_1931_gb300 import hk
    return hk.hk_sync_status(lab.ctx, hk._stream_handle(None))


@pytest.mark.parametrize("case", ["rod", "critical"])
def test_capped_loops_report_timeout_and_the_next_call_is_exact(case):
    from paper_1405_1931_gb300 import hk
    lab = hk.Labeller(0)
    if case == "rod":
        phi = _rod_z(32, 32, 2048)                        # 128 tiles chained along z
        per = (1, 1, 1)
    else:
        phi = fields.iid_field(160, 128, 128, seed=41, occupancy=fields.P_C_SIMPLE_CUBIC)
        per = (1, 1, 1)
    want = oracle.label(phi, per)

    assert _status(lab) == hk.HK_OK
    lab.set_loop_cap(1)
    _label(lab, phi, per)
    assert _status(lab) == hk.HK_ERR_TIMEOUT             # a capped loop gave up and said so
    assert _status(lab) == hk.HK_OK                      # reading the status clears it

    lab.set_loop_cap(0)                                  # natural bounds: exact again
    got = _label(lab, phi, per)
    assert _status(lab) == hk.HK_OK
    assert got[3] == want[3]
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    np.testing.assert_array_equal(got[2], want[2])
    # the GPU is still usable by others: a plain torch computation
    x = torch.arange(1 << 20, device="cuda", dtype=torch.float32)
    assert float(x.sum().item()) == float(np.arange(1 << 20, dtype=np.float64).sum())
    lab.close()


def test_loop_cap_is_rejected_when_negative():
    from paper_1405_1931_gb300 import hk
    lab = hk.Labeller(0)
    assert hk.hk_set_loop_cap(lab.ctx, -1) == hk.HK_ERR_ARG
    assert hk.hk_set_loop_cap(lab.ctx, 0) == hk.HK_OK
    lab.close()
