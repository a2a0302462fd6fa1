"""Parity of the droplet-size histogram by R_c (Fig. 5) with the oracle.

The sizes come from the GPU labelling of emulsion fields (bit-exact with the
oracle by the parity tests); the histogram must equal the oracle's exactly and
the sum of R_c within 1e-12 relative (cube roots and summation order differ).
"""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGES = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0, 12.0, 15.0, 20.0]


@pytest.fixture(scope="module")
def labeller():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    yield lab
    lab.close()


def test_rc_histogram_single_and_stacked(labeller):
    from paper_1405_1931_gb300 import hk
    stacked = np.zeros(len(EDGES) + 1, dtype=np.int64)
    stacked_sum = 0.0
    acc = None
    for seed in (21, 22, 23):
        phi = fields.emulsion_field(96, 80, 64, 60, seed=seed)
        labels, sizes, hist, ncl = labeller.label(torch.from_numpy(phi).cuda(), (1, 1, 1))
        n = int(ncl.item())
        want_h, want_s = oracle.rc_histogram(sizes[:n].cpu().numpy(), EDGES)
        got_h, got_s = hk.rc_histogram(sizes, ncl, EDGES)
        np.testing.assert_array_equal(got_h.cpu().numpy(), want_h)
        assert abs(float(got_s.item()) - want_s) <= 1e-12 * max(1.0, want_s)
        stacked += want_h
        stacked_sum += want_s
        acc = hk.rc_histogram(sizes, ncl, EDGES, out=acc, accumulate=acc is not None)
    np.testing.assert_array_equal(acc[0].cpu().numpy(), stacked)
    assert abs(float(acc[1].item()) - stacked_sum) <= 1e-12 * stacked_sum


def test_rc_histogram_respects_capacity_and_edges(labeller):
    from paper_1405_1931_gb300 import hk
    sizes = torch.tensor([1, 8, 27, 1000, 5, 7], dtype=torch.int64, device="cuda")
    ncl = torch.tensor([6], dtype=torch.int64, device="cuda")
    h, s = hk.rc_histogram(sizes, ncl, [0.5, 1.0, 2.0, 5.0, 10.0], cap=4)   # only the first four
    assert h.cpu().tolist() == [0, 1, 2, 0, 1, 0]
    want_h, want_s = oracle.rc_histogram([1, 8, 27, 1000], [0.5, 1.0, 2.0, 5.0, 10.0])
    assert abs(float(s.item()) - want_s) <= 1e-12 * want_s
