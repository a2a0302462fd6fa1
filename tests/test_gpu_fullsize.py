"""Parity at the full sizes of the benchmarked workloads, in the launch configuration
bench.py times (default tile 32x16x16, device-resident fields).

- 1024^3 critical site percolation (p = 0.3116, periodic xyz): every label, size and
  histogram bin against the oracle (about 10 s of serial CPU work);
- the full 96-lattice uneven batch (axes up to 384), labelled in one batched call,
  every lattice against the oracle;
- the largest lattice the library takes: 1291 x 1290 x 1289 = 2,146,687,710 sites, just below
  2^31, ragged along every axis, critical percolation, periodic xyz, against the oracle
  (site indices, labels and keys near the int32 limit);
- the benchmark pattern of Sec. 3 at 1024^3 (alternating cubic domains touching only at
  edges and corners), against its closed form: (1024 / b)^3 / 2 clusters of b^3 sites,
  each labelled by its corner; b = 1 is the maximum V / 2 clusters.
The fields are generated on the device and copied to the host, so the oracle labels
exactly the bytes the GPU labels.
"""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields
import closed_forms

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def labeller():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    yield lab
    lab.close()


def test_critical_1024_full_parity(labeller):
    from paper_1405_1931_gb300 import hk
    L = 1024
    phi = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    assert hk.hk_gen_iid(phi.data_ptr(), L, L, L, 0, fields.P_C_SIMPLE_CUBIC, 0) == 0
    labels, sizes, hist, ncl = labeller.label(phi, (1, 1, 1))
    labeller.sync_status()
    n = int(ncl.item())
    phi_h = phi.cpu().numpy()
    del phi
    got_labels = labels.cpu().numpy()
    got_sizes = sizes[:n].cpu().numpy()
    got_hist = hist.cpu().numpy()
    del labels, sizes, hist
    torch.cuda.empty_cache()
    want = oracle.label(phi_h, (1, 1, 1))
    assert n == want[3]
    assert np.array_equal(got_labels, want[0])
    assert np.array_equal(got_sizes, want[1])
    assert np.array_equal(got_hist, want[2])


def test_uneven_batch_96_full_parity(labeller):
    from paper_1405_1931_gb300 import hk
    params = fields.batch_params(96, master_seed=2)
    s = torch.cuda.current_stream()
    items = []
    for prm in params:
        d = torch.empty((prm["nz"], prm["ny"], prm["nx"]), dtype=torch.float32, device="cuda")
        assert hk.hk_gen_iid(d.data_ptr(), prm["nx"], prm["ny"], prm["nz"], prm["seed"], prm["occupancy"],
                             hk._stream_handle(s)) == 0
        items.append((d, prm["periodic"], labeller.alloc_outputs(d.shape, d.device)))
    labeller.label_batched(items)
    labeller.sync_status()
    for prm, (d, per, (labels, sizes, hist, ncl, cap)) in zip(params, items):
        want = oracle.label(d.cpu().numpy(), per)
        n = int(ncl.item())
        assert n == want[3], prm
        assert np.array_equal(labels.cpu().numpy(), want[0]), prm
        assert np.array_equal(sizes[:n].cpu().numpy(), want[1]), prm
        assert np.array_equal(hist.cpu().numpy(), want[2]), prm


@pytest.mark.parametrize("b", [1, 2, 16, 256])
def test_block_benchmark_1024_closed_form(labeller, b):
    L = 1024
    phi = fields.block_field_device(L, b)
    labels, sizes, hist, ncl = labeller.label(phi, (1, 1, 1))
    labeller.sync_status()
    del phi
    n = int(ncl.item())
    assert n == (L // b) ** 3 // 2
    assert bool((sizes[:n] == b ** 3).all())
    want_hist = torch.zeros(32, dtype=torch.int64, device="cuda")
    want_hist[(b ** 3).bit_length() - 1] = n
    assert torch.equal(hist, want_hist)
    assert torch.equal(labels, closed_forms.block_labels_device(L, b))


def test_near_max_sites_full_parity(labeller):
    from paper_1405_1931_gb300 import hk
    nx, ny, nz = 1291, 1290, 1289
    assert nx * ny * nz < 2 ** 31 and nx * ny * nz > 2 ** 31 - 2 ** 20
    phi = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    assert hk.hk_gen_iid(phi.data_ptr(), nx, ny, nz, 7, fields.P_C_SIMPLE_CUBIC, 0) == 0
    labels, sizes, hist, ncl = labeller.label(phi, (1, 1, 1))
    labeller.sync_status()
    n = int(ncl.item())
    phi_h = phi.cpu().numpy()
    del phi
    got_labels = labels.cpu().numpy()
    got_sizes = sizes[:n].cpu().numpy()
    got_hist = hist.cpu().numpy()
    del labels, sizes, hist
    torch.cuda.empty_cache()
    want = oracle.label(phi_h, (1, 1, 1))
    del phi_h
    assert n == want[3]
    assert np.array_equal(got_sizes, want[1])
    assert np.array_equal(got_hist, want[2])
    assert np.array_equal(got_labels, want[0])
