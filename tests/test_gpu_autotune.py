"""The autotuner on the GPU: it times every tile shape and merge schedule on an uneven
batch, keeps the fastest, and the batch labelled with the chosen configuration is
bit-identical to the oracle (every candidate computes the same result; only the time
differs).  Each merge schedule is also checked against the oracle directly."""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(lab, n, seed, cap_side=128):
    params = fields.batch_params(n, master_seed=seed)
    items, wants = [], []
    for prm in params:
        dims = tuple(min(prm[k], cap_side) for k in ("nx", "ny", "nz"))
        phi = fields.iid_field(*dims, seed=prm["seed"], occupancy=prm["occupancy"])
        d = torch.from_numpy(phi).cuda()
        items.append((d, prm["periodic"], lab.alloc_outputs(d.shape, d.device)))
        wants.append(oracle.label(phi, prm["periodic"]))
    return items, wants


def _check(items, wants):
    for (d, per, (labels, sizes, hist, ncl, cap)), want in zip(items, wants):
        n = int(ncl.item())
        assert n == want[3]
        np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
        np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1])
        np.testing.assert_array_equal(hist.cpu().numpy(), want[2])


def test_tune_picks_a_schedule_and_its_result_is_exact():
    from paper_1405_1931_gb300 import autotune
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    items, wants = _batch(lab, 10, seed=7)
    got = autotune.tune(lab, items, reps=1, cache=None)
    assert not got["cached"]
    assert got["tile"] in autotune.TILES and got["merge"] in autotune.MERGES
    assert len(got["ms"]) == len(autotune.TILES) + len(autotune.MERGES) - 1
    assert lab.tile == got["tile"] and lab.merge == got["merge"]
    for _, _, out in items:
        out[0].fill_(-7)
    lab.label_batched(items)
    lab.sync_status()
    _check(items, wants)
    lab.close()


@pytest.mark.parametrize("merge", [(1, 1), (2, 1), (4, 1), (1, 0), (2, 0), (4, 0)])
def test_every_merge_schedule_is_exact(merge):
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_small_path(False)
    lab.set_merge(*merge)
    items, wants = _batch(lab, 6, seed=11, cap_side=96)
    lab.label_batched(items)
    lab.sync_status()
    _check(items, wants)
    phi_np = fields.iid_field(160, 96, 80, seed=3, occupancy=fields.P_C_SIMPLE_CUBIC)
    want = oracle.label(phi_np, (1, 1, 1))
    labels, sizes, hist, ncl = lab.label(torch.from_numpy(phi_np).cuda(), (1, 1, 1))
    lab.sync_status()
    n = int(ncl.item())
    assert n == want[3]
    np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
    np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1])
    lab.close()
