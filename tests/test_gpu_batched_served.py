"""Batched (CUDA-graph replay) and served (continuous batching) forms against
labelling alone and against the oracle.  Outputs are integers: tolerance 0."""
import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check(out, want, what):
    labels, sizes, hist, ncl = out[:4]
    n = int(ncl.item())
    assert n == want[3], what
    np.testing.assert_array_equal(labels.cpu().numpy(), want[0], err_msg=what)
    np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1], err_msg=what)
    np.testing.assert_array_equal(hist.cpu().numpy(), want[2], err_msg=what)


def test_batched_graph_replay_is_exact():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_graphs(True)
    params = fields.batch_params(12, master_seed=5)
    items, wants = [], []
    for prm in params:
        dims = tuple(min(prm[k], 96) for k in ("nx", "ny", "nz"))
        phi = fields.iid_field(*dims, seed=prm["seed"], occupancy=prm["occupancy"])
        d = torch.from_numpy(phi).cuda()
        items.append((d, prm["periodic"], lab.alloc_outputs(d.shape, d.device)))
        wants.append(oracle.label(phi, prm["periodic"]))
    s = torch.cuda.Stream()
    for call in range(3):            # 1st: run + capture, then two replays
        for _, _, out in items:
            out[0].fill_(-7)
            out[1].fill_(-7)
            out[2].fill_(-7)
        with torch.cuda.stream(s):
            lab.label_batched(items, stream=s)
        lab.sync_status(s)
        for (d, per, out), want in zip(items, wants):
            _check(out, want, f"call {call}")
    lab.close()


def test_single_lattice_graph_replay_is_exact():
    """hk_label with graphs on: the first call runs and captures, later calls replay, on the
    one-launch path (32^3 and 64 x 48 x 40: a cluster kernel) and on the tiled passes
    (160 x 96 x 64, dependent launches)."""
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_graphs(True)
    s = torch.cuda.Stream()
    for shape, per in [((32, 32, 32), (1, 1, 1)), ((64, 48, 40), (1, 0, 1)), ((160, 96, 64), (1, 1, 0))]:
        phi_np = fields.iid_field(*shape, seed=13, occupancy=0.3116)
        want = oracle.label(phi_np, per)
        phi = torch.from_numpy(phi_np).cuda()
        out = lab.alloc_outputs(phi.shape, phi.device)
        for call in range(3):
            out[0].fill_(-7)
            out[1].fill_(-7)
            out[2].fill_(-7)
            with torch.cuda.stream(s):
                lab.label(phi, per, out=out, stream=s)
            lab.sync_status(s)
            _check(out, want, f"{shape} call {call}")
    lab.close()


def test_served_results_equal_alone_and_oracle():
    from paper_1405_1931_gb300 import serve
    from paper_1405_1931_gb300.hk import Labeller
    reqs = serve.request_stream(24, rate=3000.0, seed=9, l_lo=24, l_hi=72)
    srv = serve.Server(0, cap_bytes=2 * serve.GB, workers=3, max_batch=8)
    stats = srv.serve(reqs, keep_outputs=True)
    srv.close()
    assert stats["requests"] == 24
    lab = Labeller(0)
    for k, r in enumerate(stats["done"]):
        alone = lab.alloc_outputs(r.phi.shape, r.phi.device)
        lab.label(r.phi, r.periodic, out=alone)
        torch.cuda.synchronize()
        n = int(alone[3].item())
        assert int(r.out[3].item()) == n == r.n_clusters
        assert torch.equal(r.out[0], alone[0])
        assert torch.equal(r.out[1][:n], alone[1][:n])
        assert torch.equal(r.out[2], alone[2])
        if k < 8:   # the exact bytes that were labelled, against the oracle
            _check(r.out, oracle.label(r.phi.cpu().numpy(), r.periodic), f"request {r.rid}")
    lab.close()


def test_served_mix_up_to_256_equals_alone_and_oracle():
    """Small requests mixed with ones of several hundred thousand to 16 M sites (sides
    log-uniform in [24, 256], fields ready at arrival and generated on arrival): every
    result equals labelling the request alone; the largest three and the smallest three
    also equal the oracle."""
    from paper_1405_1931_gb300 import serve
    from paper_1405_1931_gb300.hk import Labeller
    srv = serve.Server(0, cap_bytes=8 * serve.GB, workers=4, max_side=256)
    lab = Labeller(0)
    for lead in (0.05, 0.0):
        reqs = serve.request_stream(20, rate=2000.0, seed=17, l_lo=24, l_hi=256)
        stats = srv.serve(reqs, keep_outputs=True, gen_lead_s=lead)
        assert stats["requests"] == 20 and stats["failed"] == 0
        done = sorted(stats["done"], key=lambda r: r.sites)
        assert done[-1].L >= 150 and done[0].L <= 40          # a real mix of sizes
        for r in done:
            alone = lab.alloc_outputs(r.phi.shape, r.phi.device)
            lab.label(r.phi, r.periodic, out=alone)
            torch.cuda.synchronize()
            n = int(alone[3].item())
            assert int(r.out[3].item()) == n == r.n_clusters
            assert torch.equal(r.out[0], alone[0])
            assert torch.equal(r.out[1][:n], alone[1][:n])
            assert torch.equal(r.out[2], alone[2])
        if lead > 0:
            for r in done[:3] + done[-3:]:
                _check(r.out, oracle.label(r.phi.cpu().numpy(), r.periodic), f"request {r.rid} L={r.L}")
    lab.close()
    srv.close()


def test_served_fifo_matches_continuous():
    from paper_1405_1931_gb300 import serve
    a = serve.Server(0, cap_bytes=1 * serve.GB, workers=2, max_batch=6)
    ra = a.serve(serve.request_stream(16, rate=5000.0, seed=11, l_lo=20, l_hi=64), keep_outputs=True)
    rb = a.serve(serve.request_stream(16, rate=5000.0, seed=11, l_lo=20, l_hi=64), mode="fifo", keep_outputs=True)
    a.close()
    by_id = {r.rid: r for r in rb["done"]}
    for r in ra["done"]:
        q = by_id[r.rid]
        assert r.n_clusters == q.n_clusters
        assert torch.equal(r.out[0], q.out[0])
        assert torch.equal(r.out[2], q.out[2])
    assert ra["p99_ms"] >= ra["p50_ms"] > 0
