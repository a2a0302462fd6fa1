"""Host logic of the served workload, on the CPU: the seeded request stream and the
admission size of a request (no GPU)."""
import math

import numpy as np

from paper_1405_1931_gb300 import hk, serve


def test_request_stream_is_seeded_and_shaped():
    a = serve.request_stream(400, rate=400.0, seed=3)
    b = serve.request_stream(400, rate=400.0, seed=3)
    assert [(r.arrival, r.kind, r.L) for r in a] == [(r.arrival, r.kind, r.L) for r in b]
    arrivals = np.array([r.arrival for r in a])
    assert (np.diff(arrivals) > 0).all()
    # exponential gaps of mean 1/rate: the mean of 400 gaps within 4 standard errors
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert abs(gaps.mean() - 1 / 400.0) < 4 * (1 / 400.0) / math.sqrt(400)
    kinds = [r.kind for r in a]
    frac = kinds.count("emulsion") / len(kinds)
    assert abs(frac - 0.8) < 4 * math.sqrt(0.8 * 0.2 / 400)
    sides = np.array([r.L for r in a])
    assert sides.min() >= 64 and sides.max() <= 512
    # log-uniform sides: log(L / 64) / log(8) is uniform on [0, 1]
    v = np.log(sides / 64.0) / math.log(8.0)
    assert abs(v.mean() - 0.5) < 4 * math.sqrt(1 / 12 / 400)


def test_request_contents():
    for r in serve.request_stream(200, seed=5):
        if r.kind == "emulsion":
            centres, radii = r.spheres
            want = max(1, int(round(0.3 * r.L ** 3 / (4.0 / 3.0 * math.pi * 1250.0))))
            assert len(radii) == want and centres.shape == (want, 3)
            assert (radii >= 5).all() and (radii <= 15).all()
        else:
            assert len(r.axes) == 3
            assert all(min(10.0, r.L / 2 - 2) <= a <= min(60.0, r.L / 2 - 2) for a in r.axes)


def test_admission_bytes():
    r = serve.request_stream(1, seed=1)[0]
    n = r.L ** 3
    assert r.nbytes() == 8 * n + 8 * ((n + 1) // 2) + hk.hk_workspace_bytes(r.L, r.L, r.L)
    assert hk.hk_workspace_bytes(r.L, r.L, r.L) > 0


def _sched(n_small=2, workers=4):
    """A Server with only the scheduling state that `_pick` reads (no device)."""
    srv = object.__new__(serve.Server)
    srv.n_small, srv.small_sites, srv.max_batch, srv.small_batch_sites = n_small, 1 << 21, 3, 1 << 23
    srv.streams = [None] * workers
    return srv


def test_pick_queues_large_requests_on_one_stream_in_arrival_order():
    from collections import deque
    srv = _sched()
    reqs = [serve.Request(k, 0.001 * k, "emulsion", L) for k, L in enumerate([200, 64, 300, 80, 96, 256])]
    ready = deque(reqs)
    nbusy = [0, 0, 0, 0]
    picks = []
    while ready:
        w, batch = srv._pick(ready, nbusy)
        if not batch:
            break
        nbusy[w] += 1
        picks.append((w, [r.rid for r in batch]))
    # large ones to worker 2 whatever it has in flight, oldest first; the small ones
    # (<= 128^3) batched, oldest first, on an idle small worker
    assert [p for p in picks if p[0] == 2] == [(2, [0]), (2, [2]), (2, [5])]
    assert [p for p in picks if p[0] != 2] == [(0, [1, 3, 4])]
    assert nbusy == [1, 0, 3, 0]


def test_pick_small_batches_wait_for_an_idle_worker():
    from collections import deque
    srv = _sched()
    ready = deque(serve.Request(k, 0.0, "emulsion", 64) for k in range(7))
    nbusy = [1, 1, 2, 0]
    w, batch = srv._pick(ready, nbusy)          # both small workers busy: the idle last worker
    assert w == 3 and [r.rid for r in batch] == [0, 1, 2]   # max_batch 3
    nbusy[3] = 1
    assert srv._pick(ready, nbusy) == (-1, [])  # nobody idle: wait
    nbusy[0] = 0
    w, batch = srv._pick(ready, nbusy)
    assert w == 0 and [r.rid for r in batch] == [3, 4, 5]
