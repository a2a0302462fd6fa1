"""Host logic of the slab decomposition across ranks, on the CPU: the slab bounds and the
all_gather helper of paper_1405_1931_gb300/distributed.py over gloo with two processes."""
import multiprocessing as mp
import socket

import pytest

from paper_1405_1931_gb300 import distributed as D

torch = pytest.importorskip("torch")


def test_slab_bounds_cover_the_lattice_in_order():
    for nz in (1, 2, 5, 64, 1000):
        for R in range(1, min(nz, 9) + 1):
            planes = []
            for r in range(R):
                z0, n = D.slab_bounds(nz, R, r)
                assert n >= 1 and n in (nz // R, nz // R + 1)
                planes.extend(range(z0, z0 + n))
            assert planes == list(range(nz))
    with pytest.raises(ValueError):
        D.slab_bounds(3, 4, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_all_gather_two_ranks_on_gloo():
    import dist_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=dist_worker.gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (a, b)) for r, a, b in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        a, b = got[r]
        assert a.tolist() == [list(range(6)), [10 + i for i in range(6)]]
        assert b.reshape(-1).tolist() == [3, 4]
