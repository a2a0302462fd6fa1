"""The domain-decomposed scheme of Sec. 3 across ranks against the oracle.

Ranks are processes of a gloo group on the one GPU (each its own context), so the
face exchange passes through the host; the kernels of one rank never wait on
another's.  For each case the slabs' labels, concatenated along z, must equal the
oracle's labels of the whole lattice; the ranks' own size lists, concatenated in
rank order, its sizes; and the summed histogram and count, its histogram and count.
Cases: critical percolation with every periodic set, uneven slabs over three ranks,
slabs of one plane, a serpentine that crosses every slab face many times, a dense
spanning field, an empty lattice and a column that wraps through z.
"""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    pc = fields.P_C_SIMPLE_CUBIC
    out = [(fields.iid_field(64, 48, 40, seed=31, occupancy=pc), (1, 1, 1)),
           (fields.iid_field(64, 48, 41, seed=32, occupancy=pc), (0, 1, 0)),
           (fields.iid_field(33, 20, 6, seed=33, occupancy=0.5), (1, 0, 1)),
           (fields.iid_field(50, 40, 60, seed=34, occupancy=0.6), (1, 1, 1)),
           (fields.iid_field(40, 30, 3, seed=35, occupancy=0.45), (1, 1, 1)),
           (np.full((12, 10, 9), -1.0, np.float32), (1, 1, 1))]
    snake = np.full((30, 16, 24), -1.0, np.float32)           # a serpentine through every plane
    snake[:, 2, :] = 1.0
    snake[:, 3:13, 23] = 1.0
    snake[:, 12, :] = 1.0
    for z in range(30):
        snake[z, 2 if z % 2 else 12, 0] = -1.0
    out.append((snake, (0, 0, 0)))
    col = np.full((24, 8, 8), -1.0, np.float32)                # one column: one cluster only with the z wrap
    col[:, 3, 5] = 1.0
    col[11, 3, 5] = -1.0
    out.append((col, (0, 0, 1)))
    out.append((col, (0, 0, 0)))
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_across_ranks_equal_the_oracle(world):
    import dist_worker
    cases = _cases()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=dist_worker.slab_worker, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for i, (phi, per) in enumerate(cases):
        want = oracle.label(phi, per)
        parts = [got[r][i] for r in range(world)]
        labels = np.concatenate([pt[1] for pt in parts], axis=0)
        np.testing.assert_array_equal(labels, want[0], err_msg=f"case {i} labels")
        sizes = np.concatenate([pt[2] for pt in parts])
        np.testing.assert_array_equal(sizes, want[1], err_msg=f"case {i} sizes")
        assert [pt[3] for pt in parts] == list(np.cumsum([0] + [len(pt[2]) for pt in parts[:-1]])), f"case {i} offsets"
        for pt in parts:
            assert pt[4] == want[3], f"case {i} count"
            np.testing.assert_array_equal(pt[5], want[2], err_msg=f"case {i} hist")
