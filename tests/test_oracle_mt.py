"""The paper's parallel scheme (Sec. 3) on host threads against the serial oracle.

One slab of planes along z per thread: local serial labelling, Eq. 1's global ids,
halo equivalences across the slab faces (and the periodic z edge), resolution at the
root and relabelling.  The output is unique, so it must equal ``oracle.label`` bit for
bit for every thread count, including more threads than planes.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

PERS = list(itertools.product((0, 1), repeat=3))


def same(a, b, what):
    assert a[3] == b[3], what
    np.testing.assert_array_equal(a[0], b[0], err_msg=what)
    np.testing.assert_array_equal(a[1], b[1], err_msg=what)
    np.testing.assert_array_equal(a[2], b[2], err_msg=what)


def test_random_small_lattices_every_thread_count():
    rng = np.random.default_rng(3)
    for it in range(200):
        shape = tuple(int(v) for v in rng.integers(1, 10, size=3))
        occ = rng.random(shape) < rng.uniform(0.1, 0.9)
        phi = np.where(occ, 1.0, -1.0).astype(np.float32)
        per = PERS[it % 8]
        for threads in (1, 2, 3, int(rng.integers(4, 12))):
            same(oracle.label_mt(phi, per, threads=threads), oracle.label(phi, per), f"{shape} {per} {threads}")


@pytest.mark.parametrize("threads", [2, 5, 16])
def test_critical_field(threads):
    """64 x 48 x 40 at p_c with every periodic flag set: clusters span every slab face."""
    phi = fields.iid_field(64, 48, 40, seed=9, occupancy=0.3116)
    for per in [(1, 1, 1), (0, 0, 0), (0, 0, 1)]:
        same(oracle.label_mt(phi, per, threads=threads), oracle.label(phi, per), f"{per}")


def test_closed_forms_across_slabs():
    """The alternating patterns of Sec. 3 split over slabs: V/2 single sites, and blocks."""
    z, y, x = np.meshgrid(np.arange(16), np.arange(12), np.arange(10), indexing="ij")
    checker = np.where((x + y + z) % 2 == 0, 1.0, -1.0).astype(np.float32)
    got = oracle.label_mt(checker, (0, 0, 0), threads=4)
    assert got[3] == 16 * 12 * 10 // 2 and (got[1] == 1).all()
    blocks = np.where(((x // 5) + (y // 3) + (z // 4)) % 2 == 0, 1.0, -1.0).astype(np.float32)
    got = oracle.label_mt(blocks, (1, 1, 1), threads=4)   # 2 x 4 x 4 domains: even counts, periodic-safe
    assert got[3] == (2 * 4 * 4) // 2 and (got[1] == 5 * 3 * 4).all()


def test_capacity_and_arguments():
    phi = fields.iid_field(20, 20, 20, seed=2, occupancy=0.3)
    want = oracle.label(phi, (1, 1, 1))
    got = oracle.label_mt(phi, (1, 1, 1), threads=3, sizes_cap=5)
    assert got[3] == want[3]
    np.testing.assert_array_equal(got[1], want[1][:5])
    lib = oracle.load()
    per = np.ones(3, dtype=np.int32)
    out = np.empty(phi.shape, dtype=np.int32)
    hist = np.zeros(32, dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    assert lib.hk_oracle_mt_label(phi.ctypes.data, 20, 20, 20, per.ctypes.data, 0, out.ctypes.data, None, 0,
                                  hist.ctypes.data, n.ctypes.data) == oracle.ERR_ARG


def test_two_process_wrap_merge():
    """The situation of Fig. 2 (whose lattice is not reproducible): two processes on a
    periodic lattice whose local clusters are joined only through the face between them,
    the periodic z edge and the x wrap, leaving two clusters.  Lattice (z rows, x columns,
    ny = 1), slabs z = 0-1 and z = 2-3:
        z=0: X . X . . X
        z=1: X . . . . .
        z=2: X . . . X .
        z=3: . . X . X X
    Process 0 has local clusters {x=0 column, x=5 via the x wrap} and {(2,0)}; process 1
    has three.  The face z=1|z=2 and the z wrap join them into {7 sites, first site 0} and
    {(2,0), (2,3)}; without periodic edges there are five clusters."""
    rows = ["X.X..X", "X.....", "X...X.", "..X.XX"]
    occ = np.array([[c == "X" for c in r] for r in rows]).reshape(4, 1, 6)
    phi = np.where(occ, 1.0, -1.0).astype(np.float32)
    for got in (oracle.label(phi, (1, 1, 1)), oracle.label_mt(phi, (1, 1, 1), threads=2)):
        assert got[3] == 2
        assert got[1].tolist() == [7, 2]
        lab = got[0].reshape(4, 6)
        assert set(lab[occ.reshape(4, 6)].tolist()) == {0, 2}
        assert lab[0, 2] == 2 and lab[3, 2] == 2 and lab[3, 5] == 0
    assert oracle.label_mt(phi, (0, 0, 0), threads=2)[3] == 5
