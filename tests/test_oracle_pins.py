"""Pins for the CPU oracle: brute force, closed forms, invariants and the paper's printed values.

Every check here is independent of the oracle's own code: the expected values
come from brute-force flood fill or relaxation (``brute.py``), from scipy's
labeller on the non-periodic special case, from closed forms derived by hand
for structured patterns, or from values the paper states (``golden/``).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields
from brute import bfs_label, relax_label, canonical_from_partition, log2_hist
import closed_forms

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PERIODIC_ALL = list(itertools.product((0, 1), repeat=3))


def occ_to_phi(occ):
    return np.where(occ, np.float32(1.0), np.float32(-1.0)).astype(np.float32)


def assert_same(got, want):
    gl, gs, gh, gn = got
    wl, ws, wh, wn = want
    assert gn == wn
    np.testing.assert_array_equal(gl, wl)
    np.testing.assert_array_equal(gs, ws)
    np.testing.assert_array_equal(gh, wh)


# --------------------------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 2, 3)])
def test_exhaustive_small_vs_bfs(shape):
    """Every occupancy pattern of 2x2x2 and 3x2x2 (nx=3) under all 8 periodic flag sets."""
    n = int(np.prod(shape))
    for bits in range(1 << n):
        occ = np.array([(bits >> i) & 1 for i in range(n)], dtype=bool).reshape(shape)
        phi = occ_to_phi(occ)
        for per in PERIODIC_ALL:
            assert_same(oracle.label(phi, per), bfs_label(occ, per))


@pytest.mark.parametrize("shape", [(1, 1, 5), (1, 5, 1), (5, 1, 1), (1, 2, 7), (2, 1, 3), (1, 1, 1), (3, 1, 2)])
def test_degenerate_axes_vs_bfs(shape):
    """Axis lengths 1 and 2 with periodic wraps: self-edges and doubled edges."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        occ = rng.random(shape) < 0.6
        for per in PERIODIC_ALL:
            assert_same(oracle.label(occ_to_phi(occ), per), bfs_label(occ, per))


@pytest.mark.parametrize("p", [0.1, 0.3, 0.5, 0.7, 0.9])
def test_random_vs_bfs(p):
    rng = np.random.default_rng(int(p * 100))
    for _ in range(6):
        shape = tuple(int(v) for v in rng.integers(1, 9, size=3))
        occ = rng.random(shape) < p
        for per in PERIODIC_ALL:
            assert_same(oracle.label(occ_to_phi(occ), per), bfs_label(occ, per))


@pytest.mark.parametrize("shape,p", [((32, 32, 32), 0.3116), ((17, 40, 23), 0.3), ((9, 64, 33), 0.25)])
def test_random_vs_relaxation(shape, p):
    rng = np.random.default_rng(11)
    occ = rng.random(shape) < p
    for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1), (0, 1, 0)]:
        assert_same(oracle.label(occ_to_phi(occ), per), relax_label(occ, per))


def test_nonperiodic_vs_scipy():
    """Without periodic edges, clusters are scipy.ndimage.label's with the 6-neighbour structure."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    struct = ndimage.generate_binary_structure(3, 1)
    for shape, p in [((40, 33, 21), 0.3116), ((64, 64, 64), 0.2), ((16, 48, 80), 0.45)]:
        occ = rng.random(shape) < p
        part, _ = ndimage.label(occ, structure=struct)
        want = canonical_from_partition(np.where(occ, part, -1))
        assert_same(oracle.label(occ_to_phi(occ), (0, 0, 0)), want)


def test_generated_fields_vs_relaxation():
    """The seeded fields of the workloads (small instances), with the exact float32 bytes."""
    phi, per = fields.small_iid()
    assert_same(oracle.label(phi, per), relax_label(phi > 0, per))
    phi = fields.emulsion_field(48, 40, 32, 12, seed=1)
    assert_same(oracle.label(phi, (1, 1, 1)), relax_label(phi > 0, (1, 1, 1)))


# --------------------------------------------------------------------------------------------
# occupancy rule: phi > 0 strictly
# --------------------------------------------------------------------------------------------

def test_occupancy_is_strictly_positive():
    """Sec. 2: phi > 0 is a cluster site, phi <= 0 is the medium; +0, -0 and NaN are medium."""
    vals = np.array([0.0, -0.0, np.nan, -np.inf, -1e-45, 1e-45, np.inf, 2.0], dtype=np.float32)
    phi = vals.reshape(1, 1, 8)
    labels, sizes, hist, n = oracle.label(phi, (0, 0, 0))
    # occupied: 1e-45 (x=5), inf (x=6), 2.0 (x=7): one run of three
    np.testing.assert_array_equal(labels.reshape(-1), [-1, -1, -1, -1, -1, 5, 5, 5])
    assert n == 1 and sizes.tolist() == [3]
    zero = np.zeros((4, 4, 4), dtype=np.float32)
    assert oracle.label(zero, (1, 1, 1))[3] == 0


# --------------------------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("per", PERIODIC_ALL)
def test_empty_and_full(per):
    dims = (7, 5, 3)
    phi = np.full(dims[::-1], -0.5, dtype=np.float32)
    labels, sizes, hist, n = oracle.label(phi, per)
    assert n == 0 and sizes.size == 0 and hist.sum() == 0 and (labels == -1).all()
    phi[:] = 0.5
    labels, sizes, hist, n = oracle.label(phi, per)
    N = phi.size
    assert n == 1 and sizes.tolist() == [N] and (labels == 0).all()
    assert hist[N.bit_length() - 1] == 1 and hist.sum() == 1


def _read_golden(name):
    cases, cur = [], {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, v = (t.strip() for t in line.split("="))
        if k == "dims" and cur:
            cases.append(cur)
            cur = {}
        cur[k] = [int(t) for t in v.split()]
    cases.append(cur)
    return cases


@pytest.mark.parametrize("case", _read_golden("ncl_max_alternating.txt"))
def test_ncl_max_alternating(case):
    """Sec. 3: n_cl,max = V/2 for single sites alternating along every axis."""
    nx, ny, nz = case["dims"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    occ = (x + y + z) % 2 == 0
    for per in PERIODIC_ALL:
        labels, sizes, hist, n = oracle.label(occ_to_phi(occ), per)
        assert n == case["expected_n_clusters"][0] == nx * ny * nz // 2
        assert (sizes == case["expected_size"][0]).all()
        idx = np.arange(occ.size).reshape(occ.shape)
        np.testing.assert_array_equal(labels, np.where(occ, idx, -1))


@pytest.mark.parametrize("case", _read_golden("block_benchmark.txt"))
def test_block_benchmark_pattern(case):
    """Sec. 3 benchmark: alternating rectangular domains touching only at corners/edges."""
    nx, ny, nz = case["dims"]
    bx, by, bz = case["block"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    occ = ((x // bx) + (y // by) + (z // bz)) % 2 == 0
    for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
        labels, sizes, hist, n = oracle.label(occ_to_phi(occ), per)
        assert n == case["expected_n_clusters"][0]
        assert (sizes == case["expected_size"][0]).all()
        assert hist[case["expected_size"][0].bit_length() - 1] == n


@pytest.mark.parametrize("L,b", [(8, 1), (16, 2), (16, 4), (32, 8)])
def test_block_benchmark_closed_form_helpers(L, b):
    """The closed form used at 1024^3 on the GPU (fields.block_field_device / closed_forms.block_labels_device,
    run here with torch on the CPU) agrees with the oracle: corner labels, (L/b)^3/2 clusters of b^3."""
    torch = pytest.importorskip("torch")
    from paper_1405_1931_gb300 import fields
    phi = fields.block_field_device(L, b, device="cpu").numpy()
    labels, sizes, hist, n = oracle.label(phi, (1, 1, 1))
    np.testing.assert_array_equal(labels, closed_forms.block_labels_device(L, b, device="cpu").numpy())
    assert n == (L // b) ** 3 // 2 and (sizes == b ** 3).all()
    assert hist[(b ** 3).bit_length() - 1] == n


def test_checkerboard_odd_periodic_axis():
    """Odd periodic axis: the wrap joins (nx-1, y, z) and (0, y, z), which have the same parity.

    nx=3 periodic, ny=nz=2 not periodic, occupied iff x+y+z even: each (y,z) with y+z even
    gives one cluster {x=0, x=2} of size 2, each with y+z odd gives the single site x=1.
    """
    z, y, x = np.meshgrid(np.arange(2), np.arange(2), np.arange(3), indexing="ij")
    occ = (x + y + z) % 2 == 0
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), (1, 0, 0))
    assert n == 4
    # min indices in raster order: (y,z)=(0,0): site 0 size 2; (1,0): site 4 (x=1) size 1;
    # (0,1): site 7 (x=1,y=0,z=1) size 1; (1,1): site 9 (x=0,y=1,z=1) size 2
    assert sizes.tolist() == [2, 1, 1, 2]
    assert labels[0, 0, 2] == 0 and labels[1, 1, 2] == 9
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), (0, 0, 0))
    assert n == 6 and (sizes == 1).all()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_broken_rod(axis):
    """A rod spanning one axis, broken at one site: 2 clusters open, 1 with that axis periodic."""
    L = 11
    shape = [3, 3, 3]
    shape[2 - axis] = L
    occ = np.zeros(shape, dtype=bool)
    sl = [1, 1, 1]
    sl[2 - axis] = slice(None)
    occ[tuple(sl)] = True
    cut = [1, 1, 1]
    cut[2 - axis] = 4
    occ[tuple(cut)] = False
    per_open = [1, 1, 1]
    per_open[axis] = 0
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), tuple(per_open))
    assert n == 2 and sorted(sizes.tolist()) == [4, 6]
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), (1, 1, 1))
    assert n == 1 and sizes.tolist() == [10]


def test_serpentine_forces_equivalence_chains():
    """A serpentine (one long path folding back and forth) is a single cluster.

    In raster order each new fold starts a fresh label that is only joined to the
    previous ones through rule 3 further down, so the label-of-labels list must
    chain every fold into one class.
    """
    ny, nx = 15, 12
    occ2 = np.zeros((ny, nx), dtype=bool)
    occ2[0::2, :] = True                  # horizontal strokes
    for k, yy in enumerate(range(1, ny, 2)):
        occ2[yy, nx - 1 if k % 2 == 0 else 0] = True   # alternating connectors
    occ = occ2[None, :, :]
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), (0, 0, 0))
    assert n == 1 and sizes.tolist() == [int(occ.sum())]
    # comb: vertical teeth joined only at the bottom row -> each tooth gets its own label first
    comb = np.zeros((1, 9, 13), dtype=bool)
    comb[0, :, 0::2] = True
    comb[0, 8, :] = True
    labels, sizes, hist, n = oracle.label(occ_to_phi(comb), (0, 0, 0))
    assert n == 1 and (labels[comb] == 0).all()


def test_isolated_spheres():
    """Well-separated balls: one cluster each, sizes = directly counted voxels, in raster order."""
    L = 40
    centres = [(8.3, 9.1, 7.7), (30.2, 10.4, 12.9), (12.5, 29.6, 30.1), (31.0, 31.0, 28.4)]
    radii = [5.2, 6.7, 4.9, 6.1]
    g = np.arange(L, dtype=np.float64)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    occ = np.zeros((L, L, L), dtype=bool)
    counts = []
    for (cx, cy, cz), r in zip(centres, radii):
        ball = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 < r * r
        counts.append((int(np.nonzero(ball.reshape(-1))[0].min()), int(ball.sum())))
        occ |= ball
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), (1, 1, 1))
    assert n == 4
    assert sizes.tolist() == [c for _, c in sorted(counts)]


@pytest.mark.parametrize("axes", [(10, 10, 10), (13.5, 21.0, 17.2), (30.0, 12.0, 25.5)])
def test_capsule_two_clusters(axes):
    """Sec. 6 steps 3-4: a closed shell separates interior and exterior -> exactly two clusters."""
    L = 64
    phi = fields.capsule_field(L, axes)
    labels, sizes, hist, n = oracle.label(phi, (1, 1, 1))
    assert n == 2
    interior = closed_forms.capsule_interior_count(L, axes)
    shell = int((phi < 0).sum())
    assert sorted(sizes.tolist()) == sorted([interior, L ** 3 - shell - interior])
    assert labels[0, 0, 0] == 0                        # exterior holds site 0
    assert labels[L // 2, L // 2, L // 2] > 0          # centre is interior


# --------------------------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(v) for v in rng.integers(5, 40, size=3))
    p = float(rng.uniform(0.1, 0.9))
    occ = rng.random(shape) < p
    per = tuple(int(v) for v in rng.integers(0, 2, size=3))
    labels, sizes, hist, n = oracle.label(occ_to_phi(occ), per)
    flat = labels.reshape(-1)
    idx = np.arange(flat.size)
    o = occ.reshape(-1)
    assert sizes.sum() == o.sum()
    assert hist.sum() == n
    assert n <= (flat.size + 1) // 2
    assert (flat[~o] == -1).all()
    assert (flat[o] <= idx[o]).all()
    assert (flat[flat[o]] == flat[o]).all()          # labels name the cluster's own root site
    np.testing.assert_array_equal(np.sort(np.unique(flat[o])), np.sort(np.nonzero(flat == idx)[0]))
    # neighbouring occupied sites share a label (6-connectivity incl. periodic edges)
    for axis, per_a in ((2, per[0]), (1, per[1]), (0, per[2])):
        a = labels
        b = np.roll(labels, -1, axis=axis)
        oa = occ
        ob = np.roll(occ, -1, axis=axis)
        both = oa & ob
        if not per_a:
            last = [slice(None)] * 3
            last[axis] = -1
            both[tuple(last)] = False
        assert (a[both] == b[both]).all()
    np.testing.assert_array_equal(hist, log2_hist(sizes))


def test_capacity_and_arguments():
    phi = occ_to_phi((np.indices((4, 4, 4)).sum(axis=0) % 2) == 0)   # 32 clusters
    labels, sizes, hist, n = oracle.label(phi, (0, 0, 0), sizes_cap=10)
    assert n == 32 and sizes.size == 10 and hist.sum() == 32
    assert oracle.status(phi, (0, 0, 0), sizes_cap=10) == oracle.ERR_CAPACITY
    assert oracle.status(phi, (0, 0, 0), sizes_cap=32) == oracle.OK


def test_singleton_fraction_at_p_c():
    """Statistical sanity (not parity): on a periodic i.i.d. lattice a site is a one-site
    cluster iff it is occupied and its six neighbours are empty, so the expected number of
    size-1 clusters per site is p (1 - p)^6 (0.0332 at p = 0.3116).  64^3 sites: within 4 %."""
    from paper_1405_1931_gb300 import fields
    p = 0.3116
    phi = fields.iid_field(64, 64, 64, seed=4, occupancy=p)
    labels, sizes, hist, n = oracle.label(phi, (1, 1, 1))
    occ = phi > 0
    assert hist[0] == int((sizes == 1).sum())
    per_site = hist[0] / phi.size
    assert abs(per_site - p * (1 - p) ** 6) < 0.04 * p * (1 - p) ** 6
    # and directly from the definition on the same lattice
    empty_nbrs = np.ones_like(occ)
    for axis in range(3):
        for d in (-1, 1):
            empty_nbrs &= ~np.roll(occ, d, axis=axis)
    assert hist[0] == int((occ & empty_nbrs).sum())


def test_gyroid_labyrinths_are_one_cluster_each():
    """A bijel is one cluster (Sec. 5).  The stand-in is the gyroid
    sin x cos y + sin y cos z + sin z cos x over one period: each of its two interpenetrating
    labyrinths is connected, so phi > 0 and phi < 0 are one cluster each, with and without
    periodic edges."""
    for L in (24, 32):
        t = 2 * np.pi * np.arange(L) / L
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        phi = (np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)).astype(np.float32)
        for per in [(1, 1, 1), (0, 0, 0)]:
            for f in (phi, -phi):
                labels, sizes, hist, n = oracle.label(f, per)
                assert n == 1 and sizes[0] == int((f > 0).sum())
