"""The one-launch path for small lattices against the oracle, element by element.

Two kernels (hk_small.cu): one CTA holds a lattice of at most 32768 sites and 2048
row segments in shared memory; a cluster of 16 CTAs (8 where the device cannot
co-schedule 16) holds a lattice whose rows, cut into that many blocks, come to at
most 1024 row segments a block, the CTAs reaching each other's runs through
distributed shared memory.  Under each kernel alone, labels,
sizes, histogram and count must equal the oracle's exactly on every shape and
periodic set it takes: axes of length 1 and 2, ragged x, the size limits, the site
checkerboard with its V/2 clusters at the limit, empty and full lattices, and
batches of more lattices than one launch holds.  Lattices just beyond a limit take
the tiled passes, also checked.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PERIODIC_ALL = list(itertools.product((0, 1), repeat=3))


@pytest.fixture(scope="module", params=[("one_cta", 2), ("cluster", 3)], ids=lambda p: p[0])
def labeller(request):
    """A context whose small path uses one kernel only."""
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_small_path(request.param[1])
    yield lab
    lab.close()


@pytest.fixture(scope="module")
def cluster_labeller():
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_small_path(3)
    yield lab
    lab.close()


def gpu_label(lab, phi_np, per):
    phi = torch.from_numpy(np.ascontiguousarray(phi_np)).cuda()
    labels, sizes, hist, ncl = lab.label(phi, per)
    lab.sync_status()
    n = int(ncl.item())
    return labels.cpu().numpy(), sizes[:n].cpu().numpy(), hist.cpu().numpy(), n


def assert_parity(lab, phi_np, per, what=""):
    want = oracle.label(phi_np, per)
    got = gpu_label(lab, phi_np, per)
    assert got[3] == want[3], f"{what}: n_clusters {got[3]} != {want[3]}"
    np.testing.assert_array_equal(got[0], want[0], err_msg=f"{what}: labels")
    np.testing.assert_array_equal(got[1], want[1], err_msg=f"{what}: sizes")
    np.testing.assert_array_equal(got[2], want[2], err_msg=f"{what}: hist")


SMALL_SHAPES = [(1, 1, 1), (2, 2, 2), (1, 1, 40), (40, 1, 1), (1, 37, 1), (33, 1, 1), (5, 7, 3), (31, 17, 9),
                (32, 16, 16), (33, 17, 17), (64, 32, 16), (65, 9, 30), (100, 13, 7), (2, 64, 3), (1, 128, 16),
                (32, 32, 32), (16, 32, 64), (96, 20, 17)]


@pytest.mark.parametrize("shape", SMALL_SHAPES)
def test_small_shapes_all_periodic(labeller, shape):
    from paper_1405_1931_gb300 import hk
    nx, ny, nz = shape
    assert nx * ny * nz <= 32768
    for i, p in enumerate((0.2, 0.3116, 0.6)):
        phi = fields.iid_field(nx, ny, nz, seed=41 + i, occupancy=p)
        for per in PERIODIC_ALL:
            assert_parity(labeller, phi, per, f"{shape} p={p} per={per}")


def test_small_special_patterns(labeller):
    # the site checkerboard at both limits: V/2 clusters of one site (16384 runs)
    for shape in [(32, 32, 32), (16, 32, 64)]:
        nx, ny, nz = shape
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        chk = np.where((x + y + z) % 2 == 0, 1.0, -1.0).astype(np.float32)
        for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
            assert_parity(labeller, chk, per, f"checkerboard {shape} {per}")
        assert_parity(labeller, -chk, (1, 1, 1), f"shifted checkerboard {shape}")
    # empty, full, one site
    for shape in [(32, 32, 32), (7, 5, 3)]:
        nx, ny, nz = shape
        assert_parity(labeller, np.full((nz, ny, nx), -1.0, np.float32), (1, 1, 1), "empty")
        assert_parity(labeller, np.full((nz, ny, nx), 1.0, np.float32), (1, 1, 1), "full")
        assert_parity(labeller, np.full((nz, ny, nx), 1.0, np.float32), (0, 0, 0), "full open")
    one = np.full((4, 5, 6), -1.0, np.float32)
    one[2, 3, 4] = 0.5
    assert_parity(labeller, one, (1, 1, 1), "one site")
    # serpentine along x through every row: one long cluster, long union chains
    nx, ny, nz = 32, 32, 32
    phi = np.full((nz, ny, nx), -1.0, np.float32)
    phi[:, ::2, :] = 1.0
    phi[:, 1::4, -1] = 1.0
    phi[:, 3::4, 0] = 1.0
    assert_parity(labeller, phi, (0, 0, 0), "serpentine")
    assert_parity(labeller, phi, (1, 1, 1), "serpentine periodic")


def test_just_beyond_the_one_cta_limit(labeller):
    """Lattices just beyond the one-CTA kernel's limits: the one-CTA context labels them
    with the tiled passes, the cluster context with the cluster kernel where they fit it
    (the last, 32769 rows of one segment, fits neither)."""
    for shape in [(33, 993, 1), (32, 32, 33), (1, 1, 32769)]:
        phi = fields.iid_field(*shape, seed=7, occupancy=0.3116)
        for per in [(1, 1, 1), (0, 1, 0)]:
            assert_parity(labeller, phi, per, f"beyond the limit {shape} {per}")


def test_small_path_equals_tiled_passes():
    from paper_1405_1931_gb300.hk import Labeller
    a, b = Labeller(0), Labeller(0)
    b.set_small_path(False)
    for shape, p in [((32, 32, 32), 0.3116), ((17, 40, 25), 0.45), ((64, 16, 30), 0.25)]:
        phi = torch.from_numpy(fields.iid_field(*shape, seed=5, occupancy=p)).cuda()
        ra = a.label(phi, (1, 0, 1))
        rb = b.label(phi, (1, 0, 1))
        torch.cuda.synchronize()
        n = int(ra[3].item())
        assert n == int(rb[3].item())
        assert torch.equal(ra[0], rb[0]) and torch.equal(ra[1][:n], rb[1][:n]) and torch.equal(ra[2], rb[2])
    a.close()
    b.close()


def test_small_batch_over_one_launch(labeller):
    """100 small lattices (two launches of at most 64 lattices), every output against the oracle."""
    rng = np.random.default_rng(9)
    items, phis, pers = [], [], []
    for i in range(100):
        shape = tuple(int(v) for v in rng.integers(1, 33, size=3))
        phi = fields.iid_field(*shape, seed=500 + i, occupancy=float(rng.uniform(0.15, 0.6)))
        per = tuple(int(v) for v in rng.integers(0, 2, size=3))
        d = torch.from_numpy(phi).cuda()
        items.append((d, per, labeller.alloc_outputs(d.shape, d.device)))
        phis.append(phi)
        pers.append(per)
    labeller.label_batched(items)
    labeller.sync_status()
    for (d, per, (labels, sizes, hist, ncl, cap)), phi in zip(items, phis):
        want = oracle.label(phi, per)
        n = int(ncl.item())
        assert n == want[3]
        np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
        np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1])
        np.testing.assert_array_equal(hist.cpu().numpy(), want[2])


def test_small_capacity_rule(labeller):
    phi_np = fields.iid_field(32, 32, 32, seed=3, occupancy=0.3)
    want = oracle.label(phi_np, (1, 1, 1))
    n = want[3]
    from paper_1405_1931_gb300 import hk
    phi = torch.from_numpy(phi_np).cuda()
    out = labeller.alloc_outputs(phi.shape, phi.device, sizes_cap=n)
    labeller.label(phi, (1, 1, 1), out=out)
    np.testing.assert_array_equal(out[1][:n].cpu().numpy(), want[1])
    short = labeller.alloc_outputs(phi.shape, phi.device, sizes_cap=n - 1)
    with pytest.raises(hk.HKError) as e:
        labeller.label(phi, (1, 1, 1), out=short)
    assert e.value.status == hk.HK_ERR_CAPACITY
    np.testing.assert_array_equal(short[0].cpu().numpy(), want[0])
    assert int(short[3].item()) == n


CLUSTER_SHAPES = [(64, 64, 64), (96, 32, 48), (64, 1, 4096), (40, 70, 30), (1, 2048, 4), (33, 8, 500),
                  (3, 5, 7), (32, 1, 9), (64, 96, 80)]


def cluster_fits(nx, ny, nz, blocks=8):
    """The cluster kernel's limit as include/hk.h states it: the rows cut into equal
    blocks (8, or 16 on a device that runs clusters of 16) come to at most 1024 row
    segments (32 sites along x) a block."""
    return -(-ny * nz // blocks) * -(-nx // 32) <= 1024


@pytest.mark.parametrize("shape", CLUSTER_SHAPES)
def test_cluster_shapes(cluster_labeller, shape):
    """Lattices the one-CTA kernel cannot hold (and a few tiny ones, with CTAs left
    without rows): rows split unevenly over the 8 CTAs, rows crossing CTAs through every
    periodic edge, the segment limit of a CTA reached exactly."""
    nx, ny, nz = shape
    assert cluster_fits(nx, ny, nz, blocks=16)
    for i, p in enumerate((0.2, 0.3116, 0.55)):
        phi = fields.iid_field(nx, ny, nz, seed=61 + i, occupancy=p)
        for per in [(1, 1, 1), (0, 0, 0), (1, 0, 1), (0, 1, 1)]:
            assert_parity(cluster_labeller, phi, per, f"{shape} p={p} per={per}")


def test_cluster_special_patterns(cluster_labeller):
    # the site checkerboard at 64^3: 131072 clusters of one site, 16384 runs per CTA (the limit)
    nx = ny = nz = 64
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    chk = np.where((x + y + z) % 2 == 0, 1.0, -1.0).astype(np.float32)
    for per in [(1, 1, 1), (0, 0, 0)]:
        assert_parity(cluster_labeller, chk, per, f"checkerboard 64^3 {per}")
    # one cluster through every CTA: a serpentine along x and y in every plane, planes
    # joined at one corner each, so the union chains cross every CTA boundary
    phi = np.full((nz, ny, nx), -1.0, np.float32)
    phi[:, ::2, :] = 1.0
    phi[:, 1::4, -1] = 1.0
    phi[:, 3::4, 0] = 1.0
    assert_parity(cluster_labeller, phi, (0, 0, 0), "serpentine planes")
    phi[:, :, :] = -1.0
    phi[:, 0, 0] = 1.0        # a column along z: one cluster spanning all 8 CTAs, joined by the wrap
    assert_parity(cluster_labeller, phi, (0, 0, 1), "z column periodic")
    assert_parity(cluster_labeller, phi, (0, 0, 0), "z column open")
    full = np.full((nz, ny, nx), 1.0, np.float32)
    assert_parity(cluster_labeller, full, (1, 1, 1), "full")


def test_cluster_limit_and_beyond():
    """Lattices at the cluster kernel's limits -- the largest that fit 8 blocks, the
    largest that fit 16 (a device that runs clusters of 8 labels these with the tiled
    passes) -- and the first beyond both (the tiled passes); all against the oracle."""
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    for shape, fits8 in [((32, 1, 8192), True), ((32, 1, 8193), False), ((64, 64, 65), False), ((32, 1, 16384), False),
                         ((32, 1, 16385), False), ((64, 128, 128), False)]:
        assert cluster_fits(*shape) == fits8
        phi = fields.iid_field(*shape, seed=71, occupancy=0.3116)
        assert_parity(lab, phi, (1, 1, 1), f"cluster limit {shape}")
    lab.close()


def test_cluster_batches():
    """Batches through the cluster kernel: a few lattices of mixed shapes (clusters by
    default), and more lattices than the cluster threshold that only the cluster holds."""
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    rng = np.random.default_rng(13)
    for count, lo, hi in ((5, 8, 64), (20, 40, 64)):
        items, phis, pers = [], [], []
        for i in range(count):
            shape = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
            phi = fields.iid_field(*shape, seed=800 + 37 * count + i, occupancy=float(rng.uniform(0.2, 0.5)))
            per = tuple(int(v) for v in rng.integers(0, 2, size=3))
            d = torch.from_numpy(phi).cuda()
            items.append((d, per, lab.alloc_outputs(d.shape, d.device)))
            phis.append(phi)
            pers.append(per)
        lab.label_batched(items)
        lab.sync_status()
        for (d, per, (labels, sizes, hist, ncl, cap)), phi in zip(items, phis):
            want = oracle.label(phi, per)
            n = int(ncl.item())
            assert n == want[3]
            np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
            np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1])
            np.testing.assert_array_equal(hist.cpu().numpy(), want[2])
    lab.close()


@pytest.mark.parametrize("mode", [2, 3], ids=["one_cta", "cluster"])
def test_small_kernels_capped_unions_report_or_are_exact(mode):
    """With the union retries capped at one (hk_set_loop_cap), each call of a small-path
    kernel either reports the cap through the status word or returns exact results; at
    the natural bound every call is exact and the status stays clear."""
    from paper_1405_1931_gb300 import hk
    lab = hk.Labeller(0)
    lab.set_small_path(mode)
    shapes = [(32, 32, 32), (64, 64, 64)] if mode == 3 else [(32, 32, 32), (16, 32, 64)]
    for shape in shapes:
        for i, p in enumerate((0.3116, 0.45)):
            phi = fields.iid_field(*shape, seed=90 + i, occupancy=p)
            want = oracle.label(phi, (1, 1, 1))
            lab.set_loop_cap(1)
            got = gpu_label_raw(lab, phi, (1, 1, 1))
            rc = hk.hk_sync_status(lab.ctx, hk._stream_handle(None))
            assert rc in (hk.HK_OK, hk.HK_ERR_TIMEOUT)
            if rc == hk.HK_OK:
                assert got[3] == want[3]
                np.testing.assert_array_equal(got[0], want[0])
            lab.set_loop_cap(0)
            got = gpu_label_raw(lab, phi, (1, 1, 1))
            assert hk.hk_sync_status(lab.ctx, hk._stream_handle(None)) == hk.HK_OK
            assert got[3] == want[3]
            np.testing.assert_array_equal(got[0], want[0])
            np.testing.assert_array_equal(got[1], want[1])
            np.testing.assert_array_equal(got[2], want[2])
    lab.close()


def gpu_label_raw(lab, phi_np, per):
    """Labels without reading the status word (the caller reads it)."""
    phi = torch.from_numpy(np.ascontiguousarray(phi_np)).cuda()
    labels, sizes, hist, ncl = lab.label(phi, per)
    torch.cuda.synchronize()
    n = int(ncl.item())
    return labels.cpu().numpy(), sizes[:n].cpu().numpy(), hist.cpu().numpy(), n
