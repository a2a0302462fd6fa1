"""Parity of the CUDA path with the oracle, element by element, through the C ABI.

Labels, sizes, histogram and cluster count must be bit-identical (the output
is integer and unique).  Inputs are seeded host fields uploaded to the device,
so the oracle always labels exactly the bytes the GPU labels.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1405_1931_gb300 import fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILES = [(8, 8), (16, 8), (16, 16), (32, 8)]
PERIODIC_ALL = list(itertools.product((0, 1), repeat=3))


@pytest.fixture(scope="module")
def labeller():
    """The tiled passes for every lattice (the one-CTA path for small lattices is tested in
    test_gpu_small.py)."""
    from paper_1405_1931_gb300.hk import Labeller
    lab = Labeller(0)
    lab.set_small_path(False)
    yield lab
    lab.close()


def gpu_label(lab, phi_np, per, sizes_cap=None):
    phi = torch.from_numpy(np.ascontiguousarray(phi_np)).cuda()
    labels, sizes, hist, ncl = lab.label(phi, per, sizes_cap=sizes_cap)
    lab.sync_status()
    n = int(ncl.item())
    cap = sizes.numel() if sizes_cap is None else sizes_cap
    return labels.cpu().numpy(), sizes[:min(n, cap)].cpu().numpy(), hist.cpu().numpy(), n


def assert_parity(lab, phi_np, per, what=""):
    want = oracle.label(phi_np, per)
    got = gpu_label(lab, phi_np, per)
    assert got[3] == want[3], f"{what}: n_clusters {got[3]} != {want[3]}"
    np.testing.assert_array_equal(got[0], want[0], err_msg=f"{what}: labels")
    np.testing.assert_array_equal(got[1], want[1], err_msg=f"{what}: sizes")
    np.testing.assert_array_equal(got[2], want[2], err_msg=f"{what}: hist")


@pytest.mark.parametrize("tile", TILES)
def test_small_iid_all_tiles(labeller, tile):
    """32^3, occupancy 0.3, seed 0, periodic in x, y, z -- every tile shape."""
    labeller.set_tile(*tile)
    phi, per = fields.small_iid()
    for p in PERIODIC_ALL:
        assert_parity(labeller, phi, p, f"tile {tile} per {p}")
    labeller.set_tile(16, 16)


SHAPES = [(1, 1, 1), (2, 2, 2), (1, 1, 40), (40, 1, 1), (1, 37, 1), (33, 1, 1), (5, 7, 3), (31, 17, 9),
          (32, 16, 16), (33, 17, 17), (64, 32, 32), (65, 9, 70), (96, 40, 24), (100, 33, 47), (2, 64, 3)]


@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes_all_periodic(labeller, shape):
    """Several tiles per axis with ragged tails, axis lengths 1 and 2, all 8 periodic sets."""
    nx, ny, nz = shape
    for i, p in enumerate((0.2, 0.3116, 0.6)):
        phi = fields.iid_field(nx, ny, nz, seed=17 + i, occupancy=p)
        for per in PERIODIC_ALL:
            assert_parity(labeller, phi, per, f"{shape} p={p} per={per}")


@pytest.mark.parametrize("tile", TILES)
def test_ragged_shapes_other_tiles(labeller, tile):
    labeller.set_tile(*tile)
    for shape in [(70, 45, 19), (33, 9, 65), (128, 64, 40)]:
        phi = fields.iid_field(*shape, seed=5, occupancy=0.3116)
        for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1), (0, 1, 0)]:
            assert_parity(labeller, phi, per, f"tile {tile} {shape} {per}")
    labeller.set_tile(16, 16)


def test_empty_full_and_signed_zero(labeller):
    for shape in [(1, 1, 1), (37, 19, 23), (64, 64, 64)]:
        nx, ny, nz = shape
        for v in (-1.0, 0.0, -0.0, 1.0):
            phi = np.full((nz, ny, nx), v, dtype=np.float32)
            for per in [(0, 0, 0), (1, 1, 1)]:
                assert_parity(labeller, phi, per, f"{shape} const {v}")
    phi = np.array([0.0, -0.0, np.nan, 1e-45, -1e-45, np.inf, 1.0, -np.inf], dtype=np.float32)
    phi = np.tile(phi, 8).reshape(1, 1, 64)
    assert_parity(labeller, phi, (1, 1, 1), "special values")


def test_max_clusters_checkerboard(labeller):
    """n_cl,max = V/2 (single sites alternating along every axis)."""
    for shape in [(64, 32, 32), (33, 17, 5), (96, 48, 16)]:
        nx, ny, nz = shape
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        phi = np.where((x + y + z) % 2 == 0, 1.0, -1.0).astype(np.float32)
        for per in PERIODIC_ALL:
            assert_parity(labeller, phi, per, f"checkerboard {shape} {per}")


def test_mixed_run_density_tiles(labeller):
    """Tiles of very different run counts in one lattice: sparse random tiles next to
    checkerboard tiles (16 runs a row) and tiles whose rows alternate between 16 runs
    and one full run (few runs, but 16 union pairs a row along y and z), so that the
    dense tiles are labelled by the second tile pass and joined to the others."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 133, 67, 71
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kind = rng.integers(0, 4, size=((nz + 15) // 16, (ny + 15) // 16, (nx + 31) // 32))
    k = kind[z // 16, y // 16, x // 32]
    occ = rng.random((nz, ny, nx)) < 0.3                      # kind 0: p = 0.3
    occ = np.where(k == 1, (x + y + z) % 2 == 0, occ)         # kind 1: checkerboard
    occ = np.where(k == 2, (y % 2 == 1) | (x % 2 == 0), occ)  # kind 2: 16-run rows under full rows
    occ = np.where(k == 3, rng.random((nz, ny, nx)) < 0.6, occ)
    phi = np.where(occ, 1.0, -1.0).astype(np.float32)
    for tile in TILES:
        labeller.set_tile(*tile)
        for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
            assert_parity(labeller, phi, per, f"mixed density tile {tile} {per}")
    labeller.set_tile(16, 16)


def test_many_boundary_pieces(labeller):
    """Short rods along z on the (x + y) even columns, three sites at each end of
    every 8-plane slab: with 32x32x8 tiles each tile holds 1024 boundary pieces
    (two per column, each joined to the next slab across the z face)."""
    nx, ny, nz = 64, 64, 24
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    occ = ((x + y) % 2 == 0) & np.isin(z % 8, [0, 1, 2, 5, 6, 7])
    phi = np.where(occ, 1.0, -1.0).astype(np.float32)
    for tile in TILES:
        labeller.set_tile(*tile)
        for per in [(0, 0, 0), (1, 1, 1)]:
            assert_parity(labeller, phi, per, f"boundary pieces tile {tile} {per}")
    labeller.set_tile(16, 16)


def test_block_pattern_and_rods(labeller):
    nx, ny, nz = 64, 48, 40
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.where(((x // 8) + (y // 6) + (z // 5)) % 2 == 0, 1.0, -1.0).astype(np.float32)
    for per in PERIODIC_ALL:
        assert_parity(labeller, phi, per, f"blocks {per}")
    # long rods along each axis crossing many tiles, broken once
    for axis in range(3):
        shape = [20, 20, 20]
        shape[2 - axis] = 200
        occ = np.zeros(shape, dtype=bool)
        sl = [7, 11, 3]
        sl[2 - axis] = slice(None)
        occ[tuple(sl)] = True
        cut = [7, 11, 3]
        cut[2 - axis] = 77
        occ[tuple(cut)] = False
        phi = np.where(occ, 1.0, -1.0).astype(np.float32)
        for per in PERIODIC_ALL:
            assert_parity(labeller, phi, per, f"rod axis {axis} {per}")


def test_spiral_across_tiles(labeller):
    """A serpentine spanning many tiles: long chains of cross-tile unions."""
    ny, nx = 150, 130
    occ2 = np.zeros((ny, nx), dtype=bool)
    occ2[0::2, :] = True
    for k, yy in enumerate(range(1, ny, 2)):
        occ2[yy, nx - 1 if k % 2 == 0 else 0] = True
    phi = np.where(np.repeat(occ2[None], 3, axis=0), 1.0, -1.0).astype(np.float32)
    for per in [(0, 0, 0), (1, 1, 1)]:
        assert_parity(labeller, phi, per, "serpentine")


def test_capsule_and_emulsion_small(labeller):
    phi = fields.capsule_field(96, (40.0, 25.5, 33.3))
    assert_parity(labeller, phi, (1, 1, 1), "capsule")
    phi = fields.emulsion_field(96, 80, 64, 40, seed=1)
    assert_parity(labeller, phi, (1, 1, 1), "emulsion small")


def test_emulsion_256(labeller):
    """256^3 emulsion-like field: 600 droplets, r in [5, 15], periodic."""
    phi, per = fields.emulsion_256()
    assert_parity(labeller, phi, per, "emulsion 256")


def test_critical_256(labeller):
    phi = fields.iid_field(256, 256, 256, seed=0, occupancy=fields.P_C_SIMPLE_CUBIC)
    assert_parity(labeller, phi, (1, 1, 1), "critical 256")


def test_capacity_error_keeps_labels(labeller):
    from paper_1405_1931_gb300.hk import HKError, HK_ERR_CAPACITY
    phi = fields.iid_field(48, 40, 24, seed=9, occupancy=0.25)
    want = oracle.label(phi, (1, 1, 1))
    cap = want[3] // 3
    d = torch.from_numpy(phi).cuda()
    out = labeller.alloc_outputs(d.shape, d.device, sizes_cap=cap)
    with pytest.raises(HKError) as ei:
        labeller.label(d, (1, 1, 1), out=out)
    assert ei.value.status == HK_ERR_CAPACITY
    labels, sizes, hist, ncl, _ = out
    torch.cuda.synchronize()
    assert int(ncl.item()) == want[3]
    np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
    np.testing.assert_array_equal(sizes[:cap].cpu().numpy(), want[1][:cap])
    np.testing.assert_array_equal(hist.cpu().numpy(), want[2])


def test_host_buffer_entry(labeller):
    phi = fields.iid_field(100, 60, 50, seed=4, occupancy=0.3116)
    want = oracle.label(phi, (1, 0, 1))
    got = labeller.label_host(phi, (1, 0, 1))
    assert got[3] == want[3]
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    np.testing.assert_array_equal(got[2], want[2])


def _batch_items(params):
    items, phis = [], []
    for prm in params:
        phi = fields.iid_field(prm["nx"], prm["ny"], prm["nz"], seed=prm["seed"], occupancy=prm["occupancy"])
        phis.append(phi)
    return phis


def test_batched_matches_oracle_and_single(labeller):
    """Uneven batch (shapes from the batch recipe, axes capped at 160 to keep the oracle quick)."""
    params = fields.batch_params(24, master_seed=2)
    for prm in params:
        prm["nx"], prm["ny"], prm["nz"] = (min(prm[k], 160) for k in ("nx", "ny", "nz"))
    phis = _batch_items(params)
    items, outs = [], []
    for prm, phi in zip(params, phis):
        d = torch.from_numpy(phi).cuda()
        out = labeller.alloc_outputs(d.shape, d.device)
        items.append((d, prm["periodic"], out))
        outs.append(out)
    labeller.label_batched(items)
    labeller.sync_status()
    for prm, phi, (labels, sizes, hist, ncl, cap) in zip(params, phis, outs):
        want = oracle.label(phi, prm["periodic"])
        n = int(ncl.item())
        assert n == want[3]
        np.testing.assert_array_equal(labels.cpu().numpy(), want[0])
        np.testing.assert_array_equal(sizes[:n].cpu().numpy(), want[1])
        np.testing.assert_array_equal(hist.cpu().numpy(), want[2])


def test_batched_more_than_one_launch_chunk(labeller):
    """More lattices than fit in one launch's descriptor table (split into chunks)."""
    from paper_1405_1931_gb300.hk import Labeller
    rng = np.random.default_rng(1)
    items, phis, pers = [], [], []
    for i in range(140):
        shape = tuple(int(v) for v in rng.integers(1, 40, size=3))
        phi = fields.iid_field(*shape, seed=300 + i, occupancy=float(rng.uniform(0.15, 0.6)))
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


def test_device_generator_matches_host():
    from paper_1405_1931_gb300 import hk
    nx, ny, nz = 70, 33, 21
    d = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    assert hk.hk_gen_iid(d.data_ptr(), nx, ny, nz, 7, 0.3116, 0) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), fields.iid_field(nx, ny, nz, seed=7, occupancy=0.3116))
    L = 64
    c = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    assert hk.hk_gen_capsule(c.data_ptr(), L, 20.0, 13.5, 17.25, 0) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c.cpu().numpy(), fields.capsule_field(L, (20.0, 13.5, 17.25)))
