"""Host logic of the autotuner on the CPU: batch signatures and the cache path (a
cached batch sets its tile shape and merge schedule without timing anything)."""
import json

import pytest

from paper_1405_1931_gb300 import autotune

torch = pytest.importorskip("torch")


def items(shapes):
    return [(torch.empty(s, dtype=torch.float32), (1, 1, 1), None) for s in shapes]


def test_signature_rounds_to_powers_of_two():
    a = autotune.signature(items([(40, 50, 60), (10, 10, 10)]))
    b = autotune.signature(items([(33, 63, 35), (12, 9, 11)]))     # same rounded counts and largest shape
    assert a == b
    assert a.startswith("n2_")
    assert autotune.signature(items([(64, 64, 64)])) != autotune.signature(items([(64, 64, 128)]))


def test_cached_batch_sets_its_schedule(tmp_path):
    batch = items([(32, 48, 64)])
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({autotune.signature(batch): {"tile": [32, 8], "merge": [4, 0],
                                                              "ms": {"32x8/u4h0": 1.0}}}))

    class Lab:
        tile = None
        merge = None

        def set_tile(self, ty, tz):
            self.tile = (ty, tz)

        def set_merge(self, u, h):
            self.merge = (u, h)

    lab = Lab()
    got = autotune.tune(lab, batch, cache=str(cache))
    assert got["cached"] and got["tile"] == (32, 8) and lab.tile == (32, 8)
    assert got["merge"] == (4, 0) and lab.merge == (4, 0)


def test_candidates_cover_every_tile_and_schedule():
    assert set(autotune.TILES) == {(8, 8), (16, 8), (16, 16), (32, 8)}
    assert {u for u, _ in autotune.MERGES} == {1, 2, 4} and {h for _, h in autotune.MERGES} == {0, 1}
    assert autotune.DEFAULT_MERGE in autotune.MERGES
