"""Planted mistakes: the pins must reject every plausible slip in the oracle.

Each case copies ``oracle/hk_oracle.c``, applies one textual mutation (a dropped
term, a wrong sign or index, a swapped operand), compiles the copy to a
temporary library on the CPU and runs a fast battery of the pins from
``test_oracle_pins.py``.  The battery must fail for every mutant and pass for
the unmodified source.
"""
import itertools
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from brute import bfs_label, interior_state, interior_tags, log2_hist

SRC = os.path.join(os.path.dirname(oracle.__file__), "hk_oracle.c")

MUTATIONS = {
    "drop_z_neighbour": ("if (z > 0 && l[s - sz] > 0) nb[n_nb++] = l[s - sz];", ""),
    "drop_y_neighbour": ("if (y > 0 && l[s - sy] > 0) nb[n_nb++] = l[s - sy];\n                if (z > 0 &&",
                         "if (z > 0 &&"),
    # (taking the max instead of the min in rule 3 is an equivalent mutant: the final
    # relabelling reduces every id to its class minimum, so it is not listed)
    "rule3_first_pair_only": ("for (int j = i + 1; j < n_nb; ++j)\n                            store_equivalence(t.lol",
                              "for (int j = i + 1; j < 2; ++j)\n                            store_equivalence(t.lol"),
    "rule3_no_equivalence": ("store_equivalence(t.lol, nb[i], nb[j]);", "(void)j;"),
    "link_larger_end_wrong_way": ("if (ea < eb) lol[eb] = ea;", "if (ea < eb) lol[ea] = eb;"),
    "occupancy_ge": ("(phi[s] > 0.0f) ? -1 : 0", "(phi[s] >= 0.0f) ? -1 : 0"),
    "drop_x_wrap": ("if (periodic[0] && nx >= 2)", "if (0)"),
    "drop_z_wrap": ("if (periodic[2] && nz >= 2)", "if (0)"),
    "wrap_off_by_one": ("                int64_t a = x * sx + (ny - 1) * sy + z * sz",
                        "                int64_t a = x * sx + (ny - 2) * sy + z * sz"),
    "wrap_axis_swapped": ("if (periodic[1] && ny >= 2)", "if (periodic[0] && ny >= 2)"),
    "hist_off_by_one": ("while (((int64_t)2 << b) <= size) ++b;", "while (((int64_t)1 << b) <= size) ++b;"),
    "label_is_compact_id": ("l[s] = (int32_t)t.first[root];", "l[s] = compact[root];"),
    "sizes_shifted": ("if (c - 1 < sizes_cap) sizes_out[c - 1] = size;",
                      "if (c - 1 < sizes_cap) sizes_out[(c % n)] = size;"),
    "raster_y_stride": ("const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;\n    const int64_t N =",
                        "const int64_t sx = 1, sy = ny, sz = (int64_t)nx * ny;\n    const int64_t N ="),
    # interior/exterior identification (Sec. 6, steps 3-5)
    "interior_vote_sign": ("const int sign = (v < 0.0f) ? -1 : (v > 0.0f) ? 1 : 0;",
                           "const int sign = (v < 0.0f) ? 1 : (v > 0.0f) ? -1 : 0;"),
    "interior_far_le": ("far[s] = (index[s] < -0.5f) ? 1.0f : -1.0f;", "far[s] = (index[s] <= -0.5f) ? 1.0f : -1.0f;"),
    "interior_no_vote_wrap": ("if (!periodic[axis]) continue;", "continue;"),
    "interior_tag_swapped": ("(int8_t)(votes[k] < 0 ? 1 : votes[k] > 0 ? 0 : -1)",
                             "(int8_t)(votes[k] < 0 ? 1 : votes[k] > 0 ? 0 : 1)"),
    "interior_vote_x_only": ("for (int axis = 0; axis < 3; ++axis)", "for (int axis = 0; axis < 1; ++axis)"),
    # per-site interior state and its incremental update (Sec. 6)
    "state_near_side_le": ("return (int8_t)(v < 0.0f ? 1 : 0);", "return (int8_t)(v <= 0.0f ? 1 : 0);"),
    "state_far_takes_side": ("(index[s] < -0.5f) ? inside[rank[labels[s]]] : near_side(index[s]);",
                             "(index[s] < -0.5f) ? near_side(index[s]) : near_side(index[s]);"),
    "update_keeps_near_sites": ("state_out[s] = (index[s] < -0.5f) ? state_prev[s] : near_side(index[s]);",
                                "state_out[s] = state_prev[s];"),
    "update_far_le": ("state_out[s] = (index[s] < -0.5f) ? state_prev[s] : near_side(index[s]);",
                      "state_out[s] = (index[s] <= -0.5f) ? state_prev[s] : near_side(index[s]);"),
    # the paper's parallel scheme on host threads (Sec. 3)
    "mt_drop_halo": ("if (la > 0 && lb > 0) {", "if (0) {"),
    "mt_no_z_wrap": ("((J->periodic[2] && J->nz >= 2 && J->P >= 2) ? 0 : -1)", "(-1)"),
    "mt_offset_collides": ("D->rc = mt_push_pair(D, w * n_max + la, next * n_max + lb);",
                           "D->rc = mt_push_pair(D, la, lb);"),
    # droplet-size histogram by R_c (Fig. 5)
    "rc_bin_shift": ("if (V >= ((e * e) * e) * four_thirds_pi) bin = b + 1;", "if (V >= ((e * e) * e) * four_thirds_pi) bin = b;"),
    "rc_radius_not_cubed": ("if (V >= ((e * e) * e) * four_thirds_pi) bin = b + 1;",
                            "if (V >= (e * e) * four_thirds_pi) bin = b + 1;"),
}


def battery(lib):
    """Fast subset of the pins; raises AssertionError on the first disagreement."""
    def lab(occ, per):
        return oracle.label(np.where(occ, 1.0, -1.0).astype(np.float32), per, lib=lib)

    def same(got, want):
        assert got[3] == want[3]
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
        np.testing.assert_array_equal(got[2], want[2])

    pers = list(itertools.product((0, 1), repeat=3))
    for bits in range(256):
        occ = np.array([(bits >> i) & 1 for i in range(8)], dtype=bool).reshape(2, 2, 2)
        for per in pers:
            same(lab(occ, per), bfs_label(occ, per))
    rng = np.random.default_rng(5)
    for _ in range(30):
        shape = tuple(int(v) for v in rng.integers(1, 7, size=3))
        occ = rng.random(shape) < rng.uniform(0.2, 0.8)
        for per in pers:
            same(lab(occ, per), bfs_label(occ, per))
    # non-square shapes with distinct axis lengths
    for shape in [(3, 5, 7), (7, 3, 5), (4, 6, 9)]:
        occ = rng.random(shape) < 0.55
        for per in pers:
            same(lab(occ, per), bfs_label(occ, per))
    # occupancy rule on signed zeros
    phi = np.array([0.0, -0.0, 1.0, 0.0], dtype=np.float32).reshape(1, 1, 4)
    got = oracle.label(phi, (0, 0, 0), lib=lib)
    assert got[3] == 1 and got[0].reshape(-1).tolist() == [-1, -1, 2, -1]
    # histogram of a known size set: clusters of sizes 1, 2, 3, 4 along a row
    row = np.array([1, 0, 1, 1, 0, 1, 1, 1, 0, 1, 1, 1, 1], dtype=bool).reshape(1, 1, 13)
    got = lab(row, (0, 0, 0))
    assert got[1].tolist() == [1, 2, 3, 4]
    np.testing.assert_array_equal(got[2], log2_hist([1, 2, 3, 4]))
    # interior/exterior tags against the brute-force votes
    values = np.array([-1.0, -0.5, -0.25, 0.0, 0.25, np.nan], dtype=np.float32)
    for it in range(40):
        shape = tuple(int(v) for v in rng.integers(1, 6, size=3))
        I = values[rng.choice(len(values), size=shape, p=[0.5, 0.05, 0.2, 0.05, 0.15, 0.05])]
        per = pers[it % 8]
        got = oracle.interior(I, per, lib=lib)
        want = interior_tags(I, per)
        same(got[:4], want[:4])
        np.testing.assert_array_equal(got[4], want[4])
    # per-site interior state against the brute-force one, and the update rule by hand
    for it in range(30):
        shape = tuple(int(v) for v in rng.integers(1, 6, size=3))
        I = values[rng.choice(len(values), size=shape, p=[0.5, 0.05, 0.2, 0.05, 0.15, 0.05])]
        per = pers[it % 8]
        np.testing.assert_array_equal(oracle.interior_state(I, per, lib=lib), interior_state(I, per))
    st = np.array([1, 0, -1, 1, 0, 1, 0, 0], dtype=np.int8).reshape(1, 1, 8)
    ix = np.array([-1.0, -1.0, -1.0, 0.25, -0.25, 0.0, np.nan, -0.5], dtype=np.float32).reshape(1, 1, 8)
    assert oracle.interior_update(st, ix, lib=lib).reshape(-1).tolist() == [1, 0, -1, 0, 1, 0, 0, 1]
    # the parallel scheme against the brute force, over slabs of one to several planes
    for it in range(30):
        shape = tuple(int(v) for v in rng.integers(1, 7, size=3))
        occ = rng.random(shape) < rng.uniform(0.3, 0.7)
        per = pers[it % 8]
        same(oracle.label_mt(np.where(occ, 1.0, -1.0).astype(np.float32), per, threads=3, lib=lib),
             bfs_label(occ, per))
    # droplet-size histogram by R_c: hand-worked example
    h, rc_sum = oracle.rc_histogram([1, 8, 27, 1000], [0.5, 1.0, 2.0, 5.0, 10.0], lib=lib)
    assert h.tolist() == [0, 1, 2, 0, 1, 0]
    assert abs(rc_sum - 16 * (3 / (4 * np.pi)) ** (1 / 3)) < 1e-9


def _build(tmp_path, name, mutation):
    text = open(SRC).read()
    if mutation is not None:
        old, new = mutation
        assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
        text = text.replace(old, new)
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    out = tmp_path / f"lib{name}.so"
    oracle.build(str(src), str(out), extra=("-w",))
    return str(out)


def _battery_in_child(path):
    """Exit status of the battery run on the library at `path` in a child process
    (0: passed, 1: an assertion failed; a mutant that corrupts memory may also crash
    the child, which counts as caught without taking the test run down)."""
    code = ("import sys; sys.path[:0] = [{tests!r}, {root!r}]\n"
            "import oracle, test_oracle_mutations as m\n"
            "try:\n    m.battery(oracle.load({path!r}))\nexcept AssertionError:\n    sys.exit(1)\n")
    here = os.path.dirname(os.path.abspath(__file__))
    code = code.format(tests=here, root=os.path.dirname(here), path=path)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=600).returncode


def test_unmutated_passes(tmp_path):
    path = _build(tmp_path, "clean", None)
    battery(oracle.load(path))
    assert _battery_in_child(path) == 0      # the child harness itself works


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(tmp_path, name):
    assert _battery_in_child(_build(tmp_path, name, MUTATIONS[name])) != 0
