"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol the public headers declare; host-side argument checks and sizing need
no GPU."""
import ctypes
import os
import re

import pytest

from paper_1405_1931_gb300 import hk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("hk.h", "hk_gen.h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(hk_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for required in ("hk_create", "hk_destroy", "hk_label", "hk_label_batched", "hk_workspace_bytes",
                     "hk_strerror", "hk_label_host"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = hk.load()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(hk.EXPORTED)


def test_strerror_and_status_codes():
    assert hk.hk_strerror(hk.HK_OK) == "ok"
    assert "sizes_cap" in hk.hk_strerror(hk.HK_ERR_CAPACITY)
    assert hk.hk_strerror(12345) == "unknown status"


def test_workspace_bytes():
    assert hk.hk_workspace_bytes(0, 4, 4) == 0
    assert hk.hk_workspace_bytes(2048, 1024, 1024) == 0          # 2^31 sites: too large
    small = hk.hk_workspace_bytes(32, 32, 32)
    big = hk.hk_workspace_bytes(1024, 1024, 1024)
    assert 0 < small < big
    # linear in the number of tiles: 1024^3 has 32768x the tiles of 32^3
    assert big < 40000 * small
    # generous upper bound on bytes per site (mask, counts, faces, piece table)
    assert big / 1024 ** 3 < 4.0


def test_host_argument_errors_need_no_gpu():
    lib = hk.load()
    assert lib.hk_create(None, 0) == hk.HK_ERR_ARG
    per = (ctypes.c_int * 3)(1, 1, 1)
    # a NULL context is rejected before any CUDA call
    assert lib.hk_label(None, None, 4, 4, 4, per, None, None, 0, None, None, None) == hk.HK_ERR_ARG
    assert lib.hk_label_batched(None, None, 1, None) == hk.HK_ERR_ARG
    assert lib.hk_set_tile(None, 16, 16) == hk.HK_ERR_ARG
    assert lib.hk_gen_iid(None, 4, 4, 4, 0, 0.5, None) == 1
    # the later entry points check their arguments before any CUDA call too
    assert lib.hk_label_host_async(None, None, 4, 4, 4, per, None, None, 0, None, None, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_state(None, None, 4, 4, 4, per, None, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_update(None, None, -1, None, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_update(None, None, 5, None, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_update(None, None, 0, None, None) == hk.HK_OK          # nothing to do
    assert lib.hk_interior_update_sites(None, 10, None, None, -1, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_update_sites(None, 10, None, None, 3, None) == hk.HK_ERR_ARG
    assert lib.hk_interior_update_sites(None, 10, None, None, 0, None) == hk.HK_OK
    assert lib.hk_set_loop_cap(None, 4) == hk.HK_ERR_ARG
    assert lib.hk_set_small_path(None, 1) == hk.HK_ERR_ARG


def test_build_entry_compiles_everything():
    import __graft_entry__ as g
    g.build()
    assert os.path.exists(hk.lib_path())


def test_headers_are_plain_c_and_link(tmp_path):
    """The boundary is a C ABI: a C99 program that includes both headers and takes the
    address of every declared entry point compiles with gcc and links against libhk.so."""
    lib = hk.load()
    names = declared_symbols()
    src = tmp_path / "use_abi.c"
    src.write_text('#include "hk.h"\n#include "hk_gen.h"\n#include <stdio.h>\n'
                   "int main(void) {\n    const void *entries[] = {\n"
                   + "".join(f"        (const void *)&{n},\n" for n in names)
                   + "    };\n    printf(\"%d\\n\", (int)(sizeof entries / sizeof entries[0]));\n"
                   "    return 0;\n}\n")
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(lib._name)
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lhk", f"-Wl,-rpath,{libdir}"], check=True)
