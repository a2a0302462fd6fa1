"""CPU oracle for Hoshen-Kopelman labelling -- TEST INFRASTRUCTURE ONLY.

The serial algorithm of Frijters, Krueger and Harting (CPC 2014), Sec. 2
(raster scan, rules 1-3, label-of-labels list, final relabelling and
compactification) plus the periodic edges of Sec. 3, written in plain C in
``hk_oracle.c``.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It does not import the CUDA package and the CUDA package never
imports it.

``label(phi, periodic)`` takes a C-contiguous float32 array of shape
(nz, ny, nx) (x fastest) and returns ``(labels, sizes, hist, n_clusters)``:
labels int32 (nz, ny, nx), each site's smallest row-major site index in its
cluster or -1 on the medium; sizes int64[n_clusters] ordered by that index;
hist int64[32] over floor(log2(size)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hk_oracle.c")
_LIB = os.path.join(_HERE, "libhk_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_TOO_LARGE, ERR_CAPACITY, ERR_NOMEM = 0, 1, 2, 3, 6


def build(src: str = _SRC, out: str = _LIB, extra: tuple = ()) -> str:
    """Compile the oracle with gcc (portable flags only: it runs on x86 and Arm)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra", *extra, "-o", out, src,
           "-lm"]
    subprocess.run(cmd, check=True)
    return out


def load(path: str | None = None):
    """Load (building first if missing or older than the source) the oracle library."""
    global _lib
    with _lock:
        if path is not None:
            return _bind(ctypes.CDLL(path))
        if _lib is None:
            if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
                build()
            _lib = _bind(ctypes.CDLL(_LIB))
        return _lib


def _bind(lib):
    f = lib.hk_oracle_label
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    h = lib.hk_oracle_rc_histogram
    h.restype = ctypes.c_int
    h.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    g = lib.hk_oracle_interior
    g.restype = ctypes.c_int
    g.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    st = lib.hk_oracle_interior_state
    st.restype = ctypes.c_int
    st.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    mt = lib.hk_oracle_mt_label
    mt.restype = ctypes.c_int
    mt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    up = lib.hk_oracle_interior_update
    up.restype = ctypes.c_int
    up.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return lib


def label(phi: np.ndarray, periodic=(1, 1, 1), sizes_cap: int | None = None, lib=None):
    """Label ``phi`` (float32, shape (nz, ny, nx)) with the serial oracle."""
    lib = lib or load()
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    if phi.ndim != 3:
        raise ValueError("phi must have shape (nz, ny, nx)")
    nz, ny, nx = phi.shape
    n = phi.size
    if sizes_cap is None:
        sizes_cap = (n + 1) // 2
    labels = np.empty(phi.shape, dtype=np.int32)
    sizes = np.zeros(max(int(sizes_cap), 1), dtype=np.int64)
    hist = np.zeros(32, dtype=np.int64)
    ncl = np.zeros(1, dtype=np.int64)
    per = np.array([int(bool(p)) for p in periodic], dtype=np.int32)
    rc = lib.hk_oracle_label(phi.ctypes.data, nx, ny, nz, per.ctypes.data, labels.ctypes.data,
                             sizes.ctypes.data, int(sizes_cap), hist.ctypes.data, ncl.ctypes.data)
    if rc not in (OK, ERR_CAPACITY):
        raise RuntimeError(f"hk_oracle_label failed with status {rc}")
    k = int(ncl[0])
    return labels, sizes[:min(k, int(sizes_cap))].copy(), hist, k


def interior(index: np.ndarray, periodic=(1, 1, 1), sizes_cap: int | None = None, lib=None):
    """Interior/exterior identification of Sec. 6, steps 3-5, on an index field.

    ``index`` is float32 (nz, ny, nx): I < -0.5 far from every membrane, I in
    [-0.5, 0.5] near one (negative inside).  Returns ``(labels, sizes, hist,
    n_clusters, inside)``: the labelling of the far sites (as ``label``) and
    int8 ``inside[k]`` = 1 interior, 0 exterior, -1 undetermined, for each
    cluster in label order.
    """
    lib = lib or load()
    index = np.ascontiguousarray(index, dtype=np.float32)
    if index.ndim != 3:
        raise ValueError("index must have shape (nz, ny, nx)")
    nz, ny, nx = index.shape
    n = index.size
    if sizes_cap is None:
        sizes_cap = (n + 1) // 2
    labels = np.empty(index.shape, dtype=np.int32)
    sizes = np.zeros(max(int(sizes_cap), 1), dtype=np.int64)
    inside = np.zeros(max(int(sizes_cap), 1), dtype=np.int8)
    hist = np.zeros(32, dtype=np.int64)
    ncl = np.zeros(1, dtype=np.int64)
    per = np.array([int(bool(p)) for p in periodic], dtype=np.int32)
    rc = lib.hk_oracle_interior(index.ctypes.data, nx, ny, nz, per.ctypes.data, labels.ctypes.data,
                                sizes.ctypes.data, int(sizes_cap), hist.ctypes.data, ncl.ctypes.data,
                                inside.ctypes.data)
    if rc not in (OK, ERR_CAPACITY):
        raise RuntimeError(f"hk_oracle_interior failed with status {rc}")
    k = min(int(ncl[0]), int(sizes_cap))
    return labels, sizes[:k].copy(), hist, int(ncl[0]), inside[:k].copy()


def label_mt(phi: np.ndarray, periodic=(1, 1, 1), threads: int = 0, sizes_cap: int | None = None, lib=None):
    """The paper's parallel scheme (Sec. 3) on host threads, one slab of planes along z
    per thread (``threads`` = 0: all host cores).  Same results as ``label``."""
    lib = lib or load()
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    if phi.ndim != 3:
        raise ValueError("phi must have shape (nz, ny, nx)")
    nz, ny, nx = phi.shape
    n = phi.size
    if sizes_cap is None:
        sizes_cap = (n + 1) // 2
    threads = threads or (os.cpu_count() or 1)
    labels = np.empty(phi.shape, dtype=np.int32)
    sizes = np.zeros(max(int(sizes_cap), 1), dtype=np.int64)
    hist = np.zeros(32, dtype=np.int64)
    ncl = np.zeros(1, dtype=np.int64)
    per = np.array([int(bool(p)) for p in periodic], dtype=np.int32)
    rc = lib.hk_oracle_mt_label(phi.ctypes.data, nx, ny, nz, per.ctypes.data, int(threads), labels.ctypes.data,
                                sizes.ctypes.data, int(sizes_cap), hist.ctypes.data, ncl.ctypes.data)
    if rc not in (OK, ERR_CAPACITY):
        raise RuntimeError(f"hk_oracle_mt_label failed with status {rc}")
    k = int(ncl[0])
    return labels, sizes[:min(k, int(sizes_cap))].copy(), hist, k


def interior_state(index: np.ndarray, periodic=(1, 1, 1), lib=None) -> np.ndarray:
    """Interior state of every site (Sec. 6): int8, 1 inside, 0 outside, -1 undetermined.

    Far sites (I < -0.5) take their cluster's tag (``interior``); near sites the
    side their value names (I < 0: 1, else 0).
    """
    lib = lib or load()
    index = np.ascontiguousarray(index, dtype=np.float32)
    if index.ndim != 3:
        raise ValueError("index must have shape (nz, ny, nx)")
    nz, ny, nx = index.shape
    state = np.empty(index.shape, dtype=np.int8)
    per = np.array([int(bool(p)) for p in periodic], dtype=np.int32)
    rc = lib.hk_oracle_interior_state(index.ctypes.data, nx, ny, nz, per.ctypes.data, state.ctypes.data)
    if rc != OK:
        raise RuntimeError(f"hk_oracle_interior_state failed with status {rc}")
    return state


def interior_update(state_prev: np.ndarray, index: np.ndarray, lib=None) -> np.ndarray:
    """Incremental interior state for slowly moving membranes (Sec. 6, last paragraph):
    sites near a membrane now (I >= -0.5) take the side their value names (I < 0: 1,
    else 0); every other site keeps its previous state."""
    lib = lib or load()
    state_prev = np.ascontiguousarray(state_prev, dtype=np.int8)
    index = np.ascontiguousarray(index, dtype=np.float32)
    if state_prev.shape != index.shape:
        raise ValueError("state_prev and index must have one shape")
    out = np.empty(index.shape, dtype=np.int8)
    rc = lib.hk_oracle_interior_update(state_prev.ctypes.data, index.ctypes.data, int(index.size), out.ctypes.data)
    if rc != OK:
        raise RuntimeError(f"hk_oracle_interior_update failed with status {rc}")
    return out


def rc_histogram(sizes, edges, lib=None):
    """Droplet-size histogram by R_c (Fig. 5) with ascending ``edges``; returns (hist, rc_sum).

    hist has len(edges) + 1 bins: below the first edge, between consecutive
    edges, and at or above the last one; rc_sum is the sum of R_c.
    """
    lib = lib or load()
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    hist = np.zeros(len(edges) + 1, dtype=np.int64)
    rc = np.zeros(1, dtype=np.float64)
    rc_ = lib.hk_oracle_rc_histogram(sizes.ctypes.data, int(sizes.size), edges.ctypes.data, int(edges.size),
                                     hist.ctypes.data, rc.ctypes.data)
    if rc_ != OK:
        raise RuntimeError(f"hk_oracle_rc_histogram failed with status {rc_}")
    return hist, float(rc[0])


def status(phi: np.ndarray, periodic=(1, 1, 1), sizes_cap: int = 0, lib=None) -> int:
    """Return the oracle's status code for a call (used by argument tests)."""
    lib = lib or load()
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    nz, ny, nx = phi.shape
    labels = np.empty(phi.shape, dtype=np.int32)
    sizes = np.zeros(max(sizes_cap, 1), dtype=np.int64)
    hist = np.zeros(32, dtype=np.int64)
    ncl = np.zeros(1, dtype=np.int64)
    per = np.array([int(bool(p)) for p in periodic], dtype=np.int32)
    return lib.hk_oracle_label(phi.ctypes.data, nx, ny, nz, per.ctypes.data, labels.ctypes.data,
                               sizes.ctypes.data, int(sizes_cap), hist.ctypes.data, ncl.ctypes.data)
