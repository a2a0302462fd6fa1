"""Thin Python binding of libhk (include/hk.h, include/hk_gen.h).

Argument marshalling only: every step of the labelling runs in the CUDA
library.  The functions named ``hk_*`` mirror the C entry points one to one
and take raw pointers (ints) and a stream handle; ``Labeller`` wraps a context
and accepts torch CUDA tensors.  There is no CPU fallback: if the library
cannot be loaded or built, importing the symbols raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HK_OK, HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_CAPACITY = 0, 1, 2, 3
HK_ERR_CUDA, HK_ERR_TIMEOUT, HK_ERR_NOMEM = 4, 5, 6

EXPORTED = ("hk_create", "hk_destroy", "hk_workspace_bytes", "hk_reserve", "hk_label", "hk_label_batched",
            "hk_label_host", "hk_label_host_async", "hk_set_tile", "hk_set_timing", "hk_get_timing", "hk_sync_status", "hk_set_graphs", "hk_last_cuda_error", "hk_strerror", "hk_label_noalloc",
            "hk_noalloc_sync_status", "hk_set_loop_cap", "hk_set_small_path", "hk_set_merge",
            "hk_label_slab", "hk_slab_faces", "hk_slab_merge",
            "hk_label_interior", "hk_rc_histogram", "hk_interior_state", "hk_interior_update",
            "hk_interior_update_sites",
            "hk_gen_iid", "hk_gen_spheres", "hk_gen_spheres_dev", "hk_gen_capsule")

_lock = threading.Lock()
_lib = None


class HKError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {hk_strerror(status)} (status {status})" if where else hk_strerror(status))


class hk_lattice(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("labels", ctypes.c_void_p), ("sizes", ctypes.c_void_p),
                ("sizes_cap", ctypes.c_int64), ("hist", ctypes.c_void_p), ("n_clusters", ctypes.c_void_p)]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libhk.so, building it first if it is missing or older than its sources."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _build.needs_build():
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        P, I, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "hk_create": (I, [ctypes.POINTER(P), I]),
            "hk_destroy": (None, [P]),
            "hk_workspace_bytes": (SZ, [I, I, I]),
            "hk_reserve": (I, [P, SZ]),
            "hk_label": (I, [P, P, I, I, I, P, P, P, I64, P, P, P]),
            "hk_label_batched": (I, [P, ctypes.POINTER(hk_lattice), I, P]),
            "hk_label_host": (I, [P, P, I, I, I, P, P, P, I64, P, P, P]),
            "hk_label_host_async": (I, [P, P, I, I, I, P, P, P, I64, P, P, P]),
            "hk_label_noalloc": (I, [P, I, I, I, P, P, P, I64, P, P, P]),
            "hk_noalloc_sync_status": (I, [P]),
            "hk_set_loop_cap": (I, [P, I64]),
            "hk_set_small_path": (I, [P, I]),
            "hk_set_merge": (I, [P, I, I]),
            "hk_label_slab": (I, [P, P, I, I, I, I64, I, I, P, P, I64, P, P, P]),
            "hk_slab_faces": (I, [P, P, I, I, I, P, P, P, I64, P, P, P, P, P]),
            "hk_slab_merge": (I, [P, I, I, I, I, I, P, P, P, P, I64, P, I, I64, P, P, I64, P, I64, P, P, P]),
            "hk_label_interior": (I, [P, P, I, I, I, P, P, P, I64, P, P, P, P]),
            "hk_rc_histogram": (I, [P, P, I64, P, I, P, P, I, P]),
            "hk_interior_state": (I, [P, P, I, I, I, P, P, P]),
            "hk_interior_update": (I, [P, P, I64, P, P]),
            "hk_interior_update_sites": (I, [P, I64, P, P, I64, P]),
            "hk_set_tile": (I, [P, I, I]),
            "hk_set_timing": (I, [P, I]),
            "hk_set_graphs": (I, [P, I]),
            "hk_get_timing": (I, [P, ctypes.POINTER(ctypes.c_float), I, ctypes.POINTER(ctypes.c_int)]),
            "hk_sync_status": (I, [P, P]),
            "hk_last_cuda_error": (I, [P]),
            "hk_strerror": (ctypes.c_char_p, [I]),
            "hk_gen_iid": (I, [P, I, I, I, ctypes.c_uint64, ctypes.c_double, P]),
            "hk_gen_spheres": (I, [P, I, I, I, P, P, I, ctypes.c_double, P]),
            "hk_gen_capsule": (I, [P, I, ctypes.c_double, ctypes.c_double, ctypes.c_double, P]),
            "hk_gen_spheres_dev": (I, [P, I, I, I, P, I, ctypes.c_double, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


# ---- one-to-one wrappers -------------------------------------------------------------------

def hk_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    rc = load().hk_create(ctypes.byref(h), int(device))
    if rc != HK_OK:
        raise HKError(rc, "hk_create")
    return h.value


def hk_destroy(ctx: int) -> None:
    load().hk_destroy(ctx)


def hk_workspace_bytes(nx: int, ny: int, nz: int) -> int:
    return int(load().hk_workspace_bytes(nx, ny, nz))


def hk_reserve(ctx: int, nbytes: int) -> int:
    return load().hk_reserve(ctx, int(nbytes))


def _per(periodic):
    return (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])


def hk_label(ctx, phi, nx, ny, nz, periodic, labels_out, sizes_out, sizes_cap, hist_out, n_clusters_out,
             stream=0) -> int:
    return load().hk_label(ctx, phi, nx, ny, nz, _per(periodic), labels_out, sizes_out, int(sizes_cap),
                           hist_out, n_clusters_out, stream)


def hk_label_interior(ctx, index, nx, ny, nz, periodic, labels_out, sizes_out, sizes_cap, hist_out, n_clusters_out,
                      inside_out, stream=0) -> int:
    return load().hk_label_interior(ctx, index, nx, ny, nz, _per(periodic), labels_out, sizes_out, int(sizes_cap),
                                    hist_out, n_clusters_out, inside_out, stream)


def hk_rc_histogram(sizes, n_clusters, sizes_cap, edges, hist_out, rc_sum_out, accumulate=False, stream=0) -> int:
    e = (ctypes.c_double * len(edges))(*[float(v) for v in edges])
    return load().hk_rc_histogram(sizes, n_clusters, int(sizes_cap), e, len(edges), hist_out, rc_sum_out,
                                  int(bool(accumulate)), stream)


def rc_histogram(sizes, ncl, edges, cap=None, out=None, accumulate=False, stream=None):
    """Droplet-size histogram by R_c on device tensors (hk_rc_histogram); returns (hist, rc_sum)."""
    import torch
    if out is None:
        out = (torch.zeros(len(edges) + 1, dtype=torch.int64, device=sizes.device),
               torch.zeros(1, dtype=torch.float64, device=sizes.device))
    hist, rc_sum = out
    cap = sizes.numel() if cap is None else int(cap)
    rc = hk_rc_histogram(sizes.data_ptr(), ncl.data_ptr(), cap, edges, hist.data_ptr(), rc_sum.data_ptr(),
                         accumulate, _stream_handle(stream))
    if rc != HK_OK:
        raise HKError(rc, "hk_rc_histogram")
    return hist, rc_sum


def hk_label_batched(ctx, lats, stream=0) -> int:
    arr = (hk_lattice * len(lats))(*lats)
    return load().hk_label_batched(ctx, arr, len(lats), stream)


def hk_label_host(ctx, phi_host, nx, ny, nz, periodic, labels_host, sizes_host, sizes_cap, hist_host,
                  n_clusters_host, stream=0) -> int:
    return load().hk_label_host(ctx, phi_host, nx, ny, nz, _per(periodic), labels_host, sizes_host,
                                int(sizes_cap), hist_host, n_clusters_host, stream)


def hk_interior_state(ctx, index, nx, ny, nz, periodic, state_out, stream=0) -> int:
    return load().hk_interior_state(ctx, index, nx, ny, nz, _per(periodic), state_out, stream)


def hk_interior_update(state_prev, index, n_sites, state_out, stream=0) -> int:
    return load().hk_interior_update(state_prev, index, int(n_sites), state_out, stream)


def hk_interior_update_sites(state, n_sites, sites, values, m, stream=0) -> int:
    return load().hk_interior_update_sites(state, int(n_sites), sites, values, int(m), stream)


def hk_label_host_async(ctx, phi_host, nx, ny, nz, periodic, labels_host, sizes_host, sizes_cap, hist_host,
                        n_clusters_host, stream=0) -> int:
    return load().hk_label_host_async(ctx, phi_host, nx, ny, nz, _per(periodic), labels_host, sizes_host,
                                      int(sizes_cap), hist_host, n_clusters_host, stream)


def hk_label_noalloc(phi, nx, ny, nz, periodic, labels_out, sizes_out, sizes_cap, hist_out, n_clusters_out,
                     stream=0) -> int:
    return load().hk_label_noalloc(phi, nx, ny, nz, _per(periodic), labels_out, sizes_out, int(sizes_cap),
                                   hist_out, n_clusters_out, stream)


def hk_noalloc_sync_status(stream=0) -> int:
    return load().hk_noalloc_sync_status(stream)


NOALLOC_SCRATCH_BYTES = 64 << 20


def hk_set_loop_cap(ctx, cap: int) -> int:
    return load().hk_set_loop_cap(ctx, int(cap))


def hk_label_slab(ctx, phi, nx, ny, nz, z0, periodic_x, periodic_y, labels_out, sizes_out, sizes_cap, roots_out,
                  n_clusters_out, stream=0) -> int:
    return load().hk_label_slab(ctx, phi, nx, ny, nz, int(z0), int(bool(periodic_x)), int(bool(periodic_y)),
                                labels_out, sizes_out, int(sizes_cap), roots_out, n_clusters_out, stream)


def hk_slab_faces(ctx, labels, nx, ny, nz, roots, sizes, n_clusters, sizes_cap, face_out, list_lab_out, list_size_out,
                  n_face_out, stream=0) -> int:
    return load().hk_slab_faces(ctx, labels, nx, ny, nz, roots, sizes, n_clusters, int(sizes_cap), face_out,
                                list_lab_out, list_size_out, n_face_out, stream)


def hk_slab_merge(ctx, nranks, rank, periodic_z, nx, ny, face_all, n_face_all, list_lab_all, list_size_all, max_face,
                  labels, nz, z0, sizes, n_clusters, sizes_cap, own_sizes_out, own_cap, own_n_out, hist_out,
                  stream=0) -> int:
    nf = (ctypes.c_int64 * len(n_face_all))(*[int(v) for v in n_face_all])
    return load().hk_slab_merge(ctx, int(nranks), int(rank), int(bool(periodic_z)), nx, ny, face_all, nf,
                                list_lab_all, list_size_all, int(max_face), labels, nz, int(z0), sizes, n_clusters,
                                int(sizes_cap), own_sizes_out, int(own_cap), own_n_out, hist_out, stream)


def hk_set_merge(ctx, unions_per_lane: int, combine_hot: int) -> int:
    return load().hk_set_merge(ctx, int(unions_per_lane), int(combine_hot))


def hk_set_small_path(ctx, enable: bool) -> int:
    return load().hk_set_small_path(ctx, int(enable))


def hk_set_tile(ctx, ty, tz) -> int:
    return load().hk_set_tile(ctx, ty, tz)


PASS_NAMES = ("occupancy", "tile_label", "face_merge", "piece_finalize", "scan", "lattice_finish", "flatten")


def hk_set_timing(ctx, enable: bool) -> int:
    return load().hk_set_timing(ctx, int(bool(enable)))


def hk_get_timing(ctx):
    """Per-pass milliseconds of the context's last timed call (synchronises on it)."""
    buf = (ctypes.c_float * 16)()
    n = ctypes.c_int(0)
    rc = load().hk_get_timing(ctx, buf, 16, ctypes.byref(n))
    if rc != HK_OK:
        raise HKError(rc, "hk_get_timing")
    return [float(buf[i]) for i in range(n.value)]


def hk_set_graphs(ctx, enable: bool) -> int:
    return load().hk_set_graphs(ctx, int(bool(enable)))


def hk_sync_status(ctx, stream=0) -> int:
    return load().hk_sync_status(ctx, stream)


def hk_last_cuda_error(ctx) -> int:
    return load().hk_last_cuda_error(ctx)


def hk_strerror(status: int) -> str:
    return load().hk_strerror(int(status)).decode()


def hk_gen_iid(phi, nx, ny, nz, seed, occupancy, stream=0) -> int:
    return load().hk_gen_iid(phi, nx, ny, nz, int(seed), float(occupancy), stream)


def hk_gen_spheres(phi, nx, ny, nz, centres, radii, reach=8.0, stream=0) -> int:
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    return load().hk_gen_spheres(phi, nx, ny, nz, c.ctypes.data, r.ctypes.data, int(r.size), float(reach), stream)


def hk_gen_spheres_dev(phi, nx, ny, nz, spheres_dev, n_spheres, reach=8.0, stream=0) -> int:
    return load().hk_gen_spheres_dev(phi, nx, ny, nz, spheres_dev, int(n_spheres), float(reach), stream)


def hk_gen_capsule(phi, L, ax, ay, az, stream=0) -> int:
    return load().hk_gen_capsule(phi, int(L), float(ax), float(ay), float(az), stream)


# ---- torch convenience ---------------------------------------------------------------------

def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Labeller:
    """A libhk context bound to one CUDA device, taking torch tensors.

    ``label(phi)`` with ``phi`` a float32 CUDA tensor of shape (nz, ny, nx)
    returns ``(labels, sizes, hist, n_clusters)`` as CUDA tensors (sizes has
    ``sizes_cap`` entries, default ceil(N/2); the first n_clusters are valid).
    """

    def __init__(self, device: int = 0, tile: tuple | None = None):
        self.device = int(device)
        self.ctx = hk_create(self.device)
        self.tile = (16, 16)
        self.merge = (1, 1)
        if tile is not None:
            self.set_tile(*tile)

    def close(self):
        if getattr(self, "ctx", None):
            hk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, ty: int, tz: int):
        rc = hk_set_tile(self.ctx, ty, tz)
        if rc != HK_OK:
            raise HKError(rc, "hk_set_tile")
        self.tile = (ty, tz)

    def set_graphs(self, enable: bool = True):
        rc = hk_set_graphs(self.ctx, enable)
        if rc != HK_OK:
            raise HKError(rc, "hk_set_graphs")

    def set_merge(self, unions_per_lane: int = 1, combine_hot: int = 1):
        """Merge schedule of the tiled passes (face-merge unions per lane, hot-root combining)."""
        rc = hk_set_merge(self.ctx, unions_per_lane, combine_hot)
        if rc != HK_OK:
            raise HKError(rc, "hk_set_merge")
        self.merge = (unions_per_lane or 1, combine_hot)

    def set_small_path(self, enable=True):
        """One-launch kernels for small lattices: True/1 the library picks (default), False/0
        the tiled passes always, 2 the one-CTA kernel only, 3 the cluster kernel only."""
        rc = hk_set_small_path(self.ctx, int(enable))
        if rc != HK_OK:
            raise HKError(rc, "hk_set_small_path")

    def set_loop_cap(self, cap: int):
        """Lower the bound of the capped union-find loops (test control; 0 restores them)."""
        rc = hk_set_loop_cap(self.ctx, cap)
        if rc != HK_OK:
            raise HKError(rc, "hk_set_loop_cap")

    def sync_status(self, stream=None):
        """Synchronise and raise if a bounded device-side loop gave up since the last check."""
        rc = hk_sync_status(self.ctx, _stream_handle(stream))
        if rc != HK_OK:
            raise HKError(rc, "hk_sync_status")

    def reserve(self, nbytes: int):
        rc = hk_reserve(self.ctx, nbytes)
        if rc != HK_OK:
            raise HKError(rc, "hk_reserve")

    @staticmethod
    def alloc_outputs(shape, device, sizes_cap=None):
        import torch
        n = int(np.prod(shape))
        cap = (n + 1) // 2 if sizes_cap is None else int(sizes_cap)
        labels = torch.empty(shape, dtype=torch.int32, device=device)
        sizes = torch.empty(max(cap, 1), dtype=torch.int64, device=device)
        hist = torch.empty(32, dtype=torch.int64, device=device)
        ncl = torch.empty(1, dtype=torch.int64, device=device)
        return labels, sizes, hist, ncl, cap

    def label(self, phi, periodic=(1, 1, 1), out=None, sizes_cap=None, stream=None, check=True):
        import torch
        if not (phi.is_cuda and phi.dtype == torch.float32 and phi.dim() == 3 and phi.is_contiguous()):
            raise ValueError("phi must be a contiguous float32 CUDA tensor of shape (nz, ny, nx)")
        nz, ny, nx = phi.shape
        if out is None:
            out = self.alloc_outputs(phi.shape, phi.device, sizes_cap)
        labels, sizes, hist, ncl, cap = out
        rc = hk_label(self.ctx, phi.data_ptr(), nx, ny, nz, periodic, labels.data_ptr(), sizes.data_ptr(), cap,
                      hist.data_ptr(), ncl.data_ptr(), _stream_handle(stream))
        if check and rc != HK_OK:
            raise HKError(rc, "hk_label")
        return labels, sizes, hist, ncl

    def label_interior(self, index, periodic=(1, 1, 1), out=None, sizes_cap=None, stream=None, check=True):
        """Sec. 6, steps 3-5 on an index field; returns (labels, sizes, hist, ncl, inside)."""
        import torch
        if not (index.is_cuda and index.dtype == torch.float32 and index.dim() == 3 and index.is_contiguous()):
            raise ValueError("index must be a contiguous float32 CUDA tensor of shape (nz, ny, nx)")
        nz, ny, nx = index.shape
        if out is None:
            out = self.alloc_outputs(index.shape, index.device, sizes_cap)
        labels, sizes, hist, ncl, cap = out
        inside = torch.empty(max(cap, 1), dtype=torch.int8, device=index.device)
        rc = hk_label_interior(self.ctx, index.data_ptr(), nx, ny, nz, periodic, labels.data_ptr(), sizes.data_ptr(),
                               cap, hist.data_ptr(), ncl.data_ptr(), inside.data_ptr(), _stream_handle(stream))
        if check and rc != HK_OK:
            raise HKError(rc, "hk_label_interior")
        return labels, sizes, hist, ncl, inside

    def interior_state(self, index, periodic=(1, 1, 1), out=None, stream=None):
        """Sec. 6: the interior state of every site (int8: 1 inside, 0 outside, -1 undetermined)."""
        import torch
        if not (index.is_cuda and index.dtype == torch.float32 and index.dim() == 3 and index.is_contiguous()):
            raise ValueError("index must be a contiguous float32 CUDA tensor of shape (nz, ny, nx)")
        nz, ny, nx = index.shape
        state = torch.empty(index.shape, dtype=torch.int8, device=index.device) if out is None else out
        rc = hk_interior_state(self.ctx, index.data_ptr(), nx, ny, nz, periodic, state.data_ptr(), _stream_handle(stream))
        if rc != HK_OK:
            raise HKError(rc, "hk_interior_state")
        return state

    def label_batched(self, items, stream=None, check=True):
        """items: list of (phi, periodic, (labels, sizes, hist, ncl, cap)) with CUDA tensors."""
        lats = []
        for phi, periodic, (labels, sizes, hist, ncl, cap) in items:
            nz, ny, nx = phi.shape
            lats.append(hk_lattice(phi.data_ptr(), nx, ny, nz, (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic]),
                                   labels.data_ptr(), sizes.data_ptr(), int(cap), hist.data_ptr(), ncl.data_ptr()))
        rc = hk_label_batched(self.ctx, lats, _stream_handle(stream))
        if check and rc != HK_OK:
            raise HKError(rc, "hk_label_batched")
        return rc

    def label_host(self, phi: np.ndarray, periodic=(1, 1, 1), sizes_cap=None, out=None, stream=None):
        """Host buffers in and out (numpy); copies run inside the call."""
        phi = np.ascontiguousarray(phi, dtype=np.float32)
        nz, ny, nx = phi.shape
        n = phi.size
        cap = (n + 1) // 2 if sizes_cap is None else int(sizes_cap)
        if out is None:
            out = (np.empty(phi.shape, np.int32), np.empty(max(cap, 1), np.int64), np.empty(32, np.int64),
                   np.empty(1, np.int64))
        labels, sizes, hist, ncl = out
        rc = hk_label_host(self.ctx, phi.ctypes.data, nx, ny, nz, periodic, labels.ctypes.data,
                           sizes.ctypes.data, cap, hist.ctypes.data, ncl.ctypes.data, _stream_handle(stream))
        if rc not in (HK_OK, HK_ERR_CAPACITY):
            raise HKError(rc, "hk_label_host")
        k = int(ncl[0])
        return labels, sizes[:min(k, cap)], hist, k

    def label_host_async(self, phi, labels, sizes, hist, ncl, periodic=(1, 1, 1), stream=None):
        """Enqueue one field held in page-locked host tensors (torch, pin_memory=True)
        and return; the outputs are valid once `stream` has passed the call, when
        sizes holds the first min(ncl[0], len(sizes)) sizes."""
        nz, ny, nx = phi.shape
        rc = hk_label_host_async(self.ctx, phi.data_ptr(), nx, ny, nz, periodic, labels.data_ptr(),
                                 sizes.data_ptr(), sizes.numel(), hist.data_ptr(), ncl.data_ptr(),
                                 _stream_handle(stream))
        if rc != HK_OK:
            raise HKError(rc, "hk_label_host_async")


def interior_update(state_prev, index, out=None, stream=None):
    """Sec. 6, last paragraph: near sites take their side now, far sites keep their state
    (CUDA tensors; out may be state_prev)."""
    if state_prev.shape != index.shape or not (state_prev.is_contiguous() and index.is_contiguous()):
        raise ValueError("state_prev and index must be contiguous tensors of one shape")
    out = state_prev if out is None else out
    rc = hk_interior_update(state_prev.data_ptr(), index.data_ptr(), index.numel(), out.data_ptr(), _stream_handle(stream))
    if rc != HK_OK:
        raise HKError(rc, "hk_interior_update")
    return out


def interior_update_sites(state, sites, values, stream=None):
    """The same step from a list of near sites (int32) and their values (float32), in place."""
    if sites.numel() != values.numel():
        raise ValueError("sites and values must have one length")
    rc = hk_interior_update_sites(state.data_ptr(), state.numel(), sites.data_ptr(), values.data_ptr(), sites.numel(),
                                  _stream_handle(stream))
    if rc != HK_OK:
        raise HKError(rc, "hk_interior_update_sites")
    return state
