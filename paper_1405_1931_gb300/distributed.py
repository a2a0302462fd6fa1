"""A lattice split into slabs along z across ranks: the domain decomposition of Sec. 3.

Each rank of a torch.distributed process group holds planes [z0, z0 + nz) of the
lattice on its own GPU.  `label_slab` labels them through the library's slab entry
points (include/hk.h: hk_label_slab, hk_slab_faces, hk_slab_merge) and moves the
face data between ranks with torch.distributed collectives: all_gather of every
rank's two face planes of face-cluster numbers (the halo of Sec. 3), of its
face-cluster labels and sizes, and of the counts.  Every rank then resolves all
equivalences on its own device, so there is no gather at a root process and no
scatter.  This module only moves buffers: every step of the labelling runs in the
library's kernels.

With the NCCL backend the buffers stay on the device; with gloo they pass through
host memory (gloo moves CPU tensors).
"""
from __future__ import annotations

from dataclasses import dataclass

from . import hk


def slab_bounds(nz_total: int, nranks: int, rank: int) -> tuple:
    """(z0, nz) of rank `rank`: nz_total planes split into nranks slabs, the first
    nz_total % nranks slabs one plane thicker.  Every slab has at least one plane."""
    if not 1 <= nranks <= nz_total or not 0 <= rank < nranks:
        raise ValueError("need 1 <= nranks <= nz_total and 0 <= rank < nranks")
    base, extra = divmod(nz_total, nranks)
    z0 = rank * base + min(rank, extra)
    return z0, base + (1 if rank < extra else 0)


@dataclass
class SlabResult:
    labels: object        # this slab's labels (device int32), site indices of the whole lattice
    own_sizes: object     # sizes of the clusters whose smallest site is in this slab, label order
    offset: int           # clusters of the earlier ranks: own_sizes[i] is global cluster offset + i
    n_clusters: int       # clusters of the whole lattice
    hist: object          # floor(log2 size) histogram of the whole lattice (device int64[32])


def _all_gather(dist, group, t, on_device):
    """all_gather of one tensor per rank (all of one shape), returned stacked."""
    import torch
    src = t if on_device else t.cpu()
    parts = [torch.empty_like(src) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, src.contiguous(), group=group)
    out = torch.stack(parts)
    return out if on_device else out.to(t.device)


def label_slab(lab: "hk.Labeller", phi_slab, z0: int, nz_total: int, periodic=(1, 1, 1), group=None,
               stream=None) -> SlabResult:
    """Label this rank's slab (device float32 tensor of shape (nz, ny, nx), planes z0 ..
    z0 + nz - 1 of an nz_total-plane lattice) together with the other ranks' slabs.

    Every rank of `group` calls this with its own slab, in rank order along z (rank r's
    slab follows rank r - 1's).  Returns this rank's share of the result, equal to
    labelling the whole lattice at once."""
    import torch
    import torch.distributed as dist
    on_device = dist.get_backend(group) == "nccl"
    R, r = dist.get_world_size(group), dist.get_rank(group)
    nz, ny, nx = phi_slab.shape
    dev = phi_slab.device
    P = nx * ny
    N = phi_slab.numel()
    cap = (N + 1) // 2
    h = hk._stream_handle(stream)
    labels = torch.empty((nz, ny, nx), dtype=torch.int32, device=dev)
    sizes = torch.empty(cap, dtype=torch.int64, device=dev)
    roots = torch.empty(cap, dtype=torch.int32, device=dev)
    ncl = torch.empty(1, dtype=torch.int64, device=dev)
    rc = hk.hk_label_slab(lab.ctx, phi_slab.data_ptr(), nx, ny, nz, z0, periodic[0], periodic[1], labels.data_ptr(),
                          sizes.data_ptr(), cap, roots.data_ptr(), ncl.data_ptr(), h)
    if rc != hk.HK_OK:
        raise hk.HKError(rc, "hk_label_slab")
    face = torch.empty(2 * P, dtype=torch.int32, device=dev)
    list_lab = torch.empty(2 * P, dtype=torch.int32, device=dev)
    list_size = torch.empty(2 * P, dtype=torch.int64, device=dev)
    nf = torch.empty(1, dtype=torch.int64, device=dev)
    rc = hk.hk_slab_faces(lab.ctx, labels.data_ptr(), nx, ny, nz, roots.data_ptr(), sizes.data_ptr(), ncl.data_ptr(),
                          cap, face.data_ptr(), list_lab.data_ptr(), list_size.data_ptr(), nf.data_ptr(), h)
    if rc != hk.HK_OK:
        raise hk.HKError(rc, "hk_slab_faces")
    (stream or torch.cuda.current_stream()).synchronize()
    # the halo exchange: every rank's face planes, face-cluster lists and counts
    nf_all = _all_gather(dist, group, nf, on_device).reshape(-1).cpu().tolist()
    max_face = max(1, max(nf_all))   # at most 2 P: a face cluster holds a face site
    face_all = _all_gather(dist, group, face, on_device)
    lab_all = _all_gather(dist, group, list_lab[:max_face], on_device)
    size_all = _all_gather(dist, group, list_size[:max_face], on_device)
    own_sizes = torch.empty(cap, dtype=torch.int64, device=dev)
    own_n = torch.empty(1, dtype=torch.int64, device=dev)
    hist = torch.empty(32, dtype=torch.int64, device=dev)
    rc = hk.hk_slab_merge(lab.ctx, R, r, periodic[2], nx, ny, face_all.data_ptr(), nf_all, lab_all.data_ptr(),
                          size_all.data_ptr(), max_face, labels.data_ptr(), nz, z0, sizes.data_ptr(), ncl.data_ptr(),
                          cap, own_sizes.data_ptr(), cap, own_n.data_ptr(), hist.data_ptr(), h)
    if rc != hk.HK_OK:
        raise hk.HKError(rc, "hk_slab_merge")
    lab.sync_status(stream)
    # offsets in the global numbering and the whole lattice's histogram
    counts = _all_gather(dist, group, own_n, on_device).reshape(-1).cpu().tolist()
    if on_device:
        dist.all_reduce(hist, group=group)
    else:
        hc = hist.cpu()
        dist.all_reduce(hc, group=group)
        hist = hc.to(dev)
    n_own = counts[r]
    return SlabResult(labels=labels, own_sizes=own_sizes[:n_own], offset=int(sum(counts[:r])),
                      n_clusters=int(sum(counts)), hist=hist)
