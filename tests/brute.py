"""Brute-force connected-component references used to pin the oracle.

None of this shares code with the oracle or the CUDA path.  Each function
defines 6-connected clusters of {phi > 0} directly from the definition of a
connected component, with per-axis periodic edges:

* ``bfs_label``: breadth-first flood fill in pure Python over an explicit
  neighbour list (tiny lattices only);
* ``relax_label``: repeated minimum propagation over the six neighbour
  shifts until nothing changes (a relaxation in the spirit of the
  Flanigan-Tamayo scheme the paper discusses in Sec. 3), vectorised with numpy;
* ``canonical_from_partition``: turns any component numbering into the
  min-row-major-index labels, sizes and log2 histogram.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def neighbours(x, y, z, dims, periodic):
    nx, ny, nz = dims
    out = []
    for axis, (c, n) in enumerate(((x, nx), (y, ny), (z, nz))):
        for d in (-1, 1):
            v = c + d
            if v < 0 or v >= n:
                if not periodic[axis]:
                    continue
                v %= n
            p = [x, y, z]
            p[axis] = v
            out.append(tuple(p))
    return out


def bfs_label(occ: np.ndarray, periodic):
    """occ: bool (nz, ny, nx).  Returns (labels, sizes, hist, n) by BFS in raster order."""
    nz, ny, nx = occ.shape
    dims = (nx, ny, nz)
    labels = np.full(occ.shape, -1, dtype=np.int64)
    sizes = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not occ[z, y, x] or labels[z, y, x] >= 0:
                    continue
                root = x + nx * (y + ny * z)
                labels[z, y, x] = root
                q = deque([(x, y, z)])
                cnt = 0
                while q:
                    cx, cy, cz = q.popleft()
                    cnt += 1
                    for (ax, ay, az) in neighbours(cx, cy, cz, dims, periodic):
                        if occ[az, ay, ax] and labels[az, ay, ax] < 0:
                            labels[az, ay, ax] = root
                            q.append((ax, ay, az))
                sizes.append(cnt)
    return labels.astype(np.int32), np.array(sizes, dtype=np.int64), log2_hist(sizes), len(sizes)


def log2_hist(sizes):
    h = np.zeros(32, dtype=np.int64)
    for s in sizes:
        h[int(s).bit_length() - 1] += 1
    return h


def _shift(a, axis, d, periodic, fill):
    """a shifted by d along array axis ``axis``; periodic wraps, else ``fill`` enters."""
    if periodic:
        return np.roll(a, d, axis=axis)
    out = np.full_like(a, fill)
    sl_dst = [slice(None)] * 3
    sl_src = [slice(None)] * 3
    if d > 0:
        sl_dst[axis] = slice(d, None)
        sl_src[axis] = slice(None, -d)
    else:
        sl_dst[axis] = slice(None, d)
        sl_src[axis] = slice(-d, None)
    out[tuple(sl_dst)] = a[tuple(sl_src)]
    return out


def relax_label(occ: np.ndarray, periodic, max_iter: int = 1_000_000):
    """Min-propagation to a fixed point: each occupied site takes the min over its cluster."""
    nz, ny, nx = occ.shape
    big = np.iinfo(np.int64).max
    idx = np.arange(occ.size, dtype=np.int64).reshape(occ.shape)
    lab = np.where(occ, idx, big)
    # array axis 2 is x, 1 is y, 0 is z
    axes = ((2, periodic[0]), (1, periodic[1]), (0, periodic[2]))
    for _ in range(max_iter):
        new = lab.copy()
        for axis, per in axes:
            for d in (-1, 1):
                sh = _shift(lab, axis, d, bool(per), big)
                new = np.minimum(new, sh)
        new = np.where(occ, new, big)
        # pointer jumping: a site may also adopt the label of the site its label names
        flat = new.reshape(-1)
        occf = occ.reshape(-1)
        jump = flat.copy()
        m = occf & (flat < big)
        jump[m] = flat[flat[m]]
        new = np.minimum(new, jump.reshape(occ.shape))
        if np.array_equal(new, lab):
            break
        lab = new
    labels = np.where(occ, lab, -1).astype(np.int64)
    return canonical_from_partition(labels)


def canonical_from_partition(part: np.ndarray):
    """Any partition numbering (-1 = medium) -> min-index labels, sizes by min index, hist."""
    flat = part.reshape(-1)
    occ = flat >= 0
    labels = np.full(flat.shape, -1, dtype=np.int64)
    if occ.any():
        ids = flat[occ]
        sites = np.nonzero(occ)[0]
        uniq, inv = np.unique(ids, return_inverse=True)
        mins = np.full(uniq.size, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(mins, inv, sites)
        labels[occ] = mins[inv]
        counts = np.bincount(inv, minlength=uniq.size)
        order = np.argsort(mins)
        sizes = counts[order].astype(np.int64)
    else:
        sizes = np.zeros(0, dtype=np.int64)
    return labels.reshape(part.shape).astype(np.int32), sizes, log2_hist(sizes), int(sizes.size)


def interior_tags(index: np.ndarray, periodic):
    """Sec. 6, step 5, from the definitions: clusters of the far sites (I < -0.5) by
    BFS; every face pair (cluster site, near site) adds the sign of I at the near
    site to its cluster (the six directions with the periodic wraps); a negative sum
    is interior (1), a positive one exterior (0), zero undetermined (-1).  Returns
    (labels, sizes, hist, n, tags) with clusters in order of their first site."""
    occ = index < -0.5
    labels, sizes, hist, n = bfs_label(occ, periodic)
    nz, ny, nx = index.shape
    dims = (nx, ny, nz)
    roots = sorted({int(v) for v in labels.reshape(-1) if v >= 0})
    order = {r: k for k, r in enumerate(roots)}
    votes = [0] * len(roots)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if occ[z, y, x]:
                    continue
                v = float(index[z, y, x])
                sign = -1 if v < 0 else (1 if v > 0 else 0)   # NaN compares false: no vote
                if sign == 0:
                    continue
                for (ax, ay, az) in neighbours(x, y, z, dims, periodic):
                    if occ[az, ay, ax]:
                        votes[order[int(labels[az, ay, ax])]] += sign
    tags = np.array([1 if v < 0 else (0 if v > 0 else -1) for v in votes], dtype=np.int8)
    return labels, sizes, hist, n, tags


def interior_state(index: np.ndarray, periodic):
    """Per-site interior state from the definitions: a far site (I < -0.5) takes the
    tag of its BFS cluster (interior_tags), a near site the side its value names:
    1 for I < 0, else 0 (NaN: 0)."""
    labels, _, _, _, tags = interior_tags(index, periodic)
    roots = sorted({int(v) for v in labels.reshape(-1) if v >= 0})
    order = {r: k for k, r in enumerate(roots)}
    state = np.empty(index.shape, dtype=np.int8)
    for pos in np.ndindex(index.shape):
        v = float(index[pos])
        if v < -0.5:
            state[pos] = tags[order[int(labels[pos])]]
        else:
            state[pos] = 1 if v < 0 else 0
    return state
