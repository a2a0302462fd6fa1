"""Seeded synthetic order-parameter fields phi (host side, numpy).

This module only draws inputs; it holds none of the labelling arithmetic and
is shared by the CUDA path's tests and benchmark and by the oracle's tests.
The paper's workloads come from lattice-Boltzmann runs (emulsions, Sec. 5;
capsules, Sec. 6) that are not reproducible here, so these seeded fields stand
in for them with the same shapes and structure.

Random stream.  u(seed, k) = (splitmix64((seed << 40) + k) >> 40) * 2**-24, an
exact float32 in [0, 1).  splitmix64 is the finaliser published by Steele, Lea
and Flood (OOPSLA 2014, "Fast splittable pseudorandom number generators"):
add the golden-ratio increment 0x9E3779B97F4A7C15, then two xor-shift /
multiply rounds (shifts 30 and 27, multipliers 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB) and a final xor-shift by 31.  The CUDA generator in the
library implements the same definition, so both sides can draw identical
fields; parity tests nevertheless always label the exact bytes they compare.

Layout: every field is a C-contiguous float32 array of shape (nz, ny, nx), so
the row-major site index is s = x + nx * (y + ny * z).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """The splitmix64 finaliser applied elementwise to a uint64 array."""
    z = np.asarray(x, dtype=np.uint64) + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, k) -> np.ndarray:
    """u(seed, k): exact float32 uniforms in [0, 1) for counters k."""
    k = np.asarray(k, dtype=np.uint64)
    h = splitmix64((np.uint64(seed) << np.uint64(40)) + k)
    return (h >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)


def uniform_scalar(seed: int, k: int) -> float:
    return float(uniform(seed, np.array([k], dtype=np.uint64))[0])


def iid_field(nx: int, ny: int, nz: int, seed: int, occupancy: float, out: np.ndarray | None = None,
              chunk_sites: int = 1 << 24) -> np.ndarray:
    """phi = u(seed, s) - (1 - occupancy) in float32 (so P[phi > 0] = occupancy).

    The subtraction is one float32 operation, exactly as on the device.
    """
    n = nx * ny * nz
    if out is None:
        out = np.empty((nz, ny, nx), dtype=np.float32)
    flat = out.reshape(-1)
    c = np.float32(1.0 - occupancy)
    for s0 in range(0, n, chunk_sites):
        s1 = min(n, s0 + chunk_sites)
        flat[s0:s1] = uniform(seed, np.arange(s0, s1, dtype=np.uint64)) - c
    return out


def constant_field(nx: int, ny: int, nz: int, value: float) -> np.ndarray:
    return np.full((nz, ny, nx), value, dtype=np.float32)


def block_field_device(L: int, b: int, device="cuda"):
    """The benchmark pattern of Sec. 3 on an L^3 lattice, built on the device with torch:
    cubic domains of b^3 sites, domain (i, j, k) occupied (phi = +1) iff i + j + k is
    even, else phi = -1.  Occupied domains touch only along edges and corners, so with
    an even number L / b of domains per axis (also across periodic wraps) there are
    (L / b)^3 / 2 clusters of b^3 sites; b = 1 is the site checkerboard, V / 2 clusters."""
    import torch
    c = (torch.div(torch.arange(L, device=device, dtype=torch.int32), b, rounding_mode="floor") & 1).to(torch.int8)
    par = (c.view(L, 1, 1) + c.view(1, L, 1) + c.view(1, 1, L)) & 1
    return (1 - 2 * par).to(torch.float32)


def sphere_params(n_spheres: int, box: tuple, seed: int, r_lo: float = 5.0, r_hi: float = 15.0):
    """Centres uniform in the box and radii uniform in [r_lo, r_hi] from stream ``seed``.

    Sphere i draws counters 4i..4i+3: (cx, cy, cz, r).  ``box`` is (nx, ny, nz).
    """
    k = np.arange(4 * n_spheres, dtype=np.uint64)
    u = uniform(seed, k).astype(np.float64).reshape(n_spheres, 4)
    centres = u[:, :3] * np.array(box, dtype=np.float64)
    radii = r_lo + (r_hi - r_lo) * u[:, 3]
    return centres, radii


def emulsion_field(nx: int, ny: int, nz: int, n_spheres: int, seed: int, r_lo: float = 5.0,
                   r_hi: float = 15.0, reach: float = 8.0) -> np.ndarray:
    """Droplet field: phi(x) = max_i tanh((r_i - d_i(x)) / 2), -1 beyond d_i > r_i + reach.

    d_i is the periodic minimum-image distance from site x to centre c_i, so
    droplets wrap around the box and overlapping droplets form one cluster.
    """
    phi = np.full((nz, ny, nx), -1.0, dtype=np.float32)
    centres, radii = sphere_params(n_spheres, (nx, ny, nz), seed, r_lo, r_hi)
    dims = (nx, ny, nz)
    for c, r in zip(centres, radii):
        ext = r + reach
        idx, dist = [], []
        for a in range(3):
            lo, hi = int(math.floor(c[a] - ext)), int(math.ceil(c[a] + ext))
            coords = np.arange(lo, hi + 1)
            if coords.size > dims[a]:
                coords = np.arange(dims[a])
            w = np.mod(coords, dims[a])
            w = np.unique(w)
            d = np.abs(w - c[a])
            d = np.minimum(d, dims[a] - d)
            idx.append(w)
            dist.append(d)
        dz, dy, dx = dist[2][:, None, None], dist[1][None, :, None], dist[0][None, None, :]
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        val = np.where(d <= ext, np.tanh((r - d) / 2.0), -1.0).astype(np.float32)
        sub = np.ix_(idx[2], idx[1], idx[0])
        phi[sub] = np.maximum(phi[sub], val)
    return phi


def capsule_field(L: int, semi_axes: tuple) -> np.ndarray:
    """Voxelised closed ellipsoidal shell: phi = -1 on the shell, +1 elsewhere.

    F(x) = sum_i ((x_i - L/2) / a_i)^2.  The shell is {F <= 1 with a
    6-neighbour F > 1}; any 6-path from F <= 1 to F > 1 crosses it, so the
    shell separates the interior from the exterior (the index-field set-up of
    Sec. 6, steps 1-3, with a one-site transition layer).  Semi-axes must be
    at most L/2 - 2 so the shell stays away from the box faces.
    """
    a = np.asarray(semi_axes, dtype=np.float64)
    if np.any(a > L / 2 - 2) or np.any(a <= 0):
        raise ValueError("semi-axes must be in (0, L/2 - 2]")
    g = np.arange(-1, L + 1, dtype=np.float64) - L / 2.0
    fx = (g / a[0]) ** 2
    fy = (g / a[1]) ** 2
    fz = (g / a[2]) ** 2
    F = fz[:, None, None] + fy[None, :, None] + fx[None, None, :]   # padded by one site
    inside = F <= 1.0
    core = inside[1:-1, 1:-1, 1:-1]
    outside_nb = np.zeros_like(core)
    for sl in ((slice(0, -2), slice(1, -1), slice(1, -1)), (slice(2, None), slice(1, -1), slice(1, -1)),
               (slice(1, -1), slice(0, -2), slice(1, -1)), (slice(1, -1), slice(2, None), slice(1, -1)),
               (slice(1, -1), slice(1, -1), slice(0, -2)), (slice(1, -1), slice(1, -1), slice(2, None))):
        outside_nb |= ~inside[sl]
    shell = core & outside_nb
    return np.where(shell, np.float32(-1.0), np.float32(1.0)).astype(np.float32)


INDEX_FAR = np.float32(-1.0)      # I_0 < -0.5: far from every membrane (Sec. 6, step 1)
INDEX_INNER = np.float32(-0.25)   # near a membrane, inner side (Sec. 6, step 2: -d)
INDEX_OUTER = np.float32(0.25)    # near a membrane, outer side (+d)


def capsule_params(n: int, shape: tuple, seed: int, a_lo: float = 6.0, a_hi: float = 20.0, tries: int = 1000):
    """Up to n non-overlapping ellipsoidal capsules inside a box of shape (nz, ny, nx).

    Candidate j draws counters 6j..6j+5 of stream ``seed``: a centre uniform in
    the box shrunk by the largest semi-axis + 3 on each side, and three semi-axes
    uniform in [a_lo, a_hi].  A candidate is kept when its bounding sphere stays
    3 sites clear of every kept one.  Returns a list of (centre_xyz, axes_xyz).
    """
    nz, ny, nx = shape
    box = (nx, ny, nz)
    kept = []
    for j in range(tries):
        if len(kept) == n:
            break
        u = uniform(seed, np.arange(6 * j, 6 * j + 6, dtype=np.uint64)).astype(np.float64)
        axes = tuple(a_lo + (a_hi - a_lo) * u[3 + i] for i in range(3))
        m = max(axes) + 3.0
        if any(2 * m >= b for b in box):
            continue
        centre = tuple(m + (box[i] - 2 * m) * u[i] for i in range(3))
        ok = all(np.linalg.norm(np.subtract(centre, c)) > m + max(a) + 3.0 for c, a in kept)
        if ok:
            kept.append((centre, axes))
    return kept


def capsule_index_field(shape: tuple, capsules) -> np.ndarray:
    """Index field I of Sec. 6 (steps 1-2) for closed ellipsoidal membranes.

    For capsule c, F_c(x) = sum_i ((x_i - c_i) / a_i)^2 (float64, summed z, y, x).
    Sites with F_c <= 1 and a 6-neighbour F_c > 1 form the inner layer
    (I = -0.25), sites with F_c > 1 and a 6-neighbour F_c <= 1 the outer layer
    (I = +0.25); every other site is far (I = -1).  The two layers close around
    each capsule, so they separate its interior from the exterior.  Capsules must
    stay clear of each other and of the box faces (``capsule_params`` ensures
    both).  F_c is evaluated only on the capsule's bounding box grown by two
    sites: beyond it F_c > 1 at a site and at all its neighbours.
    """
    nz, ny, nx = shape
    I = np.full(shape, INDEX_FAR, dtype=np.float32)
    for (cx, cy, cz), (ax, ay, az) in capsules:
        lo = [max(0, int(np.floor(c - a)) - 2) for c, a in ((cz, az), (cy, ay), (cx, ax))]
        hi = [min(n, int(np.ceil(c + a)) + 3) for c, a, n in ((cz, az, nz), (cy, ay, ny), (cx, ax, nx))]
        # coordinates of the box and one site around it (the neighbours of its sites)
        z = np.arange(lo[0] - 1, hi[0] + 1, dtype=np.float64)
        y = np.arange(lo[1] - 1, hi[1] + 1, dtype=np.float64)
        x = np.arange(lo[2] - 1, hi[2] + 1, dtype=np.float64)
        F = (((z - cz) / az) ** 2)[:, None, None] + (((y - cy) / ay) ** 2)[None, :, None] \
            + (((x - cx) / ax) ** 2)[None, None, :]
        inside = F <= 1.0
        core = inside[1:-1, 1:-1, 1:-1]
        any_out = np.zeros_like(core)
        any_in = np.zeros_like(core)
        for sl in ((slice(0, -2), slice(1, -1), slice(1, -1)), (slice(2, None), slice(1, -1), slice(1, -1)),
                   (slice(1, -1), slice(0, -2), slice(1, -1)), (slice(1, -1), slice(2, None), slice(1, -1)),
                   (slice(1, -1), slice(1, -1), slice(0, -2)), (slice(1, -1), slice(1, -1), slice(2, None))):
            any_out |= ~inside[sl]
            any_in |= inside[sl]
        box = I[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        box[~core & any_in] = INDEX_OUTER
        box[core & any_out] = INDEX_INNER
    return I


# ----------------------------------------------------------------------------------------------
# Workload recipes (shapes, sizes and value distributions of the paper's use cases)
# ----------------------------------------------------------------------------------------------

P_C_SIMPLE_CUBIC = 0.3116   # site-percolation threshold of the simple cubic lattice
AXIS_CHOICES = tuple(range(32, 385, 16))   # {32, 48, ..., 384}: 23 values


def small_iid():
    """32^3, occupancy 0.3, seed 0, periodic in x, y, z."""
    return iid_field(32, 32, 32, seed=0, occupancy=0.3), (1, 1, 1)


def emulsion_256():
    """256^3 emulsion-like field: 600 droplets, r in [5, 15], stream seed 1, periodic."""
    return emulsion_field(256, 256, 256, 600, seed=1), (1, 1, 1)


def critical_1024(out: np.ndarray | None = None):
    """1024^3 iid field at the simple-cubic percolation threshold, seed 0, periodic."""
    return iid_field(1024, 1024, 1024, seed=0, occupancy=P_C_SIMPLE_CUBIC, out=out), (1, 1, 1)


def batch_params(n_lattices: int = 96, master_seed: int = 2):
    """Shapes, occupancies, periodic flags and phi seeds of the uneven batch.

    Lattice i draws counters 8i..8i+6 of stream ``master_seed``: three axis
    lengths from {32, 48, ..., 384}, occupancy in [0.15, 0.45] and three
    Bernoulli(0.5) periodic flags; its phi uses seed 1000 + i.
    """
    out = []
    for i in range(n_lattices):
        u = uniform(master_seed, np.arange(8 * i, 8 * i + 7, dtype=np.uint64)).astype(np.float64)
        dims = tuple(AXIS_CHOICES[min(int(u[k] * len(AXIS_CHOICES)), len(AXIS_CHOICES) - 1)] for k in range(3))
        occ = 0.15 + 0.30 * u[3]
        per = tuple(int(u[4 + k] < 0.5) for k in range(3))
        out.append({"nx": dims[0], "ny": dims[1], "nz": dims[2], "occupancy": float(occ),
                    "periodic": per, "seed": 1000 + i})
    return out
