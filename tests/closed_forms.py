"""Closed-form expected values used by the tests (outputs of the method, not inputs).

- block_labels_device: the labels of the Sec. 3 benchmark pattern
  (fields.block_field_device): each occupied cubic domain is one cluster
  labelled by its corner, the smallest row-major index of the domain;
- capsule_interior_count: the number of sites a voxelised ellipsoidal shell
  encloses, counted directly from the ellipsoid's equation.
Both are pinned against the oracle at small sizes (tests/test_oracle_pins.py).
"""
import numpy as np


def block_labels_device(L: int, b: int, device="cuda"):
    """Closed-form labels of block_field_device(L, b): the smallest row-major index of
    each occupied domain (its corner), -1 for the medium."""
    import torch
    c = torch.div(torch.arange(L, device=device, dtype=torch.int32), b, rounding_mode="floor")
    corner = c * b
    lab = (corner.view(L, 1, 1) * (L * L) + corner.view(1, L, 1) * L + corner.view(1, 1, L))
    par = (c.view(L, 1, 1) + c.view(1, L, 1) + c.view(1, 1, L)) & 1
    return torch.where(par == 0, lab, torch.full_like(lab, -1))


def capsule_interior_count(L: int, semi_axes: tuple) -> int:
    """Number of interior sites: F <= 1 with all six neighbours F <= 1 (counted directly)."""
    a = np.asarray(semi_axes, dtype=np.float64)
    g = np.arange(-1, L + 1, dtype=np.float64) - L / 2.0
    F = (g / a[2])[:, None, None] ** 2 + (g / a[1])[None, :, None] ** 2 + (g / a[0])[None, None, :] ** 2
    inside = F <= 1.0
    core = inside[1:-1, 1:-1, 1:-1].copy()
    for sl in ((slice(0, -2), slice(1, -1), slice(1, -1)), (slice(2, None), slice(1, -1), slice(1, -1)),
               (slice(1, -1), slice(0, -2), slice(1, -1)), (slice(1, -1), slice(2, None), slice(1, -1)),
               (slice(1, -1), slice(1, -1), slice(0, -2)), (slice(1, -1), slice(1, -1), slice(2, None))):
        core &= inside[sl]
    return int(core.sum())
