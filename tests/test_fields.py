"""The seeded input stream, pinned to its published definition.

fields.splitmix64 is Steele, Lea and Flood's splitmix64 mix of (x + the golden gamma),
so splitmix64(k * gamma) for k = 0, 1, ... is the SplitMix64 generator seeded with 0,
whose first outputs are published; u(seed, k) keeps the top 24 bits as an exact float32.
"""
import numpy as np

from paper_1405_1931_gb300 import fields

GAMMA = 0x9E3779B97F4A7C15
# the first five outputs of SplitMix64 seeded with 0
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                    0x1B39896A51A8749B]


def test_splitmix64_published_outputs():
    states = np.array([(k * GAMMA) % 2 ** 64 for k in range(5)], dtype=np.uint64)
    assert [int(v) for v in fields.splitmix64(states)] == SPLITMIX64_SEED0


def test_uniform_is_the_top_24_bits():
    k = np.arange(1000, dtype=np.uint64)
    u = fields.uniform(7, k)
    h = fields.splitmix64((np.uint64(7) << np.uint64(40)) + k)
    assert u.dtype == np.float32 and (u >= 0).all() and (u < 1).all()
    np.testing.assert_array_equal((u * np.float32(2 ** 24)).astype(np.uint64), h >> np.uint64(40))


def test_iid_field_occupancy_rate():
    """phi = u - (1 - p): P[phi > 0] = p up to the 2^-24 grid; at 64^3 within 5 standard errors."""
    phi = fields.iid_field(64, 64, 64, seed=0, occupancy=0.3116)
    n = phi.size
    frac = float((phi > 0).mean())
    assert abs(frac - 0.3116) < 5 * (0.3116 * 0.6884 / n) ** 0.5
