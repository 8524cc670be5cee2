"""Host-side arithmetic of bench.py (CPU only)."""
import numpy as np

import bench


def _brute_hit(texels, l2_bytes, texel_bytes=8.0):
    # every texel's read probability, hottest first, filled into the cache byte by byte
    p = np.concatenate([np.full(t, 1.0 / (len(texels) * t)) for t in texels])
    p = np.sort(p)[::-1]
    slots = l2_bytes / texel_bytes
    whole = int(np.floor(slots))
    return float(p[:whole].sum() + (slots - whole) * (p[whole] if whole < p.size else 0.0))


def test_ideal_l2_hit_matches_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        texels = rng.integers(1, 400, rng.integers(1, 12)).tolist()
        total = 8.0 * sum(texels)
        for l2 in (0.0, 8.0, 0.37 * total, 0.9 * total, total, 2 * total):
            assert abs(bench.ideal_l2_hit(texels, l2) - min(1.0, _brute_hit(texels, l2))) < 1e-12


def test_ideal_l2_hit_of_equal_textures_is_the_cached_share():
    assert abs(bench.ideal_l2_hit([100] * 10, 8.0 * 250) - 0.25) < 1e-15
