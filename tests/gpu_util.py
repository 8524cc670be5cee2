"""Helpers shared by the GPU parity tests: tolerance and pick comparison."""
import numpy as np

REL, ABS = 1e-5, 1e-7          # shaded values: |g - o| <= 1e-5 |o| + 1e-7 (FP32 relative 1e-5)
# DCT-compressed textures: the kernel decodes each texel in FP32 (cospif, then five FMAs per
# channel), within ~5e-7 absolute of the FP64 decode; the GGX shade's sensitivity to the
# normal is at most 2/alpha = 40 (alpha >= 0.05), so shaded terms agree within 40 * 5e-7 =
# 2e-5 relative, written as 3e-5 * sum|terms| + 1e-7
REL_DCT = 3e-5
BOUNDARY = 1e-6                # uniforms this close to an FP64 CDF boundary may flip a pick


def compare_picks(gpu_picks, res, n_total):
    """GPU picks vs the oracle's FP64 decisions (`picks64`, the decisions its estimate is
    computed from).  Returns the mask of queries whose picks differ; every such query must
    have a uniform within 1e-6 of an FP64 CDF boundary, and their number must stay below
    1e-5 of the queries (at least one allowed).  The oracle's FP32 decisions (`picks`) are
    a diagnostic and take no part."""
    g = gpu_picks.astype(np.uint32)
    mism = np.any(g != res.picks64, axis=tuple(range(1, g.ndim)))
    bad = mism & ~(res.bdist < BOUNDARY)
    assert not bad.any(), f"{bad.sum()} pick mismatches away from any CDF boundary"
    assert mism.sum() <= max(1, int(np.ceil(1e-5 * n_total))), f"{mism.sum()} boundary mismatches"
    return mism


def assert_values(gpu, ref, mask=None, rel=REL, abs_=ABS, scale=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if mask is not None:
        gpu, ref = gpu[~mask], ref[~mask]
        if scale is not None:
            scale = scale[~mask]
    s = np.abs(ref) if scale is None else scale
    err = np.abs(gpu - ref)
    tol = rel * s + abs_
    worst = np.argmax(err / tol) if err.size else 0
    assert np.all(err <= tol), (f"max err/tol {float((err / tol).max()):.3g} at {np.unravel_index(worst, err.shape)}: "
                                f"gpu {gpu.flat[worst]!r} oracle {ref.flat[worst]!r}")
