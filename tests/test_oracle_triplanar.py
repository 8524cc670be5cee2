"""Pins of the oracle's triplanar lookups (Sec. 5 "Triplanar mapping"; Sec. 4.4 material graphs).

Each pin ties the triplanar layer to something fixed outside it: the closed-form blend of
three constant textures (weights |n_i|^4 / sum |n_j|^4 computed here in numpy), the plane
frequencies of the stochastic blend (binomial bounds), the collapse to the separately pinned
2-D lookup when the normal lies along an axis (which fixes the plane <-> coordinate mapping
and the projection of the derivatives), linearity (filter-before = filter-after under the
identity shade, through two separate code paths), and unbiasedness (the stochastic mean
converges to the exact filter-after blend)."""
import math

import numpy as np
import pytest

import oracle
import stf_synth as synth

AXES = {0: ("py", "pz"), 1: ("px", "pz"), 2: ("px", "py")}   # plane i reads these coordinates
DCOMP = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


def _const_tex(rgb, rough=0.5, n=8):
    c = np.zeros((n, n, 4), dtype=np.float32)
    c[...] = [*rgb, rough]
    return oracle.Texture([c])


def _material(n=32, seed=5):
    m = synth.material_rgba8(n, seed, octaves=4, base=2)
    return oracle.Texture(m.albedo_rough, m.normal)


def _with_normal(q, nrm):
    n = q.n
    f = lambda x: np.full(n, x, dtype=np.float32)
    return synth.TriQueries(q.px, q.py, q.pz, f(nrm[0]), f(nrm[1]), f(nrm[2]), q.dpdx, q.dpdy)


def _blend_weights(q):
    N = np.stack([q.nx, q.ny, q.nz]).astype(np.float64)
    w = N ** 4
    return (w / w.sum(axis=0)).T


def _plane_2d(q, i, scale):
    """The 2-D query plane i sees (FP32 products, as the method forms them)."""
    s = np.float32(scale)
    u = getattr(q, AXES[i][0]) * s
    v = getattr(q, AXES[i][1]) * s
    if q.dpdx is None:
        return synth.Queries(u, v)
    a, b = DCOMP[i]
    return synth.Queries(u, v, q.dpdx[a] * s, q.dpdx[b] * s, q.dpdy[a] * s, q.dpdy[b] * s)


@pytest.mark.parametrize("filter,mode", [("linear", "stochastic"), ("bspline", "stochastic"),
                                         ("linear", "ntap_before"), ("bspline", "ntap_after"),
                                         ("mitchell", "ntap_after"), ("catmull_rom", "ntap_before")])
def test_constant_textures_blend_in_closed_form(filter, mode):
    # three constant textures (one per plane) under the identity shade: every sample of every
    # mode with a non-negative filter, and the N-tap modes of any filter, return sum_i b_i c_i
    cols = [(0.9, 0.1, 0.2), (0.1, 0.8, 0.3), (0.2, 0.3, 0.7)]
    texs = [_const_tex(c) for c in cols]
    q = synth.queries_triplanar(300, 11, res=8, lod_range=2.0)
    r = oracle.triplanar_shade(texs, q, 1.0, filter, mode, "full", "linear", spp=2, seed=3)
    want = _blend_weights(q) @ np.array(cols, dtype=np.float32).astype(np.float64)
    np.testing.assert_allclose(r.rgb, want, rtol=0, atol=1e-12)


def test_stochastic_blend_draws_planes_with_the_blend_weights():
    # plane i's texture is the unit colour e_i, so each 1-spp result names the plane drawn;
    # over 20000 ids the frequency of plane i must match b_i within 5 binomial sigmas
    texs = [_const_tex(c) for c in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    base = synth.queries_triplanar(20000, 12, res=8, derivs=False)
    for nrm in ((0.2, 0.5, 0.84), (-0.7, 0.1, 0.7), (0.577, -0.577, 0.577)):
        q = _with_normal(base, nrm)
        r = oracle.triplanar_shade(texs, q, 1.0, "bspline", "stochastic", "stochastic", "linear", spp=1, seed=9)
        assert np.all(np.isin(r.rgb, (0.0, 1.0))) and np.all(r.rgb.sum(axis=1) == 1.0)
        b = _blend_weights(q)[0]
        freq = r.rgb.mean(axis=0)
        sd = np.sqrt(b * (1 - b) / q.n)
        assert np.all(np.abs(freq - b) <= 5 * sd + 1e-12), (freq, b)


@pytest.mark.parametrize("axis,sign", [(0, 1), (1, -1), (2, 1), (2, -1)])
@pytest.mark.parametrize("mode,filter,flags", [("stochastic", "bspline", 0),
                                               ("stochastic", "mitchell", oracle.FLAG_LATTICE),
                                               ("positivized", "catmull_rom", 0),
                                               ("ntap_after", "linear", oracle.FLAG_STRATIFIED),
                                               ("ntap_before", "bspline", oracle.FLAG_STRATIFIED)])
@pytest.mark.parametrize("blend", ["full", "stochastic"])
def test_axis_normal_reduces_to_the_2d_lookup(axis, sign, mode, filter, flags, blend):
    # a normal along axis i gives b = e_i: the triplanar lookup is then the 2-D lookup of
    # texture i at scale * (the other two coordinates), with the derivatives projected the
    # same way, and the same per-query uniforms
    texs = [_material(32, 5), _material(16, 6), _material(64, 7)]
    nrm = [0.0, 0.0, 0.0]
    nrm[axis] = sign
    q = _with_normal(synth.queries_triplanar(200, 13, res=32, lod_range=4.0), nrm)
    scale = 0.75
    spp = 4
    r = oracle.triplanar_shade(texs, q, scale, filter, mode, blend, "ggx", spp=spp, seed=21, flags=flags,
                               want_picks=True)
    ref = oracle.filter_shade(texs[axis], _plane_2d(q, axis, scale), filter, mode, "ggx", spp=spp, seed=21,
                              flags=flags, want_picks=True)
    np.testing.assert_allclose(r.rgb, ref.rgb, rtol=1e-13, atol=1e-15)
    assert np.array_equal(r.picks[:, :, axis, :], ref.picks)
    others = [i for i in range(3) if i != axis]
    assert np.all(r.picks[:, :, others, :] == oracle.NO_PICK)


def test_zero_normal_uses_the_z_plane():
    texs = [_material(32, 5), _material(16, 6), _material(64, 7)]
    q = _with_normal(synth.queries_triplanar(100, 14, res=32), (0.0, 0.0, 0.0))
    for blend in ("full", "stochastic"):
        r = oracle.triplanar_shade(texs, q, 1.0, "linear", "stochastic", blend, "ggx", spp=2, seed=4)
        ref = oracle.filter_shade(texs[2], _plane_2d(q, 2, 1.0), "linear", "stochastic", "ggx", spp=2, seed=4)
        np.testing.assert_allclose(r.rgb, ref.rgb, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("filter", ["linear", "bspline", "mitchell"])
def test_linear_shade_before_equals_after(filter):
    # the blend and the filters are linear: under the identity shade, blending the filtered
    # materials (one code path) equals blending the filter-after values (the 2-D lookups)
    texs = [_material(32, 5), _material(16, 6), _material(64, 7)]
    q = synth.queries_triplanar(300, 15, res=32, lod_range=4.0)
    a = oracle.triplanar_shade(texs, q, 1.3, filter, "ntap_before", "full", "linear", spp=3, seed=6)
    b = oracle.triplanar_shade(texs, q, 1.3, filter, "ntap_after", "full", "linear", spp=3, seed=6)
    np.testing.assert_allclose(a.rgb, b.rgb, rtol=0, atol=1e-12)


@pytest.mark.parametrize("filter,mode", [("bspline", "stochastic"), ("mitchell", "positivized")])
def test_stochastic_blend_is_unbiased(filter, mode):
    # Eq. stochastic-sum over the blend and the taps: the mean of many samples converges to
    # the exact filter-after blend (same jittered footprint distribution), GGX shading
    texs = [_material(32, 5), _material(16, 6), _material(64, 7)]
    q = synth.queries_triplanar(6, 16, res=32, lod_range=3.0, derivs=False)
    spp = 1 << 15
    s = oracle.triplanar_shade(texs, q, 1.0, filter, mode, "stochastic", "ggx", spp=spp, seed=7)
    a = oracle.triplanar_shade(texs, q, 1.0, filter, "ntap_after", "full", "ggx", spp=1)
    small = np.array([oracle.triplanar_shade(texs, q, 1.0, filter, mode, "stochastic", "ggx", spp=1,
                                             seed=500 + k).rgb for k in range(256)])
    sd = small.std(axis=0) + 1e-6
    z = np.abs(s.rgb - a.rgb) / (sd / math.sqrt(spp))
    assert z.max() < 4.5, z.max()


def test_invalid_arguments_are_rejected():
    texs = [_material(16, 5)] * 3
    q = synth.queries_triplanar(10, 17, res=16)
    with pytest.raises(ValueError):
        oracle.triplanar_shade(texs, q, 1.0, "linear", "positivized", "full")
    with pytest.raises(ValueError):
        oracle.triplanar_shade(texs, q, 0.0, "linear", "stochastic", "full")
    with pytest.raises(ValueError):
        oracle.triplanar_shade(texs, q, 1.0, "linear", "stochastic", "full", flags=oracle.FLAG_REUSE)
