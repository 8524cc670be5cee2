"""Parity of the CUDA triplanar lookups (Sec. 5 "Triplanar mapping"; Sec. 4.4) with the FP64 oracle.

Decisions (plane coordinates, blend weights, the plane pick, levels, texel picks) are FP32 in
the same order on both sides, so picks agree bit for bit except next to an FP64 boundary.
Values: the kernel blends with FP32 weights w_i / W (four roundings, ~5e-7 relative) on top
of the 2-D lookups' FP32 arithmetic, inside the 1e-5 relative bound of the 2-D tests."""
import numpy as np
import pytest

import oracle
import stf_synth as synth
from gpu_util import REL_DCT, assert_values, compare_picks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")



@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_06107_b300 as stf
    c = stf.Context(0)
    yield c
    c.close()


def _upload_material(ctx, m):
    return ctx.create_texture(m.albedo_rough, m.normal)


@pytest.fixture(scope="module")
def planes(ctx):
    """Three RGBA8 + RG8 materials of different sizes, one per plane."""
    ms = [synth.material_rgba8(n, s, octaves=5, base=4) for n, s in ((128, 31), (64, 32), (256, 33))]
    return [_upload_material(ctx, m) for m in ms], [oracle.Texture(m.albedo_rough, m.normal) for m in ms]


@pytest.fixture(scope="module")
def dct_planes(ctx):
    ms = [synth.material_rgba8(n, s, octaves=5, base=4) for n, s in ((128, 34), (256, 35), (128, 36))]
    hs, ts = [], []
    for m in ms:
        blocks = synth.dct_compress(m)
        w = m.albedo_rough[0].shape[1]
        hs.append(ctx.create_texture_dct(blocks, w, w))
        ts.append(oracle.Texture([lv.shape[:2] for lv in m.albedo_rough], dct=blocks))
    return hs, ts


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(ctx, hs, q, scale, filter, mode, blend, spp, seed=1, flags=0, picks=True, order=None, out=None):
    p = [_dev(q.px), _dev(q.py), _dev(q.pz)]
    nrm = [_dev(q.nx), _dev(q.ny), _dev(q.nz)]
    d = [_dev(x) for x in (*q.dpdx, *q.dpdy)] if q.dpdx is not None else None
    r, g, b, pk = ctx.triplanar_shade(hs, scale, p, nrm, d, filter, mode, blend, "ggx", spp, seed, flags,
                                      want_picks=picks, order=order, out=out)
    torch.cuda.synchronize()
    rgb = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    return rgb, (pk.cpu().numpy().view(np.uint32) if pk is not None else None)


CASES = [("linear", "stochastic", "stochastic", 1, 0), ("linear", "stochastic", "stochastic", 3, 0),
         ("bspline", "stochastic", "stochastic", 4, oracle.FLAG_LATTICE),
         ("bspline", "stochastic", "stochastic", 4, oracle.FLAG_STRATIFIED),
         ("mitchell", "stochastic", "full", 2, 0), ("catmull_rom", "stochastic", "stochastic", 2, oracle.FLAG_LOD0),
         ("catmull_rom", "positivized", "stochastic", 2, 0), ("mitchell", "positivized", "full", 2, oracle.FLAG_LATTICE),
         ("linear", "ntap_before", "full", 1, 0), ("bspline", "ntap_before", "full", 4, oracle.FLAG_STRATIFIED),
         ("linear", "ntap_after", "full", 1, 0), ("mitchell", "ntap_after", "stochastic", 2, 0),
         ("bspline", "ntap_before", "stochastic", 2, 0)]


@pytest.mark.parametrize("filter,mode,blend,spp,flags", CASES)
def test_triplanar_matches_oracle(ctx, planes, filter, mode, blend, spp, flags):
    hs, ts = planes
    q = synth.queries_triplanar(3001, 41, res=128, scale=1.5, lod_range=6.0)
    rgb, pk = _run(ctx, hs, q, 1.5, filter, mode, blend, spp, seed=7, flags=flags)
    ref = oracle.triplanar_shade(ts, q, 1.5, filter, mode, blend, "ggx", spp, 7, flags=flags, want_picks=True)
    mism = compare_picks(pk, ref, q.n * 3)
    assert_values(rgb, ref.rgb, mism, scale=ref.mag)
    # the specialised kernels (no picks) return the same values
    rgb2, _ = _run(ctx, hs, q, 1.5, filter, mode, blend, spp, seed=7, flags=flags, picks=False)
    assert_values(rgb2, ref.rgb, mism, scale=ref.mag)


@pytest.mark.parametrize("filter,mode,blend,spp", [("linear", "stochastic", "stochastic", 1),
                                                   ("linear", "ntap_before", "full", 1),
                                                   ("bspline", "stochastic", "full", 2),
                                                   ("mitchell", "positivized", "stochastic", 2)])
def test_triplanar_dct_matches_oracle(ctx, dct_planes, filter, mode, blend, spp):
    hs, ts = dct_planes
    q = synth.queries_triplanar(2500, 42, res=128, lod_range=5.0)
    rgb, pk = _run(ctx, hs, q, 1.0, filter, mode, blend, spp, seed=8)
    ref = oracle.triplanar_shade(ts, q, 1.0, filter, mode, blend, "ggx", spp, 8, want_picks=True)
    mism = compare_picks(pk, ref, q.n * 3)
    assert_values(rgb, ref.rgb, mism, rel=REL_DCT, scale=ref.mag)
    rgb2, _ = _run(ctx, hs, q, 1.0, filter, mode, blend, spp, seed=8, picks=False)
    assert_values(rgb2, ref.rgb, mism, rel=REL_DCT, scale=ref.mag)


def test_triplanar_edge_cases(ctx, planes):
    hs, ts = planes
    # no derivatives: no jitter, level 0
    q = synth.queries_triplanar(777, 43, res=128, derivs=False)
    rgb, pk = _run(ctx, hs, q, 2.0, "bspline", "stochastic", "stochastic", 2, seed=9)
    ref = oracle.triplanar_shade(ts, q, 2.0, "bspline", "stochastic", "stochastic", "ggx", 2, 9, want_picks=True)
    assert_values(rgb, ref.rgb, compare_picks(pk, ref, q.n * 3), scale=ref.mag)
    # axis-aligned and zero normals (one plane only), negative coordinates, tiny n
    q = synth.queries_triplanar(300, 44, res=128)
    nrm = np.zeros((3, q.n), dtype=np.float32)
    nrm[np.arange(q.n) % 3, np.arange(q.n)] = np.where(np.arange(q.n) % 2, 1.0, -1.0)
    nrm[:, ::7] = 0.0
    q = synth.TriQueries(-q.px, q.py - 3.0, q.pz, nrm[0], nrm[1], nrm[2], q.dpdx, q.dpdy)
    for n in (1, 255, 257, 300):
        qs = q.subset(np.arange(n))
        for blend in ("full", "stochastic"):
            rgb, pk = _run(ctx, hs, qs, 1.0, "mitchell", "stochastic", blend, 2, seed=10)
            ref = oracle.triplanar_shade(ts, qs, 1.0, "mitchell", "stochastic", blend, "ggx", 2, 10, want_picks=True)
            assert_values(rgb, ref.rgb, compare_picks(pk, ref, qs.n * 3), scale=ref.mag)


def test_triplanar_order_and_empty(ctx, planes):
    hs, _ = planes
    q = synth.queries_triplanar(5000, 45, res=128)
    perm = torch.from_numpy(np.random.default_rng(3).permutation(q.n).astype(np.int32)).cuda()
    for spp in (2, 1):    # one sample, no picks: two points per thread
        a, _ = _run(ctx, hs, q, 1.0, "linear", "stochastic", "stochastic", spp, seed=11, picks=False)
        b, _ = _run(ctx, hs, q, 1.0, "linear", "stochastic", "stochastic", spp, seed=11, picks=False, order=perm)
        assert np.array_equal(a, b)
        c, _ = _run(ctx, hs, q, 1.0, "linear", "stochastic", "stochastic", spp, seed=11, picks=True)
        assert np.array_equal(a, c)
    e = synth.queries_triplanar(0, 46, res=128)
    rgb, _ = _run(ctx, hs, e, 1.0, "linear", "stochastic", "stochastic", 1, picks=False)
    assert rgb.shape == (0, 3)


def test_triplanar_full_size_sampled(ctx):
    """The bench's launch (2^22 surface points, the 4096^2 material on all three planes, 1-tap
    trilinear, stochastic blend, 1 spp, the specialised kernel) checked on 2000 sampled
    queries that the oracle evaluates one by one with their own ids."""
    m = synth.material_rgba8(4096, 102)
    h = _upload_material(ctx, m)
    otex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_triplanar(1 << 22, 47, res=4096, lod_range=6.0)
    rgb, _ = _run(ctx, [h, h, h], q, 1.0, "linear", "stochastic", "stochastic", 1, seed=12, picks=False)
    idx = np.random.default_rng(5).choice(q.n, 2000, replace=False)
    ref = oracle.triplanar_shade([otex] * 3, q.subset(idx), 1.0, "linear", "stochastic", "stochastic", "ggx", 1, 12,
                                 ids=idx)
    # no picks from the specialised kernel: allow the boundary cases by their distance
    near = ref.bdist < 1e-6
    assert near.sum() <= 2
    assert_values(rgb[idx], ref.rgb, near, scale=ref.mag)
    ctx.destroy_texture(h)


def test_triplanar_rejects_bad_arguments(ctx, planes, dct_planes):
    import paper_2407_06107_b300 as stf
    hs, _ = planes
    q = synth.queries_triplanar(10, 48, res=128)

    def status(*args, **kw):
        with pytest.raises(stf.StfError) as e:
            _run(ctx, *args, **kw)
        return e.value.status
    assert status([hs[0], dct_planes[0][0], hs[1]], q, 1.0, "linear", "stochastic", "full", 1) == 1
    assert status(hs, q, 1.0, "linear", "stochastic", "full", 1, flags=oracle.FLAG_REUSE) == 5
    assert status(hs, q, 1.0, "linear", "positivized", "full", 1) == 5
    assert status(hs, q, 0.0, "linear", "stochastic", "full", 1) == 1
    assert status(hs, q, float("nan"), "linear", "stochastic", "full", 1) == 1
    assert status([hs[0], hs[1], 123456789], q, 1.0, "linear", "stochastic", "full", 1) == 2
    assert status(hs, q, 1.0, "ewa", "stochastic", "full", 1) == 1


def test_triplanar_nan_input_sets_status(ctx, planes):
    import paper_2407_06107_b300 as stf
    hs, _ = planes
    q = synth.queries_triplanar(64, 49, res=128)
    q.nx[5] = np.nan
    ctx.device_status()      # clear
    _run(ctx, hs, q, 1.0, "linear", "stochastic", "stochastic", 1, picks=False)
    assert ctx.device_status() & stf.DEV_NAN_INPUT
