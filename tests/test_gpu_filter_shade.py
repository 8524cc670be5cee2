"""Parity of the CUDA 2-D filter+shade path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import stf_synth as synth
from gpu_util import assert_values, compare_picks

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


def _dev(q):
    f = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = None
    if q.has_derivs():
        d = [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)]
    return f(q.u), f(q.v), d


def _run(ctx, tex_h, q, filter, mode, spp, seed=1, shade="ggx", flags=0, picks=True, id_base=0):
    u, v, d = _dev(q)
    r, g, b, pk = ctx.filter_shade(tex_h, u, v, d, filter, mode, shade, spp, seed, flags,
                                   id_base=id_base, want_picks=picks)
    torch.cuda.synchronize()
    rgb = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    return rgb, (pk.cpu().numpy().view(np.uint32) if pk is not None else None)


def _check(ctx, tex_h, otex, q, filter, mode, spp, seed=1, shade="ggx", flags=0):
    rgb, pk = _run(ctx, tex_h, q, filter, mode, spp, seed, shade, flags)
    ref = oracle.filter_shade(otex, q, filter, mode, shade, spp, seed, flags, want_picks=True)
    mism = compare_picks(pk, ref, q.n)
    # every summed term (w f_hat, or +-W f_hat) carries its own FP32 relative error, so
    # the tolerance scales with the sum of |terms|: cancellation between signed terms is
    # not mistaken for error
    assert_values(rgb, ref.rgb, mism, scale=ref.mag)
    return rgb, ref


# ---------------------------------------------------------------- config 1: RGBA32F bilinear
@pytest.fixture(scope="module")
def cfg1(ctx):
    tex = synth.texture_rgba32f(256, 101)
    q = synth.queries_uniform(65536, 1, const_derivs=(1 / 1024, 0.0, 0.0, 1 / 1024))
    return ctx.create_texture([tex]), oracle.Texture([tex]), q


@pytest.mark.parametrize("mode,spp", [("ntap_before", 1), ("stochastic", 1), ("stochastic", 16),
                                      ("ntap_after", 4)])
def test_config1_bilinear(ctx, cfg1, mode, spp):
    h, otex, q = cfg1
    _check(ctx, h, otex, q, "linear", mode, spp, seed=1)


# ---------------------------------------------------------------- material with MIPs + normals
@pytest.fixture(scope="module")
def material(ctx):
    m = synth.material_rgba8(256, 102, octaves=6, base=4)
    q = synth.queries_uniform(6000, 3, res=256, lod_range=8.0)
    return ctx.create_texture(m.albedo_rough, m.normal), oracle.Texture(m.albedo_rough, m.normal), q


CASES = [(f, m) for f in ("linear", "bspline", "catmull_rom", "mitchell")
         for m in ("ntap_before", "ntap_after", "stochastic", "positivized")
         if not (m == "positivized" and f in ("linear", "bspline"))]


@pytest.mark.parametrize("filter,mode", CASES)
def test_material_filters(ctx, material, filter, mode):
    h, otex, q = material
    _check(ctx, h, otex, q, filter, mode, spp=3, seed=7)


def test_material_linear_shade_and_stratified(ctx, material):
    h, otex, q = material
    _check(ctx, h, otex, q, "bspline", "ntap_after", spp=4, seed=5, shade="linear", flags=1)
    _check(ctx, h, otex, q, "mitchell", "stochastic", spp=9, seed=5, flags=1)


# ---------------------------------------------------------------- sizes and edge cases
@pytest.mark.parametrize("n", [1, 7, 255, 257, 4097])
def test_ragged_query_counts(ctx, material, n):
    h, otex, q = material
    _check(ctx, h, otex, q.subset(slice(0, n)), "bspline", "stochastic", spp=2, seed=11)


def test_empty_batch_is_noop(ctx, material):
    h, _, _ = material
    e = torch.empty(0, device="cuda")
    r, g, b, _ = ctx.filter_shade(h, e, e, None, "bspline", "stochastic", "ggx", 4, 1)
    assert r.numel() == 0


def test_npot_and_extreme_shapes(ctx):
    # non-power-of-two, 1-texel and maximum-width textures (random texel bytes, every MIP
    # level independent); uv far outside [0, 1) exercises wrap addressing
    rng = np.random.default_rng(12)
    for (hh, ww, lv) in [(37, 100, 1), (1, 1, 1), (2, 16384, 15), (16384, 1, 15), (300, 77, 9)]:
        dims = [(max(1, hh >> i), max(1, ww >> i)) for i in range(lv)]
        ar = [rng.integers(0, 256, (a, b, 4), dtype=np.uint8) for a, b in dims]
        nm = [rng.integers(64, 192, (a, b, 2), dtype=np.uint8) for a, b in dims]   # normals within ~30 deg of +z
        h = ctx.create_texture(ar, nm)
        otex = oracle.Texture(ar, nm)
        q = synth.queries_uniform(2000, 4, res=max(hh, ww), lod_range=float(lv))
        q.u = (q.u * 7.0 - 3.0).astype(np.float32)
        for f, mode in (("mitchell", "positivized"), ("bspline", "stochastic"), ("linear", "ntap_before"),
                        ("catmull_rom", "ntap_after")):
            rgb, _ = _check(ctx, h, otex, q, f, mode, spp=2, seed=3)
            # without pick output the specialised kernels run (the power-of-two shapes in the
            # RGBA8N family, where wrap addressing is a mask; the others in the general family):
            # the same values bit for bit
            rgb2, _ = _run(ctx, h, q, f, mode, 2, seed=3, picks=False)
            np.testing.assert_array_equal(rgb2, rgb)
        ctx.destroy_texture(h)


@pytest.mark.parametrize("filter,mode", [("mitchell", "positivized"), ("bspline", "stochastic"),
                                         ("catmull_rom", "ntap_after"), ("linear", "ntap_before")])
def test_grazing_normals(ctx, filter, mode):
    # tangent-space normals up to 85 degrees from +z, so n.l and n.v reach down to a few
    # hundredths and the GGX factors (tan^2 of the Smith terms, 1/(n.v)) are at their worst
    # conditioned; the per-term FP32 tolerance of the other parity tests must still hold
    rng = np.random.default_rng(31)
    dims = [(128 >> i, 128 >> i) for i in range(8)]
    ar = [rng.integers(0, 256, (a, b, 4), dtype=np.uint8) for a, b in dims]
    nm = []
    for a, b in dims:
        th = np.radians(85.0) * np.sqrt(rng.random((a, b)))
        ph = 2 * np.pi * rng.random((a, b))
        xy = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph)], -1)
        nm.append(np.clip(np.rint((xy + 1) * 127.5), 0, 255).astype(np.uint8))
    h = ctx.create_texture(ar, nm)
    otex = oracle.Texture(ar, nm)
    q = synth.queries_uniform(6000, 32, res=128, lod_range=7.0)
    _check(ctx, h, otex, q, filter, mode, spp=3, seed=19)
    ctx.destroy_texture(h)


def test_id_base_shards_reproduce_whole(ctx, material):
    # query ids key the Philox counter: two shards with id_base equal one launch
    h, _, q = material
    whole, _ = _run(ctx, h, q, "mitchell", "stochastic", 4, seed=21, picks=False)
    a, _ = _run(ctx, h, q.subset(slice(0, 2500)), "mitchell", "stochastic", 4, seed=21, picks=False)
    b, _ = _run(ctx, h, q.subset(slice(2500, None)), "mitchell", "stochastic", 4, seed=21, picks=False,
                id_base=2500)
    assert np.array_equal(np.concatenate([a, b]), whole)


@pytest.mark.parametrize("flags,spp", [(0, 5), (oracle.FLAG_LATTICE, 5), (0, 1)])
@pytest.mark.parametrize("filter", ["linear", "bspline", "catmull_rom", "mitchell"])
def test_specialised_path_equals_general_path(ctx, material, filter, flags, spp):
    # a stochastic call without pick output, with no flag or the lattice flag alone, runs a
    # specialised instantiation (at one sample and no flags: two queries per thread); it does
    # the same arithmetic as the general one, so the results are identical
    h, _, q = material
    with_picks, _ = _run(ctx, h, q, filter, "stochastic", spp, seed=6, flags=flags, picks=True)
    special, _ = _run(ctx, h, q, filter, "stochastic", spp, seed=6, flags=flags, picks=False)
    assert np.array_equal(with_picks, special)


def test_nan_input_sets_device_status(ctx, material):
    h, _, q = material
    q2 = q.subset(slice(0, 64))
    q2.u[5] = np.nan
    ctx.device_status()
    _run(ctx, h, q2, "linear", "stochastic", 1, picks=False)
    import paper_2407_06107_b300 as stf
    assert ctx.device_status() & stf.DEV_NAN_INPUT
    assert ctx.device_status() == 0      # read clears


def test_invalid_arguments(ctx, material):
    import paper_2407_06107_b300 as stf
    h, _, q = material
    u, v, d = _dev(q.subset(slice(0, 16)))
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade(h, u, v, d, "bspline", "positivized", "ggx", 1, 1)
    assert e.value.status == 5
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade(h, u, v, d, "bspline", "stochastic", "ggx", 0, 1)
    assert e.value.status == 1
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade(h, u, v, d, "bspline", "stochastic", "ggx", 3, 1, flags=1)   # not square
    assert e.value.status == 1
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade(h + 999, u, v, d, "bspline", "stochastic", "ggx", 1, 1)
    assert e.value.status == 2


def test_host_entry_point_matches_device(ctx, material):
    h, _, q = material
    dev, pk = _run(ctx, h, q, "mitchell", "positivized", 2, seed=8)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    r, g, b, pk2 = ctx.filter_shade_host(h, f(q.u), f(q.v), [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)],
                                         "mitchell", "positivized", "ggx", 2, 8, want_picks=True)
    assert np.array_equal(np.stack([r, g, b], 1).astype(np.float64), dev)
    assert np.array_equal(pk2, pk)


@pytest.mark.parametrize("filter,flags", [("bspline", 0), ("mitchell", 2)])
def test_host_entry_point_chunked(ctx, material, filter, flags):
    # enough queries (with picks at 8 spp) that the host path pipelines several chunks over
    # its lanes, the last one ragged; query ids stay global, so every result and pick equals
    # the one-launch device path bit for bit
    h, _, _ = material
    q = synth.queries_uniform(4_500_001, 23, res=256, lod_range=5.0)   # three chunks of <= 2^21
    dev, pk = _run(ctx, h, q, filter, "stochastic", 8, seed=4, flags=flags, id_base=77)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    r, g, b, pk2 = ctx.filter_shade_host(h, f(q.u), f(q.v), [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)],
                                         filter, "stochastic", "ggx", 8, 4, flags=flags, id_base=77,
                                         want_picks=True)
    assert np.array_equal(np.stack([r, g, b], 1).astype(np.float64), dev)
    assert np.array_equal(pk2, pk)


# ---------------------------------------------------------------- full size, sampled
@pytest.mark.parametrize("filter,mode", [("linear", "stochastic"), ("bspline", "stochastic"),
                                         ("mitchell", "stochastic"), ("mitchell", "positivized"),
                                         ("bspline", "ntap_before"), ("mitchell", "ntap_before"),
                                         ("linear", "ntap_before")])
def test_full_size_sampled(ctx, filter, mode):
    # the benchmark workload (4096^2 material with MIPs, 16M queries, 8 spp) in the
    # launch configuration bench.py times -- the 1-tap estimators and the N-tap filter-before
    # comparators (8 / 32 / 32 taps over two MIP levels) the equal-RMSE speedups are quoted
    # against; a seeded sample of queries is re-evaluated by the oracle with the same Philox ids
    m = _full_material()
    h = _full_handle(ctx, m)
    q = _full_queries()
    u, v, d = _dev(q)
    r, g, b, _ = ctx.filter_shade(h, u, v, d, filter, mode, "ggx", 8, 1)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(99).choice(q.n, 3000, replace=False))
    rgb = torch.stack([r, g, b], 1)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    ref = oracle.filter_shade(oracle.Texture(m.albedo_rough, m.normal), q.subset(idx), filter,
                              mode, "ggx", 8, 1, ids=idx)
    near = ref.bdist < 1e-6
    assert near.sum() <= 3
    assert_values(rgb, ref.rgb, near, scale=ref.mag)


@pytest.mark.parametrize("filter", ["bspline", "mitchell"])
def test_rmse_reference_matches_oracle(ctx, filter):
    # The bench's equal-RMSE reference is the GPU's exact filter-after pass with 16 x 16
    # stratified footprint samples on the first 2^16 queries of the workload (the bench may not
    # run the oracle).  Pin it to the FP64 oracle on a sample of those queries, value by value,
    # and check that an 8-spp stochastic estimate's RMSE against the GPU reference equals its
    # RMSE against the oracle's to 1e-3 relative.
    m = _full_material()
    h = _full_handle(ctx, m)
    q = _full_queries()
    idx = np.sort(np.random.default_rng(17).choice(1 << 16, 256, replace=False))
    qs = q.subset(idx)
    u, v, d = _dev(qs)
    r, g, b, _ = ctx.filter_shade(h, u, v, d, filter, "ntap_after", "ggx", 256, 1, oracle.FLAG_STRATIFIED)
    R = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    ref = oracle.filter_shade(oracle.Texture(m.albedo_rough, m.normal), qs, filter, "ntap_after", "ggx", 256, 1,
                              oracle.FLAG_STRATIFIED)
    assert_values(R, ref.rgb, scale=ref.mag)
    r, g, b, _ = ctx.filter_shade(h, u, v, d, filter, "stochastic", "ggx", 8, 7, 0)
    S = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    rmse_gpu = np.sqrt(np.mean((S - R) ** 2))
    rmse_oracle = np.sqrt(np.mean((S - ref.rgb) ** 2))
    assert abs(rmse_gpu - rmse_oracle) <= 1e-3 * rmse_oracle, (rmse_gpu, rmse_oracle)


def _full_queries():
    if "q" not in _FULL:
        _FULL["q"] = synth.queries_uniform(1 << 24, 1, res=4096, lod_range=8.0)
    return _FULL["q"]


_FULL = {}


def _full_material():
    if "m" not in _FULL:
        _FULL["m"] = synth.material_rgba8(4096, 102)
    return _FULL["m"]


def _full_handle(ctx, m):
    if "h" not in _FULL:
        _FULL["h"] = ctx.create_texture(m.albedo_rough, m.normal)
    return _FULL["h"]


@pytest.mark.parametrize("filter,mode", [("bspline", "stochastic"), ("mitchell", "positivized"),
                                         ("linear", "stochastic")])
def test_lattice_sampler(ctx, material, filter, mode):
    import oracle as _o
    h, otex, q = material
    _check(ctx, h, otex, q, filter, mode, spp=6, seed=13, flags=_o.FLAG_LATTICE)


def test_binned_order_is_permutation_and_results_identical(ctx, material):
    h, _, q = material
    u, v, d = _dev(q)
    order = ctx.bin_queries(u, v, tile_log2=4)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(q.n))
    # queries appear grouped by tile: tile index is non-decreasing along the order
    fu = np.mod(q.u.astype(np.float64), 1.0)
    fv = np.mod(q.v.astype(np.float64), 1.0)
    tile = (np.minimum((fv * 16).astype(int), 15) << 4) | np.minimum((fu * 16).astype(int), 15)
    assert np.all(np.diff(tile[o]) >= 0)
    _, otex, _ = material
    for f, mode in (("bspline", "stochastic"), ("mitchell", "positivized"), ("linear", "ntap_before")):
        a = ctx.filter_shade(h, u, v, d, f, mode, "ggx", 3, 4, want_picks=True)
        b = ctx.filter_shade(h, u, v, d, f, mode, "ggx", 3, 4, want_picks=True, order=order)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        # and the binned run against the oracle itself (each query keeps its id)
        torch.cuda.synchronize()
        ref = oracle.filter_shade(otex, q, f, mode, "ggx", 3, 4, want_picks=True)
        mism = compare_picks(b[3].cpu().numpy().view(np.uint32), ref, q.n)
        rgb = torch.stack(b[:3], 1).cpu().numpy().astype(np.float64)
        assert_values(rgb, ref.rgb, mism, scale=ref.mag)
    # one sample, no picks: the two-queries-per-thread kernel follows the order too
    a = ctx.filter_shade(h, u, v, d, "bspline", "stochastic", "ggx", 1, 4)
    b = ctx.filter_shade(h, u, v, d, "bspline", "stochastic", "ggx", 1, 4, order=order)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("filter,flags", [("bspline", 4), ("mitchell", 4), ("linear", 4), ("catmull_rom", 6)])
def test_reuse_sampler(ctx, material, filter, flags):
    # flags 4 = sample reuse; 6 = reuse on a shifted lattice
    h, otex, q = material
    _check(ctx, h, otex, q, filter, "stochastic", spp=3, seed=17, flags=flags)


@pytest.mark.parametrize("n", [1, 2, 3, 255, 257, 5999])
def test_one_sample_pairs_ragged(ctx, material, n):
    # at one sample with no flags and no picks a thread takes queries i and i + ceil(n/2);
    # odd counts leave the last thread one query.  Same values as the general path.
    h, _, q = material
    qs = q.subset(np.arange(n))
    with_picks, _ = _run(ctx, h, qs, "bspline", "stochastic", 1, seed=9, picks=True)
    special, _ = _run(ctx, h, qs, "bspline", "stochastic", 1, seed=9, picks=False)
    assert np.array_equal(with_picks, special)


def test_host_entry_point_async(ctx, material):
    # asynchronous host-buffer calls queue behind one another on the copy pipeline; after
    # synchronize() every result equals the one-launch device path bit for bit
    h, _, _ = material
    q = synth.queries_uniform(2_500_001, 24, res=256, lod_range=5.0)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hu, hv, hd = f(q.u), f(q.v), [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)]
    outs = {}
    for filt in ("linear", "bspline", "mitchell"):
        outs[filt] = [torch.empty(q.n, dtype=torch.float32).pin_memory() for _ in range(3)]
        ctx.filter_shade_host_async(h, hu, hv, hd, filt, "stochastic", "ggx", 8, 5, out=outs[filt])
    ctx.synchronize()
    for filt in ("linear", "bspline", "mitchell"):
        dev, _ = _run(ctx, h, q, filt, "stochastic", 8, seed=5, picks=False)
        assert np.array_equal(torch.stack(outs[filt], 1).numpy().astype(np.float64), dev)


def test_host_async_calls_with_changing_layouts(ctx, material):
    # asynchronous host-buffer calls of different sizes stage in differently cut lane regions;
    # queued back to back (with a binning call on the context stream in between), each still
    # equals the one-launch device path once synchronize() returns
    h, _, _ = material
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    sizes = (4_500_001, 70_001, 3_000_017, 4_500_001)
    qs = [synth.queries_uniform(n, 60 + i, res=256, lod_range=5.0) for i, n in enumerate(sizes)]
    ins = [(f(q.u), f(q.v), [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)]) for q in qs]
    outs = [[torch.empty(q.n, dtype=torch.float32).pin_memory() for _ in range(3)] for q in qs]
    bq = synth.queries_uniform(200_000, 70, res=256)
    bu, bv = torch.from_numpy(bq.u).cuda(), torch.from_numpy(bq.v).cuda()
    order = None
    for i, (hu, hv, hd) in enumerate(ins):
        ctx.filter_shade_host_async(h, hu, hv, hd, "mitchell", "stochastic", "ggx", 2, 9, out=outs[i])
        if i == 1:
            order = ctx.bin_queries(bu, bv, tile_log2=5)
    ctx.synchronize()
    for q, o in zip(qs, outs):
        dev, _ = _run(ctx, h, q, "mitchell", "stochastic", 2, seed=9, picks=False)
        assert np.array_equal(torch.stack(o, 1).numpy().astype(np.float64), dev)
    # the order within a bin depends on the scatter's atomics: check that it is a valid order
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(bq.n))
    fu = np.mod(bq.u.astype(np.float64), 1.0)
    fv = np.mod(bq.v.astype(np.float64), 1.0)
    tile = (np.minimum((fv * 32).astype(int), 31) << 5) | np.minimum((fu * 32).astype(int), 31)
    assert np.all(np.diff(tile[o]) >= 0)
