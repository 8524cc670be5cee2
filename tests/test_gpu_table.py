"""Bindless texture table (many textures of uneven sizes, one persistent launch) against
the FP64 oracle, query by query with each query's own Philox id."""
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


def _check_table(ctx, texs, n, filter, mode, spp, seed, sample=None, qseed=3):
    handles = [ctx.create_texture([t]) for t in texs]
    table = ctx.create_texture_table(handles)
    q = synth.queries_uniform(n, qseed)
    rng = np.random.default_rng(qseed + 100)
    tid = rng.integers(0, len(texs), n).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    r, g, b, pk = ctx.filter_shade_table(table, t(q.u), t(q.v), t(tid), None, filter, mode, "ggx", spp, seed,
                                         want_picks=sample is None)
    torch.cuda.synchronize()
    rgb = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    pk = pk.cpu().numpy().view(np.uint32) if pk is not None else None
    idx_all = np.arange(n) if sample is None else np.sort(np.random.default_rng(7).choice(n, sample, replace=False))
    for k in range(len(texs)):
        idx = idx_all[tid[idx_all] == k]
        if idx.size == 0:
            continue
        ref = oracle.filter_shade(oracle.Texture([texs[k]]), q.subset(idx), filter, mode, "ggx", spp, seed,
                                  want_picks=sample is None, ids=idx)
        mism = compare_picks(pk[idx], ref, idx.size) if pk is not None else (ref.bdist < 1e-6)
        assert_values(rgb[idx], ref.rgb, mism, scale=ref.mag)
    ctx.destroy_texture_table(table)
    for h in handles:
        ctx.destroy_texture(h)


@pytest.mark.parametrize("mode", ["stochastic", "positivized"])
def test_mitchell_table(ctx, mode):
    texs = synth.texture_table_rgba8(24, 5, 300, seed=105, fbm_below=300)
    _check_table(ctx, texs, 20000, "mitchell", mode, 4, 1)


def test_other_filters_table(ctx):
    texs = synth.texture_table_rgba8(10, 3, 120, seed=106, fbm_below=200)
    for f, mode in (("bspline", "stochastic"), ("linear", "ntap_before"), ("catmull_rom", "ntap_after")):
        _check_table(ctx, texs, 5000, f, mode, 2, 5)


def test_empty_batch_is_noop(ctx):
    texs = synth.texture_table_rgba8(3, 2, 64, seed=107, fbm_below=64)
    handles = [ctx.create_texture([t]) for t in texs]
    table = ctx.create_texture_table(handles)
    e = torch.empty(0, device="cuda")
    tid = torch.empty(0, dtype=torch.int32, device="cuda")
    r, _, _, _ = ctx.filter_shade_table(table, e, e, tid, None, "mitchell", "stochastic", "ggx", 4, 1)
    assert r.numel() == 0
    ctx.destroy_texture_table(table)
    for h in handles:
        ctx.destroy_texture(h)


def test_large_table_sampled(ctx):
    # 256 textures, sides 64..1024 log-uniform, 4M mixed queries, Mitchell at 4 spp
    texs = synth.texture_table_rgba8(256, 64, 1024, seed=107)
    _check_table(ctx, texs, 1 << 22, "mitchell", "stochastic", 4, 1, sample=3000)


@pytest.mark.parametrize("flags", [0, oracle.FLAG_LATTICE])
def test_specialised_path_equals_general_path(ctx, flags):
    # without pick output (no flag, or the lattice flag alone) the table launch runs a
    # specialised instantiation with the same arithmetic: identical results
    texs = synth.texture_table_rgba8(12, 5, 200, seed=109, fbm_below=200)
    handles = [ctx.create_texture([t]) for t in texs]
    table = ctx.create_texture_table(handles)
    q = synth.queries_uniform(30000, 4)
    tid = np.random.default_rng(11).integers(0, len(texs), q.n).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    outs = []
    for picks in (True, False):
        r, g, b, _ = ctx.filter_shade_table(table, t(q.u), t(q.v), t(tid), None, "mitchell", "stochastic", "ggx", 3, 2,
                                            flags=flags, want_picks=picks)
        outs.append(torch.stack([r, g, b], 1).cpu())
    assert torch.equal(outs[0], outs[1])
    ctx.destroy_texture_table(table)
    for h in handles:
        ctx.destroy_texture(h)


def test_bad_texture_id_and_lifetime(ctx):
    import paper_2407_06107_b300 as stf
    texs = synth.texture_table_rgba8(3, 8, 16, seed=108, fbm_below=32)
    hs = [ctx.create_texture([t]) for t in texs]
    table = ctx.create_texture_table(hs)
    with pytest.raises(stf.StfError):
        ctx.destroy_texture(hs[0])                    # still referenced by the table
    u = torch.rand(100, device="cuda")
    tid = torch.zeros(100, dtype=torch.int32, device="cuda")
    tid[7] = 3                                       # out of range
    ctx.device_status()
    r, g, b, _ = ctx.filter_shade_table(table, u, u, tid, None, "mitchell", "stochastic", "ggx", 2, 1)
    assert ctx.device_status() & stf.DEV_BAD_INDEX
    assert float(r[7]) == 0.0 and float(r[6]) != 0.0
    ctx.destroy_texture_table(table)
    for h in hs:
        ctx.destroy_texture(h)


def test_binned_table_identical(ctx):
    texs = synth.texture_table_rgba8(12, 20, 200, seed=109, fbm_below=300)
    hs = [ctx.create_texture([t]) for t in texs]
    table = ctx.create_texture_table(hs)
    n = 30000
    rng = np.random.default_rng(3)
    u = torch.rand(n, device="cuda")
    v = torch.rand(n, device="cuda")
    tid = torch.from_numpy(rng.integers(0, 12, n).astype(np.int32)).cuda()
    order = ctx.bin_queries(u, v, tid, ntex=12, tile_log2=3)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(n))
    assert np.all(np.diff(tid.cpu().numpy()[o]) >= 0)          # texture id is the major key
    a = ctx.filter_shade_table(table, u, v, tid, None, "mitchell", "stochastic", "ggx", 4, 1)
    b = ctx.filter_shade_table(table, u, v, tid, None, "mitchell", "stochastic", "ggx", 4, 1, order=order)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    ctx.destroy_texture_table(table)
    for hh in hs:
        ctx.destroy_texture(hh)
