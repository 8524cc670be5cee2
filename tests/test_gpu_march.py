"""Parity of the CUDA volume march (through the C ABI) with the FP64 oracle."""
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


@pytest.fixture(scope="module")
def small(ctx):
    vol = synth.volume_cloud(32, 103, zero_frac=0.9, octaves=4, base=2)
    return ctx.create_volume(vol, 20.0), vol


W, H = 40, 24


@pytest.mark.parametrize("filter", ["linear", "bspline"])
@pytest.mark.parametrize("mode", ["ntap_before", "ntap_after", "stochastic"])
def test_small_volume(ctx, small, filter, mode):
    h, vol = small
    cam = synth.camera_pinhole(W, H).as_array()
    T, pk = ctx.march_volume(h, cam, W, H, 128, filter, mode, spp=2, seed=3, want_picks=True)
    torch.cuda.synchronize()
    ref = oracle.march(vol, 20.0, cam, W, H, 128, filter, mode, spp=2, seed=3, want_picks=True)
    mism = None
    if mode == "stochastic":
        mism = compare_picks(pk.cpu().numpy().view(np.uint32), ref, W * H)
    else:
        assert np.all(pk.cpu().numpy().view(np.uint32) == oracle.NO_PICK)
    assert_values(T.cpu().numpy(), ref.T, mism)


@pytest.mark.parametrize("flags", [0, oracle.FLAG_LATTICE])
@pytest.mark.parametrize("filter,steps", [("bspline", 97), ("linear", 64)])
def test_specialised_path_equals_general_path(ctx, small, filter, steps, flags):
    # without pick output (and with no flag, or the lattice flag alone) the stochastic march
    # runs its specialised paired-step instantiation (odd step counts end with one unpaired
    # step); the densities are summed in exact fixed point, so T equals the general path's
    # bit for bit
    h, _ = small
    cam = synth.camera_pinhole(W, H).as_array()
    T1, _ = ctx.march_volume(h, cam, W, H, steps, filter, "stochastic", spp=3, seed=4, flags=flags, want_picks=True)
    T2, _ = ctx.march_volume(h, cam, W, H, steps, filter, "stochastic", spp=3, seed=4, flags=flags)
    assert torch.equal(T1, T2)


@pytest.mark.parametrize("scale,steps", [(16.0, 97), (1.0, 97), (1.9, 128), (2.0, 128)])
@pytest.mark.parametrize("filter", ["linear", "bspline"])
def test_density_sum_widths_and_odd_shapes(ctx, filter, scale, steps):
    # The 1-tap march sums the picked densities as exact d * 2^24 fixed point, in 32 bits when
    # steps x (largest density) < 256 and in 64 bits otherwise (scale 16 and 2 x 128 steps);
    # either way it equals the general path bit for bit and the oracle within tolerance.  The
    # volume is not a cube and its x size is no multiple of 8, so the bordered copy the 1-tap
    # march reads has a padded row pitch.
    base = synth.volume_cloud(24, 107, zero_frac=0.7, octaves=3, base=2)[:, :19, :13]
    vol = np.ascontiguousarray((base.astype(np.float32) * scale).astype(np.float16))
    h = ctx.create_volume(vol, 1.5)
    cam = synth.camera_pinhole(W, H).as_array()
    T1, pk = ctx.march_volume(h, cam, W, H, steps, filter, "stochastic", spp=2, seed=6, want_picks=True)
    T2, _ = ctx.march_volume(h, cam, W, H, steps, filter, "stochastic", spp=2, seed=6)
    torch.cuda.synchronize()
    assert torch.equal(T1, T2)
    ref = oracle.march(vol, 1.5, cam, W, H, steps, filter, "stochastic", spp=2, seed=6, want_picks=True)
    mism = compare_picks(pk.cpu().numpy().view(np.uint32), ref, W * H)
    assert_values(T1.cpu().numpy(), ref.T, mism)
    ctx.destroy_volume(h)


def test_stratified_and_pixel_ranges(ctx, small):
    h, vol = small
    cam = synth.camera_pinhole(W, H).as_array()
    for begin, cnt in ((0, 1), (17, 333), (W * H - 5, 5)):
        T, _ = ctx.march_volume(h, cam, W, H, 64, "bspline", "stochastic", spp=4, seed=9, flags=1,
                                pix_begin=begin, pix_count=cnt)
        ref = oracle.march(vol, 20.0, cam, W, H, 64, "bspline", "stochastic", spp=4, seed=9, flags=1,
                           pix_begin=begin, pix_count=cnt)
        near = ref.bdist < 1e-6
        assert_values(T.cpu().numpy(), ref.T, near)
    T, _ = ctx.march_volume(h, cam, W, H, 64, "bspline", "stochastic", pix_begin=3, pix_count=0)
    assert T.numel() == 0


def test_invalid_arguments(ctx, small):
    import paper_2407_06107_b300 as stf
    h, _ = small
    cam = synth.camera_pinhole(W, H).as_array()
    for kw, code in ((dict(filter="mitchell"), 5), (dict(mode="positivized"), 5), (dict(pix_begin=W * H), 1)):
        args = dict(filter="bspline", mode="stochastic", pix_begin=0)
        args.update(kw)
        with pytest.raises(stf.StfError) as e:
            ctx.march_volume(h, cam, W, H, 16, args["filter"], args["mode"], pix_begin=args["pix_begin"],
                             pix_count=1)
        assert e.value.status == code


@pytest.mark.parametrize("filter,mode,spp,flags", [("bspline", "stochastic", 1, 0), ("bspline", "ntap_before", 1, 0),
                                                   ("linear", "stochastic", 1, 0), ("bspline", "ntap_before", 8, 0),
                                                   ("bspline", "stochastic", 8, 0),
                                                   ("bspline", "stochastic", 8, oracle.FLAG_LATTICE),
                                                   ("linear", "ntap_before", 8, 0)])
def test_full_size_sampled(ctx, filter, mode, spp, flags):
    # 512^3 FP16 cloud at 1920x1080, 128 steps, in the launch configurations the benchmark
    # times (8 spp: the tricubic 64-tap and trilinear 8-tap comparators, the 1-tap estimator
    # with independent and lattice uniforms): sampled pixels re-evaluated by the oracle
    vol = _full_volume()
    h = _full_handle(ctx, vol)
    cam = synth.camera_pinhole(1920, 1080).as_array()
    seed = 1 if spp == 1 else 5
    T, _ = ctx.march_volume(h, cam, 1920, 1080, 128, filter, mode, spp=spp, seed=seed, flags=flags)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(5).choice(1920 * 1080, 400, replace=False))
    got = T[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.march(vol, 20.0, cam, 1920, 1080, 128, filter, mode, spp=spp, seed=seed, flags=flags,
                       pix_ids=idx)
    near = ref.bdist < 1e-6
    assert near.sum() <= 2 * spp
    assert_values(got, ref.T, near)


_FULL = {}


def _full_volume():
    if "v" not in _FULL:
        _FULL["v"] = synth.volume_cloud(512, 103)
    return _FULL["v"]


def _full_handle(ctx, vol):
    if "h" not in _FULL:
        _FULL["h"] = ctx.create_volume(vol, 20.0)
    return _FULL["h"]


@pytest.mark.parametrize("filter", ["linear", "bspline"])
def test_lattice_sampler(ctx, small, filter):
    h, vol = small
    cam = synth.camera_pinhole(W, H).as_array()
    T, pk = ctx.march_volume(h, cam, W, H, 128, filter, "stochastic", spp=5, seed=8, flags=oracle.FLAG_LATTICE,
                             want_picks=True)
    ref = oracle.march(vol, 20.0, cam, W, H, 128, filter, "stochastic", spp=5, seed=8, flags=oracle.FLAG_LATTICE,
                       want_picks=True)
    mism = compare_picks(pk.cpu().numpy().view(np.uint32), ref, W * H)
    assert_values(T.cpu().numpy(), ref.T, mism)


@pytest.mark.parametrize("filter", ["linear", "bspline"])
def test_reuse_sampler(ctx, small, filter):
    h, vol = small
    cam = synth.camera_pinhole(W, H).as_array()
    T, pk = ctx.march_volume(h, cam, W, H, 96, filter, "stochastic", spp=3, seed=12, flags=oracle.FLAG_REUSE,
                             want_picks=True)
    ref = oracle.march(vol, 20.0, cam, W, H, 96, filter, "stochastic", spp=3, seed=12, flags=oracle.FLAG_REUSE,
                       want_picks=True)
    mism = compare_picks(pk.cpu().numpy().view(np.uint32), ref, W * H)
    assert_values(T.cpu().numpy(), ref.T, mism)


@pytest.mark.parametrize("mode", ["stochastic", "ntap_after"])
def test_tiled_and_row_order_agree(ctx, small, mode):
    # a whole frame runs these modes with 8 x 4 pixel tiles per warp; ranges that are not whole
    # 4-row bands run in row order.  Per pixel the work is the same, so the results agree bit
    # for bit.
    h, _ = small
    cam = synth.camera_pinhole(W, H).as_array()
    full, pk_full = ctx.march_volume(h, cam, W, H, 64, "bspline", mode, spp=2, seed=21, want_picks=True)
    a, pk_a = ctx.march_volume(h, cam, W, H, 64, "bspline", mode, spp=2, seed=21, pix_begin=0, pix_count=3 * W,
                               want_picks=True)
    b, pk_b = ctx.march_volume(h, cam, W, H, 64, "bspline", mode, spp=2, seed=21, pix_begin=3 * W,
                               pix_count=(H - 3) * W, want_picks=True)
    torch.cuda.synchronize()
    rows = torch.cat([a, b]).cpu().numpy()
    assert np.array_equal(full.cpu().numpy(), rows)
    assert np.array_equal(pk_full.cpu().numpy(), torch.cat([pk_a, pk_b]).cpu().numpy())


@pytest.mark.parametrize("mode", ["ntap_before", "ntap_after"])
@pytest.mark.parametrize("w,h", [(160, 96), (40, 24), (37, 23)])
def test_staged_tricubic_equals_unstaged(ctx, small, mode, w, h):
    # the tricubic N-tap march without flags stages each warp's voxel box in shared memory by
    # TMA (8 x 4 pixel tiles when the range allows, row order otherwise; steps whose windows do
    # not fit the box or need clamping read global memory).  With pick output the unstaged
    # kernel runs.  Same voxels, same order: identical results, and both match the oracle.
    hnd, vol = small
    cam = synth.camera_pinhole(w, h).as_array()
    staged, _ = ctx.march_volume(hnd, cam, w, h, 96, "bspline", mode, spp=2, seed=7)
    plain, pk = ctx.march_volume(hnd, cam, w, h, 96, "bspline", mode, spp=2, seed=7, want_picks=True)
    torch.cuda.synchronize()
    assert torch.equal(staged, plain)
    ref = oracle.march(vol, 20.0, cam, w, h, 96, "bspline", mode, spp=2, seed=7)
    assert_values(staged.cpu().numpy(), ref.T)
    # a sub-range of whole 4-row bands and one that is not
    for begin, cnt in ((4 * w, 8 * w), (5, 3 * w + 1)):
        part, _ = ctx.march_volume(hnd, cam, w, h, 96, "bspline", mode, spp=2, seed=7, pix_begin=begin, pix_count=cnt)
        torch.cuda.synchronize()
        assert torch.equal(part, plain[begin:begin + cnt])
