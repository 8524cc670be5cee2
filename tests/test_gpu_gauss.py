"""Parity of the CUDA Gaussian filters (FRS over the 4 x 4 window, N-tap over ceil(5 sigma) + 1)
and of filter importance sampling (Sec. 4.2 FIS) with the FP64 oracle, under magnification.

FIS-Gaussian picks: the kernel's logf / sincospif and the oracle's correctly rounded log / cos
agree to an ulp or two, which can move the sample x W + o across a texel edge only when it lies
within about one ulp of x W (3e-5 texels at W = 256) of that edge: such picks are counted and
must stay rare.  Every other pick is bit-exact or sits within 1e-6 of a CDF boundary."""
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
def material(ctx):
    m = synth.material_rgba8(256, 107, octaves=6, base=4)
    return ctx.create_texture(m.albedo_rough, m.normal), oracle.Texture(m.albedo_rough, m.normal)


def _queries(n=3000, seed=31):
    # 4x magnification: the pixel footprint is a quarter texel
    return synth.queries_uniform(n, seed, const_derivs=(1 / 1024, 0.0, 0.0, 1 / 1024))


def _run(ctx, h, q, filter, mode, spp, seed, sampler, sigma, flags=0, picks=True):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = [t(q.dudx), t(q.dvdx), t(q.dudy), t(q.dvdy)] if q.has_derivs() else None
    r, g, b, pk = ctx.filter_shade(h, t(q.u), t(q.v), d, filter, mode, "ggx", spp, seed, flags, want_picks=picks,
                                   sampler=sampler, sigma=sigma)
    torch.cuda.synchronize()
    return (torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64),
            pk.cpu().numpy().view(np.uint32) if pk is not None else None)


@pytest.mark.parametrize("sigma", [0.3, 0.5, 0.8])
@pytest.mark.parametrize("mode,spp", [("stochastic", 4), ("ntap_before", 1), ("ntap_after", 1)])
def test_frs_gaussian_matches_oracle(ctx, material, sigma, mode, spp):
    h, otex = material
    q = _queries()
    rgb, pk = _run(ctx, h, q, "gauss", mode, spp, 4, "frs", sigma)
    ref = oracle.filter_shade(otex, q, "gauss", mode, "ggx", spp, 4, want_picks=True, sampler="frs", sigma=sigma)
    assert_values(rgb, ref.rgb, compare_picks(pk, ref, q.n), scale=ref.mag)


@pytest.mark.parametrize("filter", ["linear", "bspline"])
def test_fis_tent_and_bspline_match_oracle(ctx, material, filter):
    h, otex = material
    q = _queries()
    rgb, pk = _run(ctx, h, q, filter, "stochastic", 4, 6, "fis", 0.0)
    ref = oracle.filter_shade(otex, q, filter, "stochastic", "ggx", 4, 6, want_picks=True, sampler="fis")
    assert_values(rgb, ref.rgb, compare_picks(pk, ref, q.n), scale=ref.mag)


@pytest.mark.parametrize("sigma", [0.3, 0.8])
def test_fis_gaussian_matches_oracle(ctx, material, sigma):
    h, otex = material
    q = _queries()
    spp = 4
    rgb, pk = _run(ctx, h, q, "gauss", "stochastic", spp, 7, "fis", sigma)
    ref = oracle.filter_shade(otex, q, "gauss", "stochastic", "ggx", spp, 7, want_picks=True, sampler="fis",
                              sigma=sigma)
    mism = np.any(pk != ref.picks, axis=(1, 2))
    near = ref.bdist < 1e-4          # samples within a few ulp of x W of a texel edge
    assert not (mism & ~near).any(), f"{(mism & ~near).sum()} FIS pick mismatches away from a texel edge"
    assert mism.sum() <= max(3, int(1e-3 * q.n * spp)), mism.sum()
    assert_values(rgb, ref.rgb, mism, scale=ref.mag)
    # and the N-tap form (the box-convolved Gaussian) on the same queries
    rgb2, _ = _run(ctx, h, q, "gauss", "ntap_after", 1, 7, "fis", sigma, picks=False)
    ref2 = oracle.filter_shade(otex, q, "gauss", "ntap_after", "ggx", 1, 7, sampler="fis", sigma=sigma)
    assert_values(rgb2, ref2.rgb, scale=ref2.mag)


def test_gaussian_specialised_path_equals_general_path(ctx, material):
    h, _ = material
    q = _queries(4000, 33)
    for filter, sampler in (("gauss", "frs"), ("bspline", "fis"), ("gauss", "fis")):
        a, _ = _run(ctx, h, q, filter, "stochastic", 3, 2, sampler, 0.5, picks=True)
        b, _ = _run(ctx, h, q, filter, "stochastic", 3, 2, sampler, 0.5, picks=False)
        assert np.array_equal(a, b), (filter, sampler)


def test_gaussian_invalid_arguments(ctx, material):
    import paper_2407_06107_b300 as stf
    h, _ = material
    q = _queries(64)
    for args, code in (((("mitchell", "stochastic", "fis", 0.5)), 5), ((("gauss", "stochastic", "frs", 0.0)), 1),
                       ((("gauss", "positivized", "frs", 0.5)), 5), ((("gauss", "stochastic", "frs", 9.0)), 1)):
        with pytest.raises(stf.StfError) as e:
            _run(ctx, h, q, args[0], args[1], 4, 1, args[2], args[3], picks=False)
        assert e.value.status == code
    with pytest.raises(stf.StfError) as e:
        _run(ctx, h, q, "gauss", "stochastic", 4, 1, "frs", 0.5, flags=oracle.FLAG_LATTICE, picks=False)
    assert e.value.status == 5
