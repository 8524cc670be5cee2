"""Parity of the CUDA path on DCT-compressed textures (supplement "Texture compression") with
the FP64 oracle, which decodes the same blocks with its own inverse DCT.

Tolerance: the kernel decodes in FP32 (cospif, then five FMAs per channel), within ~5e-7
absolute of the FP64 decode; the GGX shade's sensitivity to the normal is at most 2/alpha = 40
(alpha >= 0.05), so shaded terms agree within 40 * 5e-7 = 2e-5 relative, written as
3e-5 * sum|terms| + 1e-7.  Picks are decided before any decode and stay bit-exact."""
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


@pytest.fixture(scope="module")
def dct_tex(ctx):
    m = synth.material_rgba8(256, 106, octaves=6, base=4)
    blocks = synth.dct_compress(m)
    sizes = [lv.shape[:2] for lv in m.albedo_rough]
    return ctx.create_texture_dct(blocks, 256, 256), oracle.Texture(sizes, dct=blocks)


def _run(ctx, h, q, filter, mode, spp, seed=1, flags=0, picks=True):
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = [t(q.dudx), t(q.dvdx), t(q.dudy), t(q.dvdy)] if q.has_derivs() else None
    r, g, b, pk = ctx.filter_shade(h, t(q.u), t(q.v), d, filter, mode, "ggx", spp, seed, flags, want_picks=picks)
    torch.cuda.synchronize()
    rgb = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    return rgb, (pk.cpu().numpy().view(np.uint32) if pk is not None else None)


@pytest.mark.parametrize("filter,mode,spp", [("linear", "stochastic", 4), ("linear", "stochastic", 1),
                                             ("mitchell", "stochastic", 1), ("linear", "ntap_before", 1),
                                             ("linear", "ntap_after", 1), ("bspline", "stochastic", 3),
                                             ("mitchell", "positivized", 2), ("ewa", "stochastic", 2),
                                             ("ewa", "ntap_before", 1)])
def test_dct_matches_oracle(ctx, dct_tex, filter, mode, spp):
    h, otex = dct_tex
    q = synth.queries_uniform(3000, 17, res=256, lod_range=6.0)
    rgb, pk = _run(ctx, h, q, filter, mode, spp, seed=5)
    ref = oracle.filter_shade(otex, q, filter, mode, "ggx", spp, 5, want_picks=True)
    mism = compare_picks(pk, ref, q.n)
    assert_values(rgb, ref.rgb, mism, rel=REL_DCT, scale=ref.mag)
    # the specialised (no flags, no picks) DCT kernels return the same values
    rgb2, _ = _run(ctx, h, q, filter, mode, spp, seed=5, picks=False)
    assert_values(rgb2, ref.rgb, mism, rel=REL_DCT, scale=ref.mag)


def test_dct_without_derivatives_and_lattice(ctx, dct_tex):
    h, otex = dct_tex
    q = synth.queries_uniform(2000, 18)
    rgb, pk = _run(ctx, h, q, "bspline", "stochastic", 4, seed=6, flags=oracle.FLAG_LATTICE)
    ref = oracle.filter_shade(otex, q, "bspline", "stochastic", "ggx", 4, 6, flags=oracle.FLAG_LATTICE,
                              want_picks=True)
    assert_values(rgb, ref.rgb, compare_picks(pk, ref, q.n), rel=REL_DCT, scale=ref.mag)


def test_dct_rejected_where_unsupported(ctx, dct_tex):
    import paper_2407_06107_b300 as stf
    h, _ = dct_tex
    with pytest.raises(stf.StfError) as e:
        ctx.create_texture_table([h])
    assert e.value.status == 5
