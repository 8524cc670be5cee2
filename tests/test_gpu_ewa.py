"""Parity of the CUDA EWA path (supplement "Stochastic EWA") and of the finest-level flag
with the FP64 oracle, on anisotropic footprints."""
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
    m = synth.material_rgba8(256, 104, octaves=6, base=4)
    return ctx.create_texture(m.albedo_rough, m.normal), oracle.Texture(m.albedo_rough, m.normal)


def _run(ctx, h, q, filter, mode, spp, seed=1, flags=0, picks=True):
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = [t(q.dudx), t(q.dvdx), t(q.dudy), t(q.dvdy)] if q.has_derivs() else None
    r, g, b, pk = ctx.filter_shade(h, t(q.u), t(q.v), d, filter, mode, "ggx", spp, seed, flags, want_picks=picks)
    torch.cuda.synchronize()
    rgb = torch.stack([r, g, b], 1).cpu().numpy().astype(np.float64)
    return rgb, (pk.cpu().numpy().view(np.uint32) if pk is not None else None)


@pytest.mark.parametrize("mode,spp", [("stochastic", 4), ("ntap_before", 1), ("ntap_after", 1)])
@pytest.mark.parametrize("lod_range,max_aniso", [(4.0, 64.0), (1.0, 8.0)])
def test_ewa_matches_oracle(ctx, material, mode, spp, lod_range, max_aniso):
    h, otex = material
    q = synth.queries_aniso(3000, 41, res=256, lod_range=lod_range, max_aniso=max_aniso)
    rgb, pk = _run(ctx, h, q, "ewa", mode, spp, seed=3)
    ref = oracle.filter_shade(otex, q, "ewa", mode, "ggx", spp, 3, want_picks=True)
    mism = compare_picks(pk, ref, q.n)
    assert_values(rgb, ref.rgb, mism, scale=ref.mag)


def test_ewa_without_derivatives_and_lod0(ctx, material):
    # no derivatives: the unit reconstruction circle at level 0; LOD0: the derivative
    # ellipse at level 0 (boxes up to a few hundred texels)
    h, otex = material
    q = synth.queries_uniform(2000, 5)
    for mode in ("stochastic", "ntap_before"):
        rgb, pk = _run(ctx, h, q, "ewa", mode, 2, seed=8)
        ref = oracle.filter_shade(otex, q, "ewa", mode, "ggx", 2, 8, want_picks=True)
        assert_values(rgb, ref.rgb, compare_picks(pk, ref, q.n), scale=ref.mag)
    qa = synth.queries_aniso(800, 6, res=256, lod_range=2.0, max_aniso=32.0)
    for mode in ("stochastic", "ntap_after"):
        rgb, pk = _run(ctx, h, qa, "ewa", mode, 2, seed=9, flags=oracle.FLAG_LOD0)
        ref = oracle.filter_shade(otex, qa, "ewa", mode, "ggx", 2, 9, flags=oracle.FLAG_LOD0, want_picks=True)
        assert_values(rgb, ref.rgb, compare_picks(pk, ref, qa.n), scale=ref.mag)


@pytest.mark.parametrize("filter,mode", [("bspline", "stochastic"), ("linear", "ntap_after"),
                                         ("mitchell", "positivized")])
def test_lod0_flag_matches_oracle(ctx, material, filter, mode):
    h, otex = material
    q = synth.queries_aniso(3000, 12, res=256, lod_range=3.0, max_aniso=16.0)
    rgb, pk = _run(ctx, h, q, filter, mode, 4, seed=2, flags=oracle.FLAG_LOD0)
    ref = oracle.filter_shade(otex, q, filter, mode, "ggx", 4, 2, flags=oracle.FLAG_LOD0, want_picks=True)
    mism = compare_picks(pk, ref, q.n)
    assert_values(rgb, ref.rgb, mism, scale=ref.mag)
    if mode != "ntap_after":
        assert np.all((pk[..., 0] >> 28) == 0)


def test_ewa_specialised_path_equals_general_path(ctx, material):
    h, _ = material
    q = synth.queries_aniso(4000, 13, res=256, lod_range=4.0)
    a, _ = _run(ctx, h, q, "ewa", "stochastic", 3, seed=5, picks=True)
    b, _ = _run(ctx, h, q, "ewa", "stochastic", 3, seed=5, picks=False)
    assert np.array_equal(a, b)


def test_ewa_invalid_arguments(ctx, material):
    import paper_2407_06107_b300 as stf
    h, _ = material
    q = synth.queries_aniso(64, 1, res=256)
    for kw, code in ((dict(mode="positivized"), 5), (dict(flags=oracle.FLAG_LATTICE), 5),
                     (dict(flags=oracle.FLAG_STRATIFIED), 5)):
        args = dict(mode="stochastic", flags=0)
        args.update(kw)
        with pytest.raises(stf.StfError) as e:
            _run(ctx, h, q, "ewa", args["mode"], 4, flags=args["flags"], picks=False)
        assert e.value.status == code
