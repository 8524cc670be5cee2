"""The no-allocation host entry point matches the regular one.

stf_filter_shade_host_noalloc exists for callers that cannot allocate device memory
while they shade (a frame loop with a fixed memory budget, a plug-in inside an
application that owns all allocations).  It stages everything in one fixed device array
of the library, so these checks run it twice in a row -- the second call reuses the
array with different sizes, filter and mode -- and compare each result with
stf_filter_shade_host, the allocating entry point, within the tolerance of the other
parity tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import stf_synth as synth
from gpu_util import assert_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_06107_b300 as stf
    ctx = stf.Context(0)
    m = synth.material_rgba8(128, 61, octaves=5, base=4)
    tex = ctx.create_texture(m.albedo_rough, m.normal)
    yield stf, ctx, tex
    ctx.close()


def _pinned(q):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return f(q.u), f(q.v), [f(q.dudx), f(q.dvdx), f(q.dudy), f(q.dvdy)]


def _compare(ctx, tex, q, filter, mode, spp, seed, id_base):
    u, v, d = _pinned(q)
    a = ctx.filter_shade_host_noalloc(tex, u, v, d, filter, mode, "ggx", spp, seed, id_base=id_base)
    b = ctx.filter_shade_host(tex, u, v, d, filter, mode, "ggx", spp, seed, id_base=id_base)
    got = np.stack(a, 1).astype(np.float64)
    ref = np.stack(b[:3], 1).astype(np.float64)
    assert np.all(np.isfinite(got))
    assert_values(got, ref)


def test_two_calls_in_a_row_match_allocating_entry_point(setup):
    _, ctx, tex = setup
    q1 = synth.queries_uniform(50000, 71, res=128, lod_range=6.0)
    _compare(ctx, tex, q1, "mitchell", "stochastic", 4, 3, 0)
    # second call: fewer queries, other filter and mode -- the array still holds the
    # first call's larger contents, which must not leak into this result
    q2 = synth.queries_uniform(30001, 72, res=128, lod_range=6.0)
    _compare(ctx, tex, q2, "catmull_rom", "positivized", 2, 9, 123)


def test_rejects_batches_beyond_the_fixed_array(setup):
    stf, ctx, tex = setup
    n = (1 << 18) + 1
    z = torch.zeros(n, dtype=torch.float32)
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade_host_noalloc(tex, z, z, None, "bspline", "stochastic", "ggx", 1, 1)
    assert e.value.status == 1 and "262144" in str(e.value)


def test_status_word_is_cleared_per_call(setup):
    stf, ctx, tex = setup
    q = synth.queries_uniform(1000, 73, res=128, lod_range=4.0)
    q.u[10] = np.nan
    u, v, d = _pinned(q)
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade_host_noalloc(tex, u, v, d, "linear", "stochastic", "ggx", 1, 1)
    assert e.value.status == 6
    q2 = synth.queries_uniform(1000, 74, res=128, lod_range=4.0)
    _compare(ctx, tex, q2, "linear", "stochastic", 1, 1, 0)


def test_lod0_and_ewa_match_allocating_entry_point(setup):
    # the same filters and flags as stf_filter_shade_host: EWA reads the context's weight
    # table (allocated with the context, so the call still allocates nothing)
    _, ctx, tex = setup
    q = synth.queries_aniso(20000, 75, res=128, lod_range=3.0, max_aniso=16.0)
    u, v, d = _pinned(q)
    for filter, mode, flags in (("ewa", "stochastic", 0), ("ewa", "ntap_before", 8), ("bspline", "stochastic", 8)):
        a = ctx.filter_shade_host_noalloc(tex, u, v, d, filter, mode, "ggx", 2, 5, flags)
        b = ctx.filter_shade_host(tex, u, v, d, filter, mode, "ggx", 2, 5, flags)
        assert_values(np.stack(a, 1).astype(np.float64), np.stack(b[:3], 1).astype(np.float64))
