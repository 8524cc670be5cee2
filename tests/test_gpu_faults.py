"""Failure handling without a GPU fault: host-injected allocation / launch failures and a
device wait that is made to run out (no MMA is issued, so nothing is in flight)."""
import os

import numpy as np
import pytest

import stf_synth as synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture
def stf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_06107_b300 as m
    yield m
    os.environ.pop("STF_FAULT", None)


def _ctx(stf, fault):
    os.environ["STF_FAULT"] = fault
    try:
        return stf.Context(0)
    finally:
        os.environ.pop("STF_FAULT", None)


def test_injected_allocation_failure(stf):
    # the context itself allocates its status word, so creation reports the failure
    os.environ["STF_FAULT"] = "alloc"
    with pytest.raises(stf.StfError) as e:
        stf.Context(0)
    assert e.value.status == 3
    os.environ.pop("STF_FAULT")


def test_injected_launch_failure_leaves_context_usable(stf):
    ctx = _ctx(stf, "launch")
    tex = ctx.create_texture([synth.texture_rgba32f(16, 1)])
    u = torch.rand(64, device="cuda")
    with pytest.raises(stf.StfError) as e:
        ctx.filter_shade(tex, u, u, None, "bspline", "stochastic", "ggx", 1, 1)
    assert e.value.status == 4 and "STF_FAULT" in str(e.value)
    ctx.close()
    ok = stf.Context(0)                      # a fresh context works normally
    t2 = ok.create_texture([synth.texture_rgba32f(16, 1)])
    r, g, b, _ = ok.filter_shade(t2, u, u, None, "bspline", "stochastic", "ggx", 1, 1)
    assert torch.isfinite(r).all()
    ok.close()


def test_decode_wait_times_out_and_reports(stf):
    ctx = _ctx(stf, "mma_timeout")
    lat, mlp = synth.ntc_init((8, 4, 2, 1), 3)
    net = ctx.neural_create(16, lat, mlp, None)
    ix = torch.arange(16, dtype=torch.int32, device="cuda")
    ctx.neural_decode(net, ix, ix)
    assert ctx.device_status() & stf.DEV_TIMEOUT
    ctx.close()
    # the GPU and a normal context are fine afterwards
    ok = stf.Context(0)
    net = ok.neural_create(16, lat, mlp, None)
    y = ok.neural_decode(net, ix, ix)
    assert torch.isfinite(y).all() and ok.device_status() == 0
    ok.close()


def test_stochastic_decode_pipeline_times_out_and_reports(stf):
    # the 1-tap neural filter's pipelined kernel: with no MMA issued, its epilogue's bounded
    # wait runs out, every role leaves its loop, and the status reports the timeout
    ctx = _ctx(stf, "mma_timeout")
    lat, mlp = synth.ntc_init((8, 4, 2, 1), 3)
    net = ctx.neural_create(16, lat, mlp, None)
    u = torch.rand(500, device="cuda")
    ctx.neural_filter_shade(net, u, u, None, "bspline", "stochastic", "ggx", 4, 1)
    assert ctx.device_status() & stf.DEV_TIMEOUT
    ctx.close()
    ok = stf.Context(0)
    net = ok.neural_create(16, lat, mlp, None)
    r, g, b = ok.neural_filter_shade(net, u, u, None, "bspline", "stochastic", "ggx", 4, 1)
    assert torch.isfinite(r).all() and ok.device_status() == 0
    ok.close()
