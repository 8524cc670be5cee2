"""The gather roofline's measured denominator (random 32-byte sector reads at L2)."""
import pytest

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


def test_sector_rate_is_plausible(ctx):
    # an L2-resident buffer must read faster than one that spills to DRAM, and both rates must
    # lie between 1e10 sectors/s and the issue limit (148 SMs x 4 schedulers x 32 lanes x 2.1 GHz)
    l2 = ctx.measure_sector_rate(32 << 20)
    dram = ctx.measure_sector_rate(1 << 30)
    assert 1e10 < dram < l2 < 148 * 4 * 32 * 2.1e9, (l2, dram)


def test_sector_rate_rejects_bad_sizes(ctx):
    import paper_2407_06107_b300 as stf
    for n in (0, 3 << 20, 1 << 19, 1 << 31):
        with pytest.raises(stf.StfError) as e:
            ctx.measure_sector_rate(n)
        assert e.value.status == 1
