"""The FMA-pipe throughput measurement (the arithmetic rooflines' denominators)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_7327_gb300 import smc as S
    return S


def test_fma_throughput_is_measured_for_each_pipe(smc):
    props = torch.cuda.get_device_properties(0)
    res = {}
    for kind, iters in ((0, 20_000), (1, 400_000), (2, 200_000)):
        fl, ms, sms = smc.smc_fma_throughput(kind, iters)
        assert sms == props.multi_processor_count
        assert ms > 0 and fl > 0
        res[kind] = fl
    # at least one FMA per SM and clock, no more than 1024 lanes' worth
    clk = 2.5e9
    for fl in res.values():
        assert fl < props.multi_processor_count * 1024 * 2 * clk
    fl1, _, _ = smc.smc_fma_throughput(3, 20_000)
    assert 0 < fl1 <= res[0] * 1.05
    with pytest.raises(smc.SmcError):
        smc.smc_fma_throughput(4, 10)
    with pytest.raises(smc.SmcError):
        smc.smc_fma_throughput(0, 0)
