"""The integer pipe probe (measurement, not the method): it runs every op
class and reports rates inside what the hardware can issue."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probe_rates_are_physical():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield as ms
    rows = ms.probe_int_pipes(torch.cuda.current_device())
    assert [r["class"] for r in rows] == list(ms.PIPE_CLASSES)
    by = {r["class"]: r for r in rows}
    for r in rows:
        # 4 schedulers x 32 lanes issue at most 128 lane operations per SM per clock
        assert 0 < r["lanes_per_sm_clk"] <= 128.5, r
        assert r["sm_mhz"] > 300 and r["tops"] > 0
    assert by["mulhi"]["lanes_per_sm_clk"] <= by["mad"]["lanes_per_sm_clk"] * 1.05
    # xor, funnel shifts and byte permutes share a 16-lane-per-scheduler pipe
    for c in ("xor", "shf", "prmt", "xor+shf"):
        assert by[c]["lanes_per_sm_clk"] <= 64.5, by[c]
    assert ms.lib.ms_probe_int_pipes(0, None, 0) == ms.MS_EINVAL
    assert ms.lib.ms_probe_int_pipes(-1, None, 10) == ms.MS_EINVAL
