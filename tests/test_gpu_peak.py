"""The integer-pipe probe (ga_int_peak) through the C ABI: every kind runs and reports a rate
that no GPU of this size can exceed -- at most one warp-instruction per clock on each of the
four sub-partitions of every SM, at the highest SM clock -- and bad arguments are refused."""
import pytest

pytestmark = pytest.mark.gpu


def test_int_peak_kinds_within_issue_limit():
    import torch
    from gpu_util import gpu_run  # noqa: F401  (builds the library)
    from paper_2405_03605_gb300 import ga
    from paper_2405_03605_gb300.workloads import RunShape
    gpu_run(RunShape(rows=1, cols=1)).close()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_limit = sms * 4 * 32 * 2.2e9  # thread-operations per second at 2.2 GHz
    for kind in (ga.PEAK_LOP3, ga.PEAK_IMAD, ga.PEAK_MIX):
        rate, sec = ga.int_peak(kind, iters=256)
        assert 0 < rate <= issue_limit, (kind, rate, issue_limit)
        assert sec > 0
    with pytest.raises(ga.GaError) as e:
        ga.int_peak(3)
    assert e.value.code == -1
    with pytest.raises(ga.GaError) as e:
        ga.int_peak(ga.PEAK_LOP3, iters=0)
    assert e.value.code == -1
