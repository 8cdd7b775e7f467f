"""The gather micro-benchmarks run and give physically ordered results:
loads that touch more cache lines, and shared loads with more bank
conflicts, are not faster; dependent loads that miss L1 and L2 take longer.
"""
import pytest

from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu


def test_gather_micro_ordering():
    ldg = [fdk.fdk_microbench(fdk.MICRO_LDG, d) for d in (1, 4, 32)]
    assert all(v > 0 for v in ldg)
    assert ldg[0] >= ldg[1] * 0.95 and ldg[1] >= ldg[2] * 0.95, ldg
    lds = [fdk.fdk_microbench(fdk.MICRO_LDS, c) for c in (1, 32)]
    assert lds[0] > 4 * lds[1], lds                  # 32-way conflicts serialise
    assert fdk.fdk_microbench(fdk.MICRO_TLD4, 64) > 0
    assert fdk.fdk_microbench(fdk.MICRO_RCP) > 0
    l1, l2 = fdk.fdk_microbench(fdk.MICRO_CHASE, 16), fdk.fdk_microbench(fdk.MICRO_CHASE, 32768)
    assert 0 < l1 < l2, (l1, l2)


def test_micro_rejects_bad_parameters():
    for which, param in ((fdk.MICRO_LDG, 3), (fdk.MICRO_LDS, 0), (fdk.MICRO_TLD4, 1),
                         (fdk.MICRO_CHASE, 0), (99, 1)):
        with pytest.raises(fdk.FdkError):
            fdk.fdk_microbench(which, param)
