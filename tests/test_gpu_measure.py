"""The random-load ceiling (include/cc_measure.h) on the GPU: a finite,
positive rate within what the hardware can serve, and an L2-resident array
served at least as fast as one several times larger than L2."""
import pytest

pytestmark = pytest.mark.gpu


def test_random_load_rate():
    import paper_2507_03695_gb300 as cc
    small = cc.cc_measure_random_loads(32 << 20)   # fits L2
    large = cc.cc_measure_random_loads(1 << 32)    # 4 GiB, far beyond L2
    # at least one load per SM per 16 clocks, at most 32 per SM per clock
    # (152 SMs at up to 2.1 GHz)
    assert 152 * 1.0e9 / 16 < small < 32 * 152 * 2.1e9
    assert 0 < large <= small * 1.05


def test_random_load_rate_rejects_bad_sizes():
    import paper_2507_03695_gb300 as cc
    for bad in (12345, 1 << 15, 1 << 33):
        with pytest.raises(cc.CCError):
            cc.cc_measure_random_loads(bad)
