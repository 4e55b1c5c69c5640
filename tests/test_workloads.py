"""The seeded input recipes (no method arithmetic): shapes, distributions, fault draws and
the FP8 E4M3 block quantiser the FP8 workload feeds to both the CUDA path and the oracle."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import workloads as wl


def test_e4m3_quantiser_power_of_two_scales_and_rounding():
    x = wl.operand((300, 260), "fp8rows", 5, 1)
    q, s = wl.quantize_e4m3(x)
    assert q.dtype == np.uint8 and q.shape == x.shape and s.shape == (3, 3)
    m, e = np.frexp(s.astype(np.float64))
    assert np.all(m == 0.5)                                  # powers of two
    full = np.repeat(np.repeat(s.astype(np.float64), 128, 0), 128, 1)[:300, :260]
    assert np.max(np.abs(x) / full) <= wl.E4M3_MAX           # no code saturates
    d = oracle.dequant_e4m3(q, s)
    # round to nearest E4M3: error at most half a unit of the last place of the code
    # (2^-4 relative for normal codes, 2^-10 of the scale in the subnormal range)
    y = np.abs(x) / full
    ulp_half = np.where(y >= 2.0 ** -6, 2.0 ** (np.floor(np.log2(np.maximum(y, 2.0 ** -6))) - 4),
                        2.0 ** -10)
    assert np.all(np.abs(d - x) / full <= ulp_half * (1 + 1e-12))


def test_e4m3_quantiser_zero_block():
    x = np.zeros((128, 256))
    x[:, 128:] = 1.0
    q, s = wl.quantize_e4m3(x)
    assert s[0, 0] == 1.0 and np.all(q[:, :128] == 0)
    assert np.all(oracle.dequant_e4m3(q, s)[:, 128:] == 1.0)


def test_group_shapes_and_faulty_instances():
    w = wl.BF16_GROUPED_4096
    shapes = wl.group_shapes(0, w)
    v = np.array(shapes)
    assert v.shape == (4096, 3) and v.min() >= 64 and v.max() <= 2048 and np.all(v % 64 == 0)
    assert len(np.unique(v[:, 0])) == 32                    # every multiple of 64 occurs
    f = wl.faulty_instances(0, 4096, 0.01)
    assert len(f) == 41 and f == sorted(set(f)) and max(f) < 4096
    assert wl.group_shapes(0, w) == shapes                   # seeded


def test_bit_flips_refuses_more_flips_than_free_blocks():
    """Flips in distinct blocks: a request the block grid cannot hold is refused at once
    (it would otherwise redraw forever)."""
    with pytest.raises(ValueError):
        wl.bit_flips(1, 320, 256, 3, distinct_blocks=(256, 256))
    with pytest.raises(ValueError):
        wl.bit_flips(1, 512, 512, 4, distinct_blocks=(256, 256), avoid_blocks=[(0, 0)])
    got = wl.bit_flips(1, 320, 256, 2, distinct_blocks=(256, 256))
    assert sorted(i // 256 for i, _, _ in got) == [0, 1]
