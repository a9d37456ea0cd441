"""GPU checks of sg_probe_gather, the gather-rate probe the benchmark reads the walk kernels
against: every mode returns a finite positive rate, dependent chains (one gather in flight per
thread) are slower than independent gathers, one 256-bit load per record gathers faster than
two 16-byte loads, and an L2-resident table serves random gathers faster than a table over
four times the L2 size."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_probe_modes_and_orderings():
    import torch
    import paper_2603_15780_gb300 as sg
    tb = 16 << 20
    stream = sg.probe_gather(sg.PROBE_STREAM, tb, 4, 256, 20)
    rand = sg.probe_gather(sg.PROBE_RANDOM, tb, 4, 256, 128)
    rand256 = sg.probe_gather(sg.PROBE_RANDOM | sg.PROBE_LD256, tb, 4, 256, 128)
    chain4 = sg.probe_gather(sg.PROBE_CHAIN, tb, 4, 256, 128)
    for r in (stream, rand, rand256, chain4):
        assert math.isfinite(r) and r > 0
    assert chain4 < rand
    assert rand256 > 1.3 * rand
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    big = 1 << (4 * l2 - 1).bit_length()           # a power of two >= 4 x L2
    rand_big = sg.probe_gather(sg.PROBE_RANDOM, min(big, 1 << 31), 4, 256, 128)
    assert rand_big < rand
    print({"stream": stream, "random": rand, "random256": rand256, "chain4": chain4, "random_hbm": rand_big})
