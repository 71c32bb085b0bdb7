"""The device generator (synth_gpu.cu) against the host generator (synth.c).

Both run the steps of synth_core.h, so a workload generated on the device
must equal the host's, packed, bit for bit: offsets, candidate lists, kinds,
true candidates and every base.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _assert_same(dev, host):
    for f in ("read_offsets", "window_offsets", "pair_read", "cand_offsets", "kinds", "true_cand"):
        np.testing.assert_array_equal(getattr(dev, f).cpu().numpy(), getattr(host, f), err_msg=f)
    np.testing.assert_array_equal(dev.reads.cpu().numpy(), host.packed_reads())
    np.testing.assert_array_equal(dev.windows.cpu().numpy(), host.packed_windows())
    assert dev.cells() == host.cells()


@pytest.mark.parametrize("name,n_reads,seed", [("parity", 1000, 3), ("throughput", 20000, 0), ("uneven", 20000, 5),
                                               ("filter", 2000, 2), ("fullmix", 8000, 9)])
def test_device_generator_equals_host(name, n_reads, seed):
    _assert_same(synth.generate_device(name, seed=seed, n_reads=n_reads),
                 synth.generate(name, seed=seed, n_reads=n_reads))


def test_device_generator_read_range_and_tiny_sets():
    _assert_same(synth.generate_device("fullmix", seed=6, n_reads=700, first_read=4_321_000),
                 synth.generate("fullmix", seed=6, n_reads=700, first_read=4_321_000))
    for n in (1, 2, 3):   # sequences sharing packed words with their neighbours at both ends
        _assert_same(synth.generate_device("uneven", seed=n, n_reads=n), synth.generate("uneven", seed=n, n_reads=n))
