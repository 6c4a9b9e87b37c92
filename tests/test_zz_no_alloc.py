"""qrng_minentropy_noalloc: the allocation-free variant of the min-entropy entry point.

It exists for callers that cannot allocate device memory (acquisition loops that must not
block on an allocation once streaming, programs whose GPU memory belongs to another allocator).
Its scratch is a fixed array inside the library, shared by every call; this test checks, through
the C ABI, that two calls in a row each agree with qrng_minentropy and with the oracle on the same
samples, so a stale histogram from the previous call would show; that a call rejected for an
out-of-range sample leaves the shared scratch fit for the next call; and that a call after the
first one on the device takes no device memory. This file sorts last so that a run stopping at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
FLOAT_KEYS = ("h_modify", "h_emp", "h_model", "d_u", "d_u_peak", "delta_fs", "delta_hm")


def _same(got, want):
    for k in ("count", "max_count", "argmax", "bits"):
        assert got[k] == want[k], k
    for k in FLOAT_KEYS:
        assert abs(got[k] - want[k]) <= TOL, (k, got[k], want[k])
    for k in ("mean", "var"):
        assert abs(got[k] - want[k]) <= TOL * max(1.0, abs(want[k])), k


def test_noalloc_matches_context_entry_point_twice(qlib, gpu, oracle_mod):
    import torch

    inputs = [
        (W.adc_samples(1 << 20, 901), 8),                                 # Gaussian ADC stream
        (W.adc_samples(300_001, 902, mu=40.0, sigma=9.0, bits=12), 12),   # different width and shape
    ]
    for samples, bits in inputs:  # two calls in a row on the shared scratch
        dev = torch.from_numpy(samples.view(np.uint8)).to("cuda")
        got = qlib.qrng_minentropy_noalloc(dev.data_ptr(), samples.size, bits, 1e-6)
        want = qlib.qrng_minentropy(gpu, dev.data_ptr(), samples.size, bits, 1e-6)
        _same(got, want)
        _same(got, oracle_mod.minentropy(samples, bits, 1e-6))


def test_noalloc_out_of_range_then_valid_call(qlib, gpu, oracle_mod):
    """A 12-bit stream with one code >= 4096 is rejected; the counters it left behind in the shared
    scratch must not leak into the next, valid call."""
    import torch

    bad = W.adc_samples(200_000, 903, mu=2000.0, sigma=300.0, bits=12)
    bad[77_777] = 4096
    dev_bad = torch.from_numpy(bad.view(np.uint8)).to("cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_minentropy_noalloc(dev_bad.data_ptr(), bad.size, 12, 1e-6)
    assert e.value.status == qlib.QRNG_EINVAL
    good = W.adc_samples(150_001, 904, mu=1000.0, sigma=200.0, bits=12)
    dev = torch.from_numpy(good.view(np.uint8)).to("cuda")
    got = qlib.qrng_minentropy_noalloc(dev.data_ptr(), good.size, 12, 1e-6)
    _same(got, qlib.qrng_minentropy(gpu, dev.data_ptr(), good.size, 12, 1e-6))
    _same(got, oracle_mod.minentropy(good, 12, 1e-6))


def test_noalloc_takes_no_device_memory_after_first_call(qlib, gpu):
    """After the first call on the device (which may load the library's device code and place its
    fixed arrays), further calls leave the device's free memory unchanged."""
    import torch

    samples = W.adc_samples(1 << 18, 905)
    dev = torch.from_numpy(samples).to("cuda")
    qlib.qrng_minentropy_noalloc(dev.data_ptr(), samples.size, 8, 1e-6)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        qlib.qrng_minentropy_noalloc(dev.data_ptr(), samples.size, 8, 1e-6)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_more_codes_than_its_scratch(qlib, gpu):
    import torch

    t = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_minentropy_noalloc(t.data_ptr(), 32, 17, 1e-6)
    assert e.value.status == qlib.QRNG_EINVAL
