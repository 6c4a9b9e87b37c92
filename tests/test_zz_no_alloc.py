"""qrng_minentropy_noalloc: the allocation-free variant of the min-entropy entry point.

It exists for callers that cannot allocate device memory (acquisition loops that must not
block on an allocation once streaming, programs whose GPU memory belongs to another allocator).
Its scratch is a fixed array inside the library, shared by every call; this test checks, through
the C ABI, that two calls in a row each agree with qrng_minentropy on the same samples, so a
stale histogram from the previous call would show. This file sorts last so that a run stopping
at the first failure has run every other test before it.
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


def test_noalloc_matches_context_entry_point_twice(qlib, gpu):
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


def test_noalloc_rejects_more_codes_than_its_scratch(qlib, gpu):
    import torch

    t = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_minentropy_noalloc(t.data_ptr(), 32, 17, 1e-6)
    assert e.value.status == qlib.QRNG_EINVAL
