"""Device-side failure detection without a GPU fault: a fault armed on the host makes the
tensor-core kernel's loader publish nothing, so every wait that depends on it runs out after its
bound; the kernel records a status, frees its tensor memory and returns. The host sees
QRNG_ETIMEOUT and the context keeps working."""
import time

import numpy as np
import pytest

import workloads as W
from gpu_util import extract, to_dev

pytestmark = pytest.mark.gpu


# QRNG_ALGO_GEMM_TC, QRNG_ALGO_GEMM_FP4, QRNG_ALGO_GEMM_FP4_PAIR, QRNG_ALGO_GEMM_KARATSUBA
@pytest.mark.parametrize("gemm", [2, 6, 7, 8])
def test_timeout_reported_and_context_recovers(qlib, gpu, gemm):
    import torch

    n, m, B = 4096, 2048, 256
    raw = W.random_bits(n * B, 61)
    seed = W.random_bits(n + m - 1, 62)
    _r, raw_p = to_dev(raw)
    _s, seed_p = to_dev(seed)
    out = torch.zeros(m * B // 8, dtype=torch.uint8, device="cuda")
    qlib.qrng_inject_fault(gpu, qlib.QRNG_FAULT_GEMM_NO_TMA)
    t0 = time.monotonic()
    qlib.qrng_toeplitz_extract(gpu, raw_p, n, m, seed_p, 0, gemm, B, out)
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_synchronize(gpu)
    assert e.value.status == qlib.QRNG_ETIMEOUT
    assert time.monotonic() - t0 < 60
    # the condition is cleared and the same context computes correctly again
    qlib.qrng_synchronize(gpu)
    got = extract(qlib, gpu, raw, n, m, seed, 0, gemm, B)
    ref = extract(qlib, gpu, raw, n, m, seed, 0, qlib.QRNG_ALGO_DIRECT, B)
    assert np.array_equal(got, ref)


def test_unknown_fault_rejected(qlib, gpu):
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_inject_fault(gpu, 99)
    assert e.value.status == qlib.QRNG_EINVAL
