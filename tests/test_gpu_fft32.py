"""The FP32 segmented FFT route (Sec. III.B circulant convolution on segments) against the oracle.

Every segment length S the autotuner can pick is run on its own: shapes whose tiles take several
inverse transforms (more segments than the proven term count T, so several rounded parities are
XORed per output), ragged tails, both forms, and the all-ones input whose sums are the largest
the bound covers. A caller that forces T past the bound on all-ones input makes sums leave FP32's
exact range: the rounding guard trips and the exact direct kernel recomputes the call, so the
output is still the oracle's. Bar: bit-exact.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import extract

pytestmark = pytest.mark.gpu

STD, MOD = 0, 1
FFT32 = 4


@pytest.fixture
def fft32(qlib, gpu):
    yield lambda seg=0, terms=0: qlib.qrng_set_fft32(gpu, seg, terms)
    qlib.qrng_set_fft32(gpu, 0, 0)


@pytest.mark.parametrize("seg", [2048, 4096, 8192])
@pytest.mark.parametrize("n,m,form,B", [
    (100, 37, STD, 3), (2048, 1024, STD, 5), (4097, 4000, STD, 2), (20000, 9000, MOD, 3),
    (70_000, 33_000, STD, 2), (150_001, 20_001, MOD, 2), (1 << 16, 36473, STD, 2),
])
def test_segment_lengths_bit_exact(qlib, gpu, oracle_mod, fft32, seg, n, m, form, B):
    fft32(seg)
    L = n + m - 1 if form == STD else n - 1
    raw = W.random_bits(n * B, 3 * n + m)
    seed = W.random_bits(L, 5 * n + m)
    qlib.qrng_reset_stats(gpu)
    got = extract(qlib, gpu, raw, n, m, seed, form, FFT32, B)
    assert np.array_equal(got, oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B))
    st = qlib.qrng_get_stats(gpu)
    assert st["last_fft32_segment"] == seg and st["fft32_recomputed"] == 0
    assert st["worst_fft32_round_err"] < 0.25


@pytest.mark.parametrize("seg", [2048, 4096, 8192])
def test_all_ones_within_the_bound(qlib, gpu, fft32, seg):
    """All raw and seed bits set: every segment-window product is as large as the bound allows, and
    T of them are summed per inverse; each output is the parity of n."""
    fft32(seg)
    T = qlib.qrng_fft32_terms_bound(seg)
    n, m, B = seg * (2 * T + 1), 3 * seg + 17, 2  # three inverses per tile
    raw = np.full(n * B // 8, 0xFF, dtype=np.uint8)
    seed = W.pack_bits(np.ones(n + m - 1, dtype=np.uint8))
    qlib.qrng_reset_stats(gpu)
    got = extract(qlib, gpu, raw, n, m, seed, STD, FFT32, B)
    bits = np.unpackbits(got, bitorder="little")[:m * B]
    assert np.all(bits == (n & 1))
    st = qlib.qrng_get_stats(gpu)
    assert st["fft32_recomputed"] == 0 and 0.0 <= st["worst_fft32_round_err"] < 0.25


def test_forced_terms_trip_the_guard_and_are_recomputed(qlib, gpu, oracle_mod, fft32):
    """T forced far past the bound on all-ones input: one inverse sums all 2048 segments, the sums
    reach 2^23 (where FP32 steps by 1), the guard trips, and the direct kernel recomputes the call."""
    fft32(4096, 4096)
    n, m, B = 1 << 23, 2000, 2
    raw = np.full(n * B // 8, 0xFF, dtype=np.uint8)
    seed = W.random_bits(n + m - 1, 9)
    qlib.qrng_reset_stats(gpu)
    got = extract(qlib, gpu, raw, n, m, seed, STD, FFT32, B)
    st = qlib.qrng_get_stats(gpu)
    assert st["worst_fft32_round_err"] >= 0.25, st
    assert st["fft32_recomputed"] == 1
    bits = np.unpackbits(got, bitorder="little")
    for b in range(B):
        idx = np.arange(b, m, 9, dtype=np.uint64)
        want = oracle_mod.toeplitz_bits(raw, n, m, seed, STD, idx, raw_off=b * n)
        assert np.array_equal(bits[b * m + idx.astype(np.int64)], want), b
    qlib.qrng_synchronize(gpu)  # a repaired trip is not an error


def test_auto_tunes_the_segment_length(qlib, gpu, oracle_mod, fft32):
    """AUTO times the FP32 route once per segment length; whatever it keeps, the bits are exact."""
    n, m, B = 1 << 16, 49152, 64
    raw = W.random_bits(n * B, 21)
    seed = W.random_bits(n - 1, 22)
    got = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_AUTO, B)
    assert not oracle_mod.freivalds(raw, n, m, seed, MOD, B, got).any()


def test_settings_rejected(qlib, gpu):
    for seg, terms in [(1024, 0), (3000, 0), (16384, 0), (4096, -1)]:
        with pytest.raises(qlib.QrngError) as e:
            qlib.qrng_set_fft32(gpu, seg, terms)
        assert e.value.status == qlib.QRNG_EINVAL
