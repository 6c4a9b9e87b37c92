"""GPU parity of qrng_toeplitz_extract against the oracle (Sec. III.B standard, Sec. III.D modified,
Sec. III.E blocks). Bar: bit-exact.

Small and medium shapes are compared in full. The full-size workloads are compared on every
block with the oracle's Freivalds check (64 random parity tests per block, escape probability
2^-64) and on sampled output bits computed one by one by the oracle.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import extract, spot_check

pytestmark = pytest.mark.gpu

STD, MOD = 0, 1
ALGOS = {"direct": 1, "gemm_tc": 2, "fft64": 3, "fft32_seg": 4, "ntt": 5, "gemm_fp4": 6, "gemm_fp4_pair": 7,
         "gemm_karatsuba": 8}
GEMMS = {"gemm_tc": 2, "gemm_fp4": 6, "gemm_fp4_pair": 7, "gemm_karatsuba": 8}


def _seed_len(n, m, form):
    return n + m - 1 if form == STD else n - 1


def _case(n, m, form, B, s):
    raw = W.random_bits(n * B, 1000 + s)
    seed = W.random_bits(_seed_len(n, m, form), 2000 + s)
    return raw, seed


SMALL = [
    (1, 1, STD, 1), (2, 1, MOD, 3), (2, 2, STD, 5), (31, 7, STD, 5), (32, 32, STD, 4), (33, 17, MOD, 7),
    (64, 1, STD, 9), (100, 99, MOD, 2), (1000, 333, STD, 5), (1000, 333, MOD, 5), (4096, 2048, STD, 1),
    (4096, 3072, MOD, 16), (4101, 1000, STD, 3), (3000, 2900, STD, 2), (2048, 1024, MOD, 40),
    (511, 257, STD, 33), (1 << 12, (1 << 12) - 1, MOD, 2), (777, 777, STD, 3),
]


@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("n,m,form,B", SMALL)
def test_small_shapes_bit_exact(qlib, gpu, oracle_mod, algo, n, m, form, B):
    raw, seed = _case(n, m, form, B, n * 31 + m + B)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    got = extract(qlib, gpu, raw, n, m, seed, form, ALGOS[algo], B)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("raw_off,seed_off,out_off", [(1, 0, 0), (0, 3, 0), (0, 0, 1), (5, 7, 2), (4, 4, 4)])
@pytest.mark.parametrize("n,m,form,B", [(4096, 2048, STD, 3), (1000, 333, MOD, 4), (256, 96, MOD, 8)])
def test_unaligned_pointers(qlib, gpu, oracle_mod, algo, raw_off, seed_off, out_off, n, m, form, B):
    raw, seed = _case(n, m, form, B, 7 + raw_off + 3 * out_off)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    got = extract(qlib, gpu, raw, n, m, seed, form, ALGOS[algo], B, raw_off, seed_off, out_off)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("algo", list(ALGOS))
def test_single_long_block_full(qlib, gpu, oracle_mod, algo):
    n, m = 1 << 16, 36_000
    raw, seed = _case(n, m, STD, 1, 99)
    want = oracle_mod.toeplitz(raw, n, m, seed, STD)
    assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, ALGOS[algo], 1), want)


@pytest.mark.parametrize("algo", list(ALGOS))
def test_identity_block_with_zero_seed(qlib, gpu, algo):
    n, m, B = 4096, 3000, 6
    raw = W.random_bits(n * B, 55)
    seed = np.zeros((n - 1 + 7) // 8, dtype=np.uint8)
    got = np.unpackbits(extract(qlib, gpu, raw, n, m, seed, MOD, ALGOS[algo], B), bitorder="little")
    bits = np.unpackbits(raw, bitorder="little")
    for b in range(B):
        assert np.array_equal(got[b * m:(b + 1) * m], bits[b * n + n - m:(b + 1) * n])


@pytest.mark.parametrize("algo", list(ALGOS))
def test_all_ones(qlib, gpu, oracle_mod, algo):
    """Every raw and seed bit set: each output is the parity of the row's seed-bit count."""
    n, m, B = 2048, 1500, 4
    raw = np.full(n * B // 8, 0xFF, dtype=np.uint8)
    seed = W.pack_bits(np.ones(n + m - 1, dtype=np.uint8))
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, STD, B)
    assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, ALGOS[algo], B), want)


@pytest.mark.parametrize("gemm", list(GEMMS))
@pytest.mark.parametrize("n,m,B", [(1 << 16, 4096, 300), (1 << 22, 1024, 8), ((1 << 22) - 96, 1000, 3)])
def test_gemm_all_ones_largest_sums(qlib, gpu, oracle_mod, gemm, n, m, B):
    """All-ones raw and seed make every tensor-core sum equal to n, the largest count the FP32
    accumulator has to hold exactly; each output is the parity of n."""
    raw = np.full(n * B // 8, 0xFF, dtype=np.uint8)
    seed = W.pack_bits(np.ones(n + m - 1, dtype=np.uint8))
    got = extract(qlib, gpu, raw, n, m, seed, STD, GEMMS[gemm], B)
    want = np.zeros(m * B, dtype=np.uint8) + (n & 1)
    assert np.array_equal(np.unpackbits(got, bitorder="little")[:m * B], want)
    # and a random seed with all-ones raw bits: each output is the parity of a seed window
    seed = W.random_bits(n + m - 1, 5)
    got = extract(qlib, gpu, raw, n, m, seed, STD, GEMMS[gemm], B)
    spot_check(oracle_mod, raw, n, m, seed, STD, got, blocks=[0, B - 1], per_block=64)


_ORACLE_CHECKED = set()  # direct-kernel references already checked against the oracle


def _checked_direct(qlib, gpu, oracle_mod, raw, n, m, seed, B, key):
    """The direct kernel's output, checked once per key against the oracle on every block
    (Freivalds, 64 random row combinations per block), so that comparisons with it reach the oracle."""
    ref = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_DIRECT, B)
    if key not in _ORACLE_CHECKED:
        assert not oracle_mod.freivalds(raw, n, m, seed, STD, B, ref).any()
        _ORACLE_CHECKED.add(key)
    return ref


@pytest.mark.parametrize("gemm", list(GEMMS))
def test_gemm_full_occupancy_repeated(qlib, gpu, oracle_mod, gemm):
    """Every SM busy (one or two tiles per CTA), long K (n = 2^16), repeated: the pipelines that
    hand raw tiles and operand stages between warps are exercised at full speed. The output equals
    the direct kernel's (checked against the oracle on every block) on every repetition."""
    n = 1 << 16
    for m, B in ((2048, 224 * 19), (4096, 256 * 19)):
        raw = W.random_bits(n * B, 321 + m)
        seed = W.random_bits(n + m - 1, 654 + m)
        ref = _checked_direct(qlib, gpu, oracle_mod, raw, n, m, seed, B, ("occupancy", m, B))
        for _ in range(3):
            assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, GEMMS[gemm], B), ref)


@pytest.mark.parametrize("algo", list(ALGOS))
def test_algorithms_agree_on_laser_stream(qlib, gpu, oracle_mod, algo):
    """Every algorithm gives byte-identical output on the full-size stream, equal to the direct
    kernel's, which is checked against the oracle on every block."""
    c = W.CFG2
    samples = W.adc_samples(c["samples"], c["sample_seed"])
    n, m = c["n"], 36473
    B = samples.size * 8 // n
    seed = W.random_bits(n + m - 1, c["seed_seed"])
    ref = _checked_direct(qlib, gpu, oracle_mod, samples, n, m, seed, B, ("laser",))
    got = extract(qlib, gpu, samples, n, m, seed, STD, ALGOS[algo], B)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("algo,bound", [("fft64", 1e-6), ("fft32_seg", 0.25)])
def test_fft_rounding_evidence(qlib, gpu, oracle_mod, algo, bound):
    """The FFT paths report the largest distance of a used convolution sum from its integer; it
    stays inside the exactness margin (the guard trips at 0.25)."""
    n, m, B = 1 << 14, 12000, 16
    raw, seed = _case(n, m, STD, B, 4711)
    qlib.qrng_reset_stats(gpu)
    got = extract(qlib, gpu, raw, n, m, seed, STD, ALGOS[algo], B)
    st = qlib.qrng_get_stats(gpu)
    assert 0.0 < st["worst_fft_round_err"] < bound, st
    assert qlib.qrng_extract_stats(gpu) == st["worst_fft_round_err"]  # the same figure, alone
    assert not oracle_mod.freivalds(raw, n, m, seed, STD, B, got).any()
    qlib.qrng_reset_stats(gpu)
    assert qlib.qrng_extract_stats(gpu) == 0.0


@pytest.mark.parametrize("log2n", [12, 18, 24])
def test_ntt_block_length_sweep_point(qlib, gpu, oracle_mod, log2n):
    """The exact number-theoretic route on the fixed 2^30-bit stream, modified form, m = 0.75 n."""
    c = W.CFG3
    n = 1 << log2n
    m = int(n * c["ratio"])
    B = c["stream_bits"] // n
    raw = W.random_bits(c["stream_bits"], c["raw_seed"])
    seed = W.random_bits(n - 1, c["seed_seed"] + log2n)
    got = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_NTT, B)
    ref = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_FFT64, B)
    assert np.array_equal(got, ref)
    spot_check(oracle_mod, raw, n, m, seed, MOD, got, blocks=[0, B - 1], per_block=128)


def test_ntt_transform_length_2_25(qlib, gpu, oracle_mod):
    """n = 2^24 in the standard form needs P = 2^25: rows of 2^13 entries and column tiles narrower
    than a byte, i.e. the route that packs the bits into entries and extracts the output from them."""
    n, m, B = 1 << 24, 4096, 2
    raw = W.random_bits(n * B, 71)
    seed = W.random_bits(n + m - 1, 72)
    got = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_NTT, B)
    ref = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_FFT64, B)
    assert np.array_equal(got, ref)
    spot_check(oracle_mod, raw, n, m, seed, STD, got, blocks=[0, B - 1], per_block=32)


@pytest.mark.parametrize("log2n", [12, 16, 20])
def test_fft64_block_length_sweep_point(qlib, gpu, oracle_mod, log2n):
    """The paper's FFT route on the fixed 2^30-bit stream, modified form, m = 0.75 n."""
    c = W.CFG3
    n = 1 << log2n
    m = int(n * c["ratio"])
    B = c["stream_bits"] // n
    raw = W.random_bits(c["stream_bits"], c["raw_seed"])
    seed = W.random_bits(n - 1, c["seed_seed"] + log2n)
    got = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_FFT64, B)
    ref = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_DIRECT, B)
    assert np.array_equal(got, ref)
    spot_check(oracle_mod, raw, n, m, seed, MOD, got, blocks=[0, B - 1], per_block=128)


def test_auto_tunes_once_per_shape(qlib, gpu, oracle_mod):
    """AUTO runs the candidates once for a new shape, keeps the fastest, and reuses it."""
    n, m, B = 8192, 6144, 512
    raw, seed = _case(n, m, STD, B, 77)
    want = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_DIRECT, B)
    qlib.qrng_set_autotune(gpu, True)
    qlib.qrng_reset_stats(gpu)
    got1 = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
    first = qlib.qrng_get_stats(gpu)
    got2 = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
    second = qlib.qrng_get_stats(gpu)
    assert np.array_equal(got1, want) and np.array_equal(got2, want)
    assert second["last_algo"] == first["last_algo"] != qlib.QRNG_ALGO_AUTO
    assert second["last_kernels"] <= first["last_kernels"]  # no candidates re-run
    qlib.qrng_set_autotune(gpu, False)
    got3 = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
    assert np.array_equal(got3, want)
    qlib.qrng_set_autotune(gpu, True)


def test_auto_tunes_once_per_m_class(qlib, gpu, oracle_mod):
    """Calls whose m differs by a few bits (a live stream's corrected min-entropy moves that much
    from call to call) share one tuning; an m outside the class (its six leading bits differ) is
    tuned again. Every output equals the oracle's."""
    n, B = 8192, 256
    qlib.qrng_set_autotune(gpu, True)  # starts with no tuned shapes
    qlib.qrng_reset_stats(gpu)
    runs = []
    for m, s in ((6144, 81), (6150, 82), (6271, 83), (4100, 84), (6145, 85)):
        raw, seed = _case(n, m, STD, B, s)
        got = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
        assert np.array_equal(got, oracle_mod.toeplitz_blocks(raw, n, m, seed, STD, B)), m
        runs.append(qlib.qrng_get_stats(gpu)["autotune_runs"])
    assert runs == [1, 1, 1, 2, 2], runs  # 6144..6271 is one class, 4100 another


@pytest.mark.parametrize("gemm", list(GEMMS))
def test_gemm_rejects_too_long_blocks(qlib, gpu, gemm):
    import torch

    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_toeplitz_extract(gpu, t, (1 << 22) + 32, 8, t, STD, GEMMS[gemm], 1, t)
    assert e.value.status == qlib.QRNG_ENOTSUP


def test_laser_stream_full_size(qlib, gpu, oracle_mod):
    """2^26 ADC samples as a 2^29-bit raw stream, n = 2^16, m = floor(n H_modify / 8), one shared seed."""
    import torch

    c = W.CFG2
    samples = W.adc_samples(c["samples"], c["sample_seed"])
    dev = torch.from_numpy(samples).to("cuda")
    rep = qlib.qrng_minentropy(gpu, dev, bits=8, eps=c["eps"])
    n = c["n"]
    m = qlib.qrng_output_length(n, rep["h_modify"], 8, 1.0)
    assert m == oracle_mod.output_length(n, oracle_mod.minentropy(samples, 8, c["eps"])["h_modify"], 8, 1.0)
    B = samples.size * 8 // n
    seed = W.random_bits(n + m - 1, c["seed_seed"])
    got = extract(qlib, gpu, samples, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
    mism = oracle_mod.freivalds(samples, n, m, seed, STD, B, got)
    assert not mism.any(), f"{np.count_nonzero(mism)} blocks fail the Freivalds check"
    spot_check(oracle_mod, samples, n, m, seed, STD, got, blocks=[0, 1, B // 2, B - 1], per_block=128)


@pytest.mark.parametrize("log2n", [10, 12, 14, 16, 18, 20, 22, 24])
def test_block_length_sweep_point(qlib, gpu, oracle_mod, log2n):
    """Fixed 2^30-bit stream, modified form, m = 0.75 n. Every block is Freivalds-checked where the
    oracle's O(nm) preparation is affordable; otherwise sampled bits of several blocks are checked."""
    c = W.CFG3
    n = 1 << log2n
    m = int(n * c["ratio"])
    B = c["stream_bits"] // n
    raw = W.random_bits(c["stream_bits"], c["raw_seed"])
    seed = W.random_bits(n - 1, c["seed_seed"] + log2n)
    got = extract(qlib, gpu, raw, n, m, seed, MOD, qlib.QRNG_ALGO_AUTO, B)
    if n * m <= (1 << 31):
        mism = oracle_mod.freivalds(raw, n, m, seed, MOD, B, got)
        assert not mism.any()
    blocks = sorted({0, 1, B // 3, B - 1})
    spot_check(oracle_mod, raw, n, m, seed, MOD, got, blocks=blocks, per_block=64 if n > (1 << 20) else 256)


def test_tensor_core_shape(qlib, gpu, oracle_mod):
    """One standard seed, m = 6144, n = 8192, 4096 blocks."""
    c = W.CFG4
    n, m, B = c["n"], c["m"], c["blocks"]
    raw = W.random_bits(n * B, c["raw_seed"])
    seed = W.random_bits(n + m - 1, c["seed_seed"])
    got = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_AUTO, B)
    assert not oracle_mod.freivalds(raw, n, m, seed, STD, B, got).any()
    spot_check(oracle_mod, raw, n, m, seed, STD, got, blocks=[0, 5, B - 1])


def test_maximum_block_length(qlib, gpu, oracle_mod):
    """n = 2^26 (the largest block), short output, every output bit checked."""
    n, m = 1 << 26, 96
    raw, seed = _case(n, m, STD, 1, 4242)
    got = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_DIRECT, 1)
    want = oracle_mod.toeplitz_bits(raw, n, m, seed, STD, np.arange(m, dtype=np.uint64))
    assert np.array_equal(np.unpackbits(got, bitorder="little")[:m], want)


def test_bad_arguments(qlib, gpu):
    import torch

    t = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    bad = [
        (64, 65, STD, 1, 1),   # m > n
        (64, 64, MOD, 1, 1),   # modified needs m < n
        (64, 0, STD, 1, 1),
        (0, 0, STD, 1, 1),
        (64, 8, 7, 1, 1),      # unknown form
        (64, 8, STD, 9, 1),    # unknown algorithm
        (64, 8, STD, 10, 1),   # unknown algorithm
        (64, 8, STD, -1, 1),   # unknown algorithm
        (64, 8, STD, 1, 0),    # no blocks
        ((1 << 26) + 1, 8, STD, 1, 1),
    ]
    for n, m, form, algo, B in bad:
        with pytest.raises(qlib.QrngError) as e:
            qlib.qrng_toeplitz_extract(gpu, t, n, m, t, form, algo, B, t)
        assert e.value.status == qlib.QRNG_EINVAL, (n, m, form, algo, B)
    with pytest.raises(qlib.QrngError):
        qlib.qrng_toeplitz_extract(gpu, 0, 64, 8, t, STD, 1, 1, t)


@pytest.mark.parametrize("bits,form,eps_lhl", [(12, MOD, 2.0 ** -4), (5, STD, 2.0 ** -20)])
def test_postprocess_host_other_widths(qlib, gpu, oracle_mod, bits, form, eps_lhl):
    """12-bit samples travel as little-endian uint16 and 5-bit ones as bytes; the raw stream is the
    sample buffer's bytes either way. (300,000 samples over 4096 codes leave a corrected entropy of
    0.084 bit per sample, so the 12-bit case takes a loose leftover-hash epsilon to keep m > 0.)"""
    samples = W.adc_samples(300_000, 33 + bits, mu=(1 << bits) / 2, sigma=(1 << bits) / 12, bits=bits)
    raw = samples.view(np.uint8)
    n = 2048
    seed = W.random_bits(2 * n - 1, 34)
    out = np.zeros(raw.size, dtype=np.uint8)
    m, B, rep = qlib.qrng_postprocess_host(gpu, samples, samples.size, bits, 1e-6, eps_lhl, n, seed, 2 * n - 1,
                                           form, qlib.QRNG_ALGO_AUTO, out, out.size)
    ref = oracle_mod.minentropy(samples, bits, 1e-6)
    want_m = oracle_mod.output_length(n, ref["h_modify"], bits, eps_lhl)
    assert want_m > 0
    if form == MOD:
        want_m = min(want_m, n - 1)
    assert m == want_m and B == raw.size * 8 // n
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    assert np.array_equal(out[:want.size], want)


def test_postprocess_host_reports_zero_output(qlib, gpu):
    """A corrected entropy that leaves no output bits is an error, with m = 0 reported."""
    samples = W.adc_samples(2000, 3)  # few samples: the finite-size term swamps the entropy
    seed = W.random_bits(8191, 1)
    out = np.zeros(16, dtype=np.uint8)
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_postprocess_host(gpu, samples, samples.size, 8, 1e-6, 2.0 ** -40, 4096, seed, 8191, STD,
                                   qlib.QRNG_ALGO_AUTO, out, out.size)
    assert e.value.status == qlib.QRNG_EINVAL


def test_postprocess_host_pipeline(qlib, gpu, oracle_mod):
    """Host buffers in, host buffer out: entropy, sizing and extraction in one call."""
    c = W.CFG1
    samples = W.adc_samples(c["samples"] * 4, 77)
    n = 4096
    seed = W.random_bits(2 * n - 1, 78)
    out = np.zeros(samples.size, dtype=np.uint8)
    m, B, rep = qlib.qrng_postprocess_host(gpu, samples, samples.size, 8, 1e-6, 1.0, n, seed, 2 * n - 1, STD,
                                           qlib.QRNG_ALGO_AUTO, out, out.size)
    ref = oracle_mod.minentropy(samples, 8, 1e-6)
    assert abs(rep["h_modify"] - ref["h_modify"]) < 1e-12
    assert m == oracle_mod.output_length(n, ref["h_modify"], 8, 1.0) and B == samples.size * 8 // n
    want = oracle_mod.toeplitz_blocks(samples, n, m, seed, STD, B)
    assert np.array_equal(out[:want.size], want)
