"""GPU parity of qrng_minentropy (histogram kernel + FP64 finaliser) against the oracle (Sec. II).

Bar: integers (count, max_count, argmax) exact; every floating-point field within 1e-12 absolute.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
FLOAT_KEYS = ("h_modify", "h_emp", "h_model", "d_u", "d_u_peak", "delta_fs", "delta_hm", "mean", "var")


def _run(q, ctx, samples, bits, eps, offset=0):
    import torch

    raw = samples.view(np.uint8)
    buf = torch.zeros(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size] = torch.from_numpy(raw).to("cuda")
    return q.qrng_minentropy(ctx, buf.data_ptr() + offset, samples.size, bits, eps)


def _compare(got, want):
    for k in ("count", "max_count", "argmax", "bits"):
        assert got[k] == want[k], k
    for k in FLOAT_KEYS:
        # entropies, distances and corrections: 1e-12 absolute; moments: 1e-12 relative
        tol = TOL * max(1.0, abs(want[k])) if k in ("mean", "var") else TOL
        assert abs(got[k] - want[k]) <= tol, (k, got[k], want[k])


def test_plain_single_block_samples(qlib, gpu, oracle_mod):
    c = W.CFG1
    s = W.adc_samples(c["samples"], c["sample_seed"])
    _compare(_run(qlib, gpu, s, 8, c["eps"]), oracle_mod.minentropy(s, 8, c["eps"]))


def test_laser_stream_full_size(qlib, gpu, oracle_mod):
    c = W.CFG2
    s = W.adc_samples(c["samples"], c["sample_seed"])
    got = _run(qlib, gpu, s, 8, c["eps"])
    _compare(got, oracle_mod.minentropy(s, 8, c["eps"]))
    assert 4.0 < got["h_modify"] < 5.4


@pytest.mark.parametrize("offset", [1, 3, 7, 15])
@pytest.mark.parametrize("count", [1, 15, 17, 1000, 65537])
def test_unaligned_and_ragged(qlib, gpu, oracle_mod, offset, count):
    s = W.adc_samples(count, 100 + count, mu=100.0, sigma=9.0)
    _compare(_run(qlib, gpu, s, 8, 1e-3, offset), oracle_mod.minentropy(s, 8, 1e-3))


@pytest.mark.parametrize("bits", [10, 13, 14, 15, 16])
@pytest.mark.parametrize("offset", [1, 2, 6, 14])
@pytest.mark.parametrize("count", [1, 7, 9, 100_003])
def test_wide_samples_unaligned_and_ragged(qlib, gpu, oracle_mod, bits, offset, count):
    """uint16 samples at any byte address (odd ones included) and counts that leave a ragged head
    and tail around the 16-byte vectors."""
    s = W.adc_samples(count, 7 * bits + count, mu=(1 << bits) / 3, sigma=(1 << bits) / 9, bits=bits)
    _compare(_run(qlib, gpu, s, bits, 1e-6, offset), oracle_mod.minentropy(s, bits, 1e-6))


@pytest.mark.parametrize("bits", [8, 16])
def test_one_code_holds_every_sample(qlib, gpu, oracle_mod, bits):
    """Every sample on one code: the per-lane 16-bit copies (8-bit) and the cluster counters (16-bit)
    must carry counts far above 2^16 into the totals."""
    s = np.full(3_000_001, 200 if bits == 8 else 40000, dtype=np.uint8 if bits == 8 else np.uint16)
    got = _run(qlib, gpu, s, bits, 1e-6)
    _compare(got, oracle_mod.minentropy(s, bits, 1e-6))
    assert got["max_count"] == s.size


@pytest.mark.parametrize("bits", [1, 2, 5, 7, 9, 12, 13, 14, 16])
def test_bit_widths(qlib, gpu, oracle_mod, bits):
    mu = (1 << bits) / 2.0
    sigma = max(0.3, (1 << bits) / 10.0)
    s = W.adc_samples(300_000 + bits, 200 + bits, mu=mu, sigma=sigma, bits=bits)
    _compare(_run(qlib, gpu, s, bits, 1e-6), oracle_mod.minentropy(s, bits, 1e-6))


def test_point_mass_and_flat(qlib, gpu, oracle_mod):
    s = np.full(5000, 77, dtype=np.uint8)
    got = _run(qlib, gpu, s, 8, 1e-6)
    _compare(got, oracle_mod.minentropy(s, 8, 1e-6))
    assert got["h_modify"] == 0.0 and got["h_emp"] == 0.0
    f = np.tile(np.arange(256, dtype=np.uint8), 1000)
    got = _run(qlib, gpu, f, 8, 1e-6)
    _compare(got, oracle_mod.minentropy(f, 8, 1e-6))
    assert abs(got["h_emp"] - 8.0) < TOL


@pytest.mark.parametrize("counts", [
    {1: 30, 2: 15, 3: 30, 5: 25},     # two codes share the largest count: the lower one is reported
    {2: 40, 3: 25, 4: 35},            # the measured peak (code 2) is not the model's (code 3)
    {0: 7, 1: 7},                     # 1-bit tie
])
@pytest.mark.parametrize("scale", [1, 1000, 100_003])
def test_ties_and_peak_distance(qlib, gpu, oracle_mod, counts, scale):
    """argmax (lowest code on ties) and the distance over U = {argmax P'}, with the samples in a
    random order and the counts large enough to spread over many CTAs."""
    bits = 1 if max(counts) < 2 else 3
    s = np.concatenate([np.full(c * scale, v, dtype=np.uint8) for v, c in counts.items()])
    W.rng(scale).shuffle(s)
    got = _run(qlib, gpu, s, bits, 1e-6)
    want = oracle_mod.minentropy(s, bits, 1e-6)
    _compare(got, want)
    assert got["argmax"] == min(v for v, c in counts.items() if c == max(counts.values()))


def test_out_of_range_sample_rejected(qlib, gpu):
    s = W.adc_samples(1000, 5, mu=8.0, sigma=3.0, bits=4)
    s[123] = 200
    with pytest.raises(qlib.QrngError) as e:
        _run(qlib, gpu, s, 4, 1e-6)
    assert e.value.status == qlib.QRNG_EINVAL


def test_bad_arguments(qlib, gpu):
    import torch

    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for bits, eps, count in [(0, 1e-6, 16), (17, 1e-6, 16), (8, 0.0, 16), (8, 1.0, 16), (8, 1e-6, 0)]:
        with pytest.raises(qlib.QrngError) as e:
            qlib.qrng_minentropy(gpu, t, count=count, bits=bits, eps=eps)
        assert e.value.status == qlib.QRNG_EINVAL
    with pytest.raises(qlib.QrngError):
        qlib.qrng_minentropy(gpu, 0, count=16, bits=8, eps=1e-6)


def test_repeated_calls_reuse_workspace(qlib, gpu, oracle_mod):
    for seed in range(3):
        s = W.adc_samples(100_000, 300 + seed)
        _compare(_run(qlib, gpu, s, 8, 1e-6), oracle_mod.minentropy(s, 8, 1e-6))
