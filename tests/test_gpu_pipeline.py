"""GPU parity of the whole pipeline on device buffers (qrng_postprocess: Sec. II estimate, Sec. III.B
sizing, Sec. III.B-E hashing of the sample stream's blocks) against the oracle, including the
block-Karatsuba route's derived operands computed beside the estimate from the previous call's m:
a hit (same m), a miss (the modified form with a different m, whose operands depend on n - m), new
sample contents at the same address, a rejected call in between, the host-buffer pipeline that
shares the same first half, and its overlapped form (calls submitted back to back)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

STD, MOD = 0, 1


def _run(q, ctx, samples_dev, count, n, seed_dev, seed_bits, form, algo, out, eps_lhl=1.0):
    m, nb, rep = q.qrng_postprocess(ctx, samples_dev, count, 8, 1e-6, eps_lhl, n, seed_dev, seed_bits, form, algo,
                                    out, out.numel())
    q.qrng_synchronize(ctx)
    return m, nb, rep


def _check(oracle_mod, q, samples, n, seed, form, m, nb, rep, out, full=True):
    ref = oracle_mod.minentropy(samples, 8, 1e-6)
    assert abs(rep["h_modify"] - ref["h_modify"]) < 1e-12
    want_m = oracle_mod.output_length(n, ref["h_modify"], 8, 1.0)
    if form == MOD:
        want_m = min(want_m, n - 1)
    assert m == want_m and nb == samples.size * 8 // n
    raw = samples.view(np.uint8)
    got = out[:(nb * m + 7) // 8].cpu().numpy()
    if full:
        assert np.array_equal(got, oracle_mod.toeplitz_blocks(raw, n, m, seed, form, nb))
    else:
        assert not oracle_mod.freivalds(raw, n, m, seed, form, nb, got).any()


def _stats(q, ctx):
    s = q.qrng_get_stats(ctx)
    return s["kara_presplits"], s["kara_presplits_used"]


@pytest.mark.parametrize("algo_name", ["GEMM_KARATSUBA", "AUTO"])
def test_pipeline_presplit_hit_and_new_contents(qlib, gpu, oracle_mod, algo_name):
    """Three calls on one stream shape: the first plans alone, the second and third find their
    derived operands computed beside the estimate; the third call's samples are new contents at the
    same address (the operands are recomputed from them, not reused)."""
    import torch

    algo = getattr(qlib, "QRNG_ALGO_" + algo_name)
    n = 1 << 16
    count = 1 << 22  # 512 blocks of the laser-stream block length
    seed = W.random_bits(2 * n - 1, 611)
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    samples_dev = torch.empty(count, dtype=torch.uint8, device="cuda")
    qlib.qrng_reset_stats(gpu)
    for call, sseed in enumerate((612, 612, 613)):
        samples = W.adc_samples(count, sseed)
        samples_dev.copy_(torch.from_numpy(samples))
        m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD, algo, out)
        _check(oracle_mod, qlib, samples, n, seed, STD, m, nb, rep, out, full=False)
    pre, used = _stats(qlib, gpu)
    if algo_name == "GEMM_KARATSUBA":
        assert pre == 2 and used == 2, (pre, used)
    else:  # AUTO takes the route its tuner picked; the pre-split only follows a Karatsuba choice
        assert used == pre


def test_pipeline_presplit_miss_modified_form(qlib, gpu, oracle_mod):
    """Modified form: the derived operands depend on n - m, so a call whose m differs from the
    previous one computes them again (and still matches the oracle)."""
    import torch

    n = 8192
    count = 1 << 20
    seed = W.random_bits(n - 1, 621)
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    samples_dev = torch.empty(count, dtype=torch.uint8, device="cuda")
    qlib.qrng_reset_stats(gpu)
    ms = []
    for sseed, sigma in ((622, 16.0), (623, 11.0), (623, 11.0)):
        samples = W.adc_samples(count, sseed, sigma=sigma)
        samples_dev.copy_(torch.from_numpy(samples))
        m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, n - 1, MOD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
        _check(oracle_mod, qlib, samples, n, seed, MOD, m, nb, rep, out, full=False)
        ms.append(m)
    assert ms[0] != ms[1] and ms[1] == ms[2]
    pre, used = _stats(qlib, gpu)
    assert pre == 2 and used == 1, (pre, used)  # the second call's guess was the first call's m


def test_pipeline_rejected_call_leaves_nothing_behind(qlib, gpu, oracle_mod):
    """An output buffer too small is refused after the estimate; the next call is still exact."""
    import torch

    n = 4096
    count = 1 << 18
    samples = W.adc_samples(count, 631)
    samples_dev = torch.from_numpy(samples).cuda()
    seed = W.random_bits(2 * n - 1, 632)
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_postprocess(gpu, samples_dev, count, 8, 1e-6, 1.0, n, seed_dev, 2 * n - 1, STD,
                              qlib.QRNG_ALGO_GEMM_KARATSUBA, small, small.numel())
    assert e.value.status == qlib.QRNG_EINVAL
    m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
    _check(oracle_mod, qlib, samples, n, seed, STD, m, nb, rep, out)


@pytest.mark.parametrize("algo_name", ["DIRECT", "NTT", "GEMM_FP4_PAIR", "AUTO"])
def test_pipeline_other_routes_match_oracle(qlib, gpu, oracle_mod, algo_name):
    """Every route through the device pipeline, small shapes compared bit for bit."""
    import torch

    algo = getattr(qlib, "QRNG_ALGO_" + algo_name)
    n = 2048
    count = 200_000
    samples = W.adc_samples(count, 641)
    seed = W.random_bits(2 * n - 1, 642)
    samples_dev = torch.from_numpy(samples).cuda()
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD, algo, out)
        _check(oracle_mod, qlib, samples, n, seed, STD, m, nb, rep, out)


def test_host_pipeline_presplit(qlib, gpu, oracle_mod):
    """The host-buffer pipeline runs the same first half: its second call on a shape finds the
    derived operands of its first (7/8) part computed beside the estimate."""
    n = 1 << 16
    count = 1 << 22
    samples = W.adc_samples(count, 651)
    seed = W.random_bits(2 * n - 1, 652)
    out = np.zeros(count, dtype=np.uint8)
    qlib.qrng_reset_stats(gpu)
    for _ in range(2):
        m, nb, rep = qlib.qrng_postprocess_host(gpu, samples, count, 8, 1e-6, 1.0, n, seed, 2 * n - 1, STD,
                                               qlib.QRNG_ALGO_GEMM_KARATSUBA, out, out.size)
        raw = samples.view(np.uint8)
        assert not oracle_mod.freivalds(raw, n, m, seed, STD, nb, out[:(nb * m + 7) // 8]).any()
    pre, used = _stats(qlib, gpu)
    assert pre == 1 and used == 1, (pre, used)


def test_host_async_pipeline_overlapping_calls(qlib, gpu, oracle_mod):
    """Calls of the overlapped host pipeline submitted back to back (the device buffers alternate
    between two slots, each call's upload and download beside another call's hash), with new sample
    contents every call, a larger shape half-way (the slots' buffers grow) and a rejected call in
    between: after the wait every output equals the oracle's."""
    import torch

    calls = [(1 << 20, 1 << 16, 701), (1 << 20, 1 << 16, 702), (1 << 20, 1 << 16, 703),
             (1 << 21, 1 << 16, 704), (1 << 21, 1 << 16, 705), (3 << 18, 4096, 706)]
    seed = W.random_bits(2 * (1 << 16) - 1, 707)
    pin_seed = torch.from_numpy(seed).pin_memory()
    done = []
    for i, (count, n, sseed) in enumerate(calls):
        samples = W.adc_samples(count, sseed)
        pin_samples = torch.from_numpy(samples).pin_memory()
        pin_out = torch.zeros(count, dtype=torch.uint8).pin_memory()
        if i == 2:  # a call whose output buffer is too small is refused; the stream of calls goes on
            small = torch.zeros(8, dtype=torch.uint8).pin_memory()
            with pytest.raises(qlib.QrngError) as e:
                qlib.qrng_postprocess_host_async(gpu, pin_samples, count, 8, 1e-6, 1.0, n, pin_seed, 2 * n - 1,
                                                 STD, qlib.QRNG_ALGO_AUTO, small, small.numel())
            assert e.value.status == qlib.QRNG_EINVAL
        m, nb, rep = qlib.qrng_postprocess_host_async(gpu, pin_samples, count, 8, 1e-6, 1.0, n, pin_seed,
                                                      2 * n - 1, STD, qlib.QRNG_ALGO_AUTO, pin_out, pin_out.numel())
        done.append((samples, pin_samples, pin_out, n, m, nb, rep))
    qlib.qrng_postprocess_host_wait(gpu)
    for samples, _, pin_out, n, m, nb, rep in done:
        ref = oracle_mod.minentropy(samples, 8, 1e-6)
        assert abs(rep["h_modify"] - ref["h_modify"]) < 1e-12
        assert m == oracle_mod.output_length(n, ref["h_modify"], 8, 1.0) and nb == samples.size * 8 // n
        got = pin_out.numpy()[:(nb * m + 7) // 8]
        raw = samples.view(np.uint8)
        seed_n = seed[:(n + m - 1 + 7) // 8]
        if n * m * nb <= 1 << 30:
            assert np.array_equal(got, oracle_mod.toeplitz_blocks(raw, n, m, seed_n, STD, nb))
        else:
            assert not oracle_mod.freivalds(raw, n, m, seed_n, STD, nb, got).any()


def _spec_stats(q, ctx):
    s = q.qrng_get_stats(ctx)
    return s["speculative_hashes"], s["speculative_misses"]


def test_speculative_hash_hits_and_misses(qlib, gpu, oracle_mod):
    """The hash enqueued before the host reads m: a call whose m is within the previous call's rows
    (rounded up to the plan's row span) keeps it; a call whose m is above them hashes again with m;
    a call with a much smaller m keeps the larger launch (its extra rows are not written). Every
    output equals the oracle's."""
    import torch

    n = 1 << 16
    count = 5 << 19  # 320 blocks
    qlib.qrng_set_karatsuba(gpu, 4, 256, 0)  # row span 256 << 4 = 4096
    try:
        seed = W.random_bits(2 * n - 1, 661)
        seed_dev = torch.from_numpy(seed).cuda()
        out = torch.zeros(count, dtype=torch.uint8, device="cuda")
        samples_dev = torch.empty(count, dtype=torch.uint8, device="cuda")
        qlib.qrng_reset_stats(gpu)
        ms, expect_miss = [], 0
        for i, (sseed, sigma) in enumerate(((662, 4.0), (663, 4.0), (664, 32.0), (665, 32.0), (666, 6.0))):
            samples = W.adc_samples(count, sseed, sigma=sigma)
            samples_dev.copy_(torch.from_numpy(samples))
            out.zero_()
            m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD,
                              qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
            _check(oracle_mod, qlib, samples, n, seed, STD, m, nb, rep, out, full=False)
            # nothing past the call's bytes is written
            assert not out[(nb * m + 7) // 8:].any()
            if i:
                cap = min(n, -(-ms[-1] // 4096) * 4096)
                expect_miss += int(m > cap)
            ms.append(m)
        hashes, misses = _spec_stats(qlib, gpu)
        assert hashes == 4 and misses == expect_miss, (ms, hashes, misses)
        assert expect_miss == 1, ms  # sigma 4 -> 32 raises m by far more than one row span
    finally:
        qlib.qrng_set_karatsuba(gpu, 0, 0, 0)


@pytest.mark.parametrize("eps_lhl", [1.0, 0.5, 1e-6, 2.0 ** -40, 3e-13])
def test_speculative_m_matches_host_arithmetic(qlib, gpu, oracle_mod, eps_lhl):
    """m computed on the device from the report equals the host's qrng_output_length for several
    leftover-hash terms (a disagreement would count as a miss and hash again)."""
    import torch

    n = 1 << 15
    count = 3 << 19  # 384 blocks
    seed = W.random_bits(2 * n - 1, 671)
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    samples = W.adc_samples(count, 672, sigma=12.0)
    samples_dev = torch.from_numpy(samples).cuda()
    qlib.qrng_reset_stats(gpu)
    for _ in range(3):
        m, nb, rep = _run(qlib, gpu, samples_dev, count, n, seed_dev, 2 * n - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA,
                          out, eps_lhl=eps_lhl)
        assert m == qlib.qrng_output_length(n, rep["h_modify"], 8, eps_lhl)
        raw = samples.view(np.uint8)
        assert not oracle_mod.freivalds(raw, n, m, seed, STD, nb, out[:(nb * m + 7) // 8].cpu().numpy()).any()
    hashes, misses = _spec_stats(qlib, gpu)
    assert hashes >= 2 and misses == 0, (hashes, misses)


def test_speculative_hash_tight_seed_and_refusals(qlib, gpu, oracle_mod):
    """A seed of exactly n + m - 1 bits caps the enqueued rows at m. Refused speculative calls
    write nothing: one whose output buffer is too small, one whose samples give a larger m than the
    seed covers. The calls after them are exact again (the first one on the ordinary path, as the
    refused call's m is beyond the seed)."""
    import torch

    n = 1 << 14
    count = 1 << 20  # 512 blocks
    s1 = W.adc_samples(count, 681, sigma=8.0)
    m1 = oracle_mod.output_length(n, oracle_mod.minentropy(s1, 8, 1e-6)["h_modify"], 8, 1.0)
    seed = W.random_bits(n + m1 - 1, 682)
    seed_dev = torch.from_numpy(seed).cuda()
    out = torch.zeros(count, dtype=torch.uint8, device="cuda")
    d1 = torch.from_numpy(s1).cuda()
    qlib.qrng_reset_stats(gpu)
    for _ in range(2):
        m, nb, rep = _run(qlib, gpu, d1, count, n, seed_dev, n + m1 - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
        assert m == m1
        _check(oracle_mod, qlib, s1, n, seed, STD, m, nb, rep, out, full=False)
    small = torch.full((64,), 0x5A, dtype=torch.uint8, device="cuda")
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_postprocess(gpu, d1, count, 8, 1e-6, 1.0, n, seed_dev, n + m1 - 1, STD,
                              qlib.QRNG_ALGO_GEMM_KARATSUBA, small, small.numel())
    assert e.value.status == qlib.QRNG_EINVAL
    qlib.qrng_synchronize(gpu)
    assert bool((small == 0x5A).all())
    s2 = W.adc_samples(count, 683, sigma=40.0)  # larger m: the seed is too short for it
    d2 = torch.from_numpy(s2).cuda()
    out.fill_(0xA5)
    with pytest.raises(qlib.QrngError) as e:
        _run(qlib, gpu, d2, count, n, seed_dev, n + m1 - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
    assert e.value.status == qlib.QRNG_EINVAL
    qlib.qrng_synchronize(gpu)
    assert bool((out == 0xA5).all())
    for full in (True, False):
        out.zero_()
        m, nb, rep = _run(qlib, gpu, d1, count, n, seed_dev, n + m1 - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, out)
        _check(oracle_mod, qlib, s1, n, seed, STD, m, nb, rep, out, full=full)
    hashes, misses = _spec_stats(qlib, gpu)
    assert hashes == 4 and misses == 0, (hashes, misses)


def test_host_async_speculative_calls(qlib, gpu, oracle_mod):
    """The overlapped host pipeline enqueues the hash before reading m as qrng_postprocess does:
    calls of one shape submitted back to back, new contents every call, one call whose m is above
    the previous call's rows (hashed again with m), all outputs equal to the oracle's."""
    import torch

    n = 1 << 16
    count = 3 << 19  # 192 blocks
    qlib.qrng_set_karatsuba(gpu, 4, 256, 0)  # row span 4096
    try:
        seed = W.random_bits(2 * n - 1, 711)
        pin_seed = torch.from_numpy(seed).pin_memory()
        qlib.qrng_reset_stats(gpu)
        done = []
        for sseed, sigma in ((712, 6.0), (713, 6.0), (714, 30.0), (715, 30.0)):
            samples = W.adc_samples(count, sseed, sigma=sigma)
            pin_samples = torch.from_numpy(samples).pin_memory()
            pin_out = torch.zeros(count, dtype=torch.uint8).pin_memory()
            m, nb, rep = qlib.qrng_postprocess_host_async(gpu, pin_samples, count, 8, 1e-6, 1.0, n, pin_seed,
                                                          2 * n - 1, STD, qlib.QRNG_ALGO_GEMM_KARATSUBA, pin_out,
                                                          pin_out.numel())
            done.append((samples, pin_samples, pin_out, m, nb, rep))
        qlib.qrng_postprocess_host_wait(gpu)
        ms = []
        for samples, _, pin_out, m, nb, rep in done:
            ref = oracle_mod.minentropy(samples, 8, 1e-6)
            assert abs(rep["h_modify"] - ref["h_modify"]) < 1e-12
            assert m == oracle_mod.output_length(n, ref["h_modify"], 8, 1.0)
            got = pin_out.numpy()
            assert not oracle_mod.freivalds(samples.view(np.uint8), n, m, seed, STD, nb, got[:(nb * m + 7) // 8]).any()
            assert not got[(nb * m + 7) // 8:].any()
            ms.append(m)
        expect_miss = sum(int(ms[i] > min(n, -(-ms[i - 1] // 4096) * 4096)) for i in range(1, len(ms)))
        s = qlib.qrng_get_stats(gpu)
        assert s["speculative_hashes"] == 3 and s["speculative_misses"] == expect_miss == 1, (ms, s)
    finally:
        qlib.qrng_set_karatsuba(gpu, 0, 0, 0)
