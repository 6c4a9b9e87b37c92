"""GPU parity of qrng_extract_batch (uneven requests, one persistent launch in a cached CUDA graph)
against the oracle. Bar: bit-exact, and every bit outside the requests' output ranges untouched.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

STD, MOD = 0, 1


def _make_batch(count, seed, log2n_lo, log2n_hi, mixed_forms=True):
    """Requests over one shared raw buffer and one output buffer, packed at odd bit offsets."""
    n, m, p = W.uneven_requests(count, seed, log2n_lo, log2n_hi)
    g = W.rng(seed + 1)
    forms = g.integers(0, 2, count) if mixed_forms else np.zeros(count, dtype=np.int64)
    m = np.where((forms == MOD) & (m >= n), n - 1, m)
    raw_offs, seeds, out_offs = [], [], []
    pos = int(g.integers(0, 8))
    for i in range(count):
        raw_offs.append(pos)
        pos += int(n[i]) + int(g.integers(0, 40))
    raw_bits = pos + 64
    # Bernoulli(p_i) raw bits per request, written into one stream
    stream = np.zeros(raw_bits, dtype=np.uint8)
    for i in range(count):
        stream[raw_offs[i]:raw_offs[i] + n[i]] = W.unpack_bits(W.random_bits(int(n[i]), 100 + i, float(p[i])), int(n[i]))
    raw = W.pack_bits(stream)
    opos = int(g.integers(0, 8))
    for i in range(count):
        L = int(n[i] + m[i] - 1) if forms[i] == STD else int(n[i] - 1)
        seeds.append(W.random_bits(L, 5000 + i))
        out_offs.append(opos)
        opos += int(m[i]) + (int(g.integers(0, 3)) if i % 3 == 0 else 0)  # mostly back to back
    return n, m, forms, raw, raw_offs, seeds, out_offs, opos


def _run(qlib, ctx, batch, sentinel=0x5A, algo=0):
    import torch

    n, m, forms, raw, raw_offs, seeds, out_offs, out_bits = batch
    raw_t, raw_p = to_dev(raw)
    seed_t = [to_dev(s) for s in seeds]
    nbytes = (out_bits + 7) // 8 + 8
    out = torch.full((nbytes,), sentinel, dtype=torch.uint8, device="cuda")
    reqs = [(raw_p, raw_offs[i], int(n[i]), int(m[i]), seed_t[i][1], int(forms[i]), out.data_ptr(), out_offs[i])
            for i in range(len(n))]
    qlib.qrng_extract_batch(ctx, reqs, algo=algo)
    qlib.qrng_synchronize(ctx)
    return out.cpu().numpy(), (raw_t, seed_t, out, reqs)


def _check(oracle_mod, batch, host, sentinel=0x5A, full_upto=1 << 14):
    n, m, forms, raw, raw_offs, seeds, out_offs, out_bits = batch
    got = np.unpackbits(host, bitorder="little")
    covered = np.zeros(got.size, dtype=bool)
    for i in range(len(n)):
        o = out_offs[i]
        covered[o:o + m[i]] = True
        k = got[o:o + m[i]]
        if n[i] <= full_upto:
            want = W.unpack_bits(oracle_mod.toeplitz(raw, int(n[i]), int(m[i]), seeds[i], int(forms[i]),
                                                     raw_off=raw_offs[i]), int(m[i]))
            assert np.array_equal(k, want), f"request {i} (n={n[i]}, m={m[i]}, form={forms[i]})"
        else:
            idx = np.unique(np.concatenate([np.arange(32), np.arange(m[i] - 32, m[i]),
                                            W.rng(i).integers(0, m[i], 96)])).astype(np.uint64)
            want = oracle_mod.toeplitz_bits(raw, int(n[i]), int(m[i]), seeds[i], int(forms[i]), idx,
                                            raw_off=raw_offs[i])
            assert np.array_equal(k[idx.astype(np.int64)], want), f"request {i} (n={n[i]}, m={m[i]})"
    sent = np.unpackbits(np.full(host.size, sentinel, dtype=np.uint8), bitorder="little")
    assert np.array_equal(got[~covered], sent[~covered]), "bits outside the requests changed"


def test_uneven_small_requests_bit_exact(qlib, gpu, oracle_mod):
    batch = _make_batch(80, 11, 5, 13)
    host, _ = _run(qlib, gpu, batch)
    _check(oracle_mod, batch, host)


def test_uneven_requests_log_uniform(qlib, gpu, oracle_mod):
    """The uneven-request shape (n log-uniform, m/n uniform in [0.5, 0.9], p uniform in
    [0.45, 0.55]) on a reduced n range the oracle checks quickly."""
    batch = _make_batch(300, 9, 12, 17)
    host, _ = _run(qlib, gpu, batch)
    _check(oracle_mod, batch, host)


def test_all_requests_on_the_transform_route(qlib, gpu, oracle_mod):
    """QRNG_ALGO_NTT sends every request through the batched number-theoretic transform."""
    batch = _make_batch(60, 13, 5, 14)
    host, _ = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_NTT)
    _check(oracle_mod, batch, host)
    assert qlib.qrng_get_stats(gpu)["last_algo"] == qlib.QRNG_ALGO_NTT


def test_all_requests_on_the_fp64_route(qlib, gpu, oracle_mod):
    """QRNG_ALGO_FFT64: seed and raw bits of a request in one complex vector, two requests per
    inverse transform; exact after rounding, with the rounding distance reported."""
    batch = _make_batch(61, 15, 5, 15)  # odd count: the last pair has one request
    qlib.qrng_reset_stats(gpu)
    host, _ = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_FFT64)
    _check(oracle_mod, batch, host)
    st = qlib.qrng_get_stats(gpu)
    assert st["last_algo"] == qlib.QRNG_ALGO_FFT64 and st["worst_fft_round_err"] < 1e-6


def test_all_requests_on_the_fp32_segmented_route(qlib, gpu, oracle_mod):
    """QRNG_ALGO_FFT32_SEG: every request's seed windows and raw segments transformed once, the
    products summed in the frequency domain up to the proven term count, parities XORed."""
    batch = _make_batch(70, 23, 5, 17)
    qlib.qrng_reset_stats(gpu)
    host, _ = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_FFT32_SEG)
    _check(oracle_mod, batch, host)
    st = qlib.qrng_get_stats(gpu)
    assert st["last_algo"] == qlib.QRNG_ALGO_FFT32_SEG and st["worst_fft_round_err"] < 0.25
    assert st["batch_requests"]["fft32_seg"] == 70


@pytest.mark.parametrize("seg", [2048, 8192])
def test_fp32_segmented_route_other_segment_lengths(qlib, gpu, oracle_mod, seg):
    batch = _make_batch(25, 25 + seg, 10, 16)
    qlib.qrng_set_fft32(gpu, seg, 0)
    try:
        host, _ = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_FFT32_SEG)
    finally:
        qlib.qrng_set_fft32(gpu, 0, 0)
    _check(oracle_mod, batch, host)


def test_auto_is_one_graph_replay_per_call(qlib, gpu, oracle_mod):
    """AUTO routes each shape class (transform length) by timing its candidates once; then every
    call of the same table is a single replay of the cached graph, whatever the routes."""
    batch = _make_batch(150, 29, 8, 21)
    host, keep = _run(qlib, gpu, batch)
    _check(oracle_mod, batch, host)
    st1 = qlib.qrng_get_stats(gpu)
    routes = st1["batch_requests"]
    assert sum(routes.values()) == 150
    k0 = st1["kernels_launched"]
    raw_t, seed_t, out, reqs = keep
    out.fill_(0x5A)
    qlib.qrng_extract_batch(gpu, reqs)
    qlib.qrng_synchronize(gpu)
    st2 = qlib.qrng_get_stats(gpu)
    assert st2["batch_requests"] == routes
    assert st2["kernels_launched"] - k0 == st2["last_kernels"]  # one replay, no tuning
    _check(oracle_mod, batch, out.cpu().numpy())


def test_mixed_routes_long_requests(qlib, gpu, oracle_mod):
    """AUTO on requests up to 2^20 bits: short ones on the persistent kernel, long ones on the
    transform route, all merged into one output buffer."""
    batch = _make_batch(120, 17, 10, 20)
    host, _ = _run(qlib, gpu, batch)
    _check(oracle_mod, batch, host)
    direct = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_DIRECT)[0]
    assert np.array_equal(host, direct)


def test_transform_route_length_2_25(qlib, gpu, oracle_mod):
    """One request long enough for a 2^25-point transform (the route without the fused bit input and
    parity output) among short ones, all forced onto the transform route."""
    shapes = [(1 << 24, 100, STD), (5000, 3000, MOD), (70000, 40000, STD)]
    n = np.array([x[0] for x in shapes])
    m = np.array([x[1] for x in shapes])
    forms = np.array([x[2] for x in shapes])
    raw_offs, pos = [], 5
    for i in range(len(shapes)):
        raw_offs.append(pos)
        pos += int(n[i]) + 11
    raw = W.random_bits(pos + 64, 81)
    seeds = [W.random_bits(int(n[i] + m[i] - 1) if forms[i] == STD else int(n[i] - 1), 90 + i)
             for i in range(len(shapes))]
    out_offs = [3, 3 + int(m[0]), 3 + int(m[0] + m[1])]
    batch = (n, m, forms, raw, raw_offs, seeds, out_offs, int(3 + m.sum()))
    host, _ = _run(qlib, gpu, batch, algo=qlib.QRNG_ALGO_NTT)
    _check(oracle_mod, batch, host)


def test_graph_replay_sees_new_data(qlib, gpu, oracle_mod):
    """An identical request table replays the cached graph; the kernels read the buffers anew."""
    import torch

    batch = _make_batch(40, 21, 6, 12)
    host1, keep = _run(qlib, gpu, batch)
    _check(oracle_mod, batch, host1)
    raw_t, seed_t, out, reqs = keep
    new_raw = W.random_bits(len(batch[3]) * 8, 777)
    raw_t[:new_raw.size] = torch.from_numpy(new_raw).to("cuda")
    out.fill_(0x5A)
    qlib.qrng_extract_batch(gpu, reqs)
    qlib.qrng_synchronize(gpu)
    batch2 = batch[:3] + (new_raw,) + batch[4:]
    _check(oracle_mod, batch2, out.cpu().numpy())


def test_batch_matches_single_block_calls(qlib, gpu):
    """One request per block of a shared-seed stream equals the stream call."""
    import torch

    n, m, B = 4096, 3000, 24
    raw = W.random_bits(n * B, 3)
    seed = W.random_bits(n + m - 1, 4)
    raw_t, raw_p = to_dev(raw)
    seed_t, seed_p = to_dev(seed)
    ref = torch.zeros((m * B + 7) // 8, dtype=torch.uint8, device="cuda")
    qlib.qrng_toeplitz_extract(gpu, raw_p, n, m, seed_p, STD, qlib.QRNG_ALGO_DIRECT, B, ref)
    out = torch.zeros_like(ref)
    qlib.qrng_extract_batch(gpu, [(raw_p, b * n, n, m, seed_p, STD, out.data_ptr(), b * m) for b in range(B)])
    qlib.qrng_synchronize(gpu)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("algo", [0, 1, 5, 3, 4])
def test_single_and_degenerate_requests(qlib, gpu, oracle_mod, algo):
    """One-bit outputs, n = 1 and n = 2 blocks, m = n standard, m = n - 1 modified, on every route."""
    shapes = [(1, 1, STD), (2, 1, MOD), (2, 2, STD), (33, 1, STD), (64, 63, MOD), (100, 100, STD)]
    n = np.array([s[0] for s in shapes])
    m = np.array([s[1] for s in shapes])
    forms = np.array([s[2] for s in shapes])
    raw_offs, pos = [], 3
    for i in range(len(shapes)):
        raw_offs.append(pos)
        pos += int(n[i]) + 5
    raw = W.random_bits(pos + 64, 8)
    seeds = [W.random_bits(int(n[i] + m[i] - 1) if forms[i] == STD else int(n[i] - 1) or 1, 40 + i)
             for i in range(len(shapes))]
    out_offs = list(np.concatenate([[1], 1 + np.cumsum(m)[:-1]]))
    batch = (n, m, forms, raw, raw_offs, seeds, [int(x) for x in out_offs], int(1 + m.sum()))
    host, _ = _run(qlib, gpu, batch, algo=algo)
    _check(oracle_mod, batch, host)


def test_batch_bad_arguments(qlib, gpu):
    import torch

    t = torch.zeros(64, dtype=torch.uint8, device="cuda")
    ok = (t, 0, 64, 32, t, STD, t, 0)
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_extract_batch(gpu, [ok], algo=qlib.QRNG_ALGO_GEMM_TC)
    assert e.value.status == qlib.QRNG_ENOTSUP
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_extract_batch(gpu, [ok, (t, 0, 64, 64, t, MOD, t, 0)])
    assert e.value.status == qlib.QRNG_EINVAL
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_extract_batch(gpu, [(0, 0, 64, 32, t, STD, t, 0)])
    assert e.value.status == qlib.QRNG_EINVAL
