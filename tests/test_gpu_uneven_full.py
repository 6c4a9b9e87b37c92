"""The uneven batch at full size against the oracle (Sec. III.B per request, Sec. III.E
independent blocks): 10,000 requests, n log-uniform in [2^12, 2^22], m = floor(rho n) with rho
uniform in [0.5, 0.9], every request with its own seed and Bernoulli(p) raw bits, p uniform in
[0.45, 0.55].

Every route the batch entry point offers hashes the whole batch, and every request's output is
checked against the oracle on sampled bits (its first and last bits and random ones, each
computed by the oracle on its own in O(n)). Bar: bit-exact, and no bit outside the requests'
outputs written.
"""
import concurrent.futures

import numpy as np
import pytest

import workloads as W
from gpu_util import host_threads

pytestmark = pytest.mark.gpu

STD = 0
SENTINEL = 0x96


@pytest.fixture(scope="module")
def batch(qlib):
    import torch

    b = W.uneven_batch()
    raw_d = torch.from_numpy(b["raw"]).to("cuda")
    seeds_d = torch.from_numpy(b["seeds"]).to("cuda")
    nbytes = (b["out_bits"] + 7) // 8
    out = torch.full((nbytes + 64,), SENTINEL, dtype=torch.uint8, device="cuda")
    reqs = [(raw_d.data_ptr(), int(b["raw_off"][i]), int(b["n"][i]), int(b["m"][i]),
             seeds_d.data_ptr() + int(b["seed_off"][i]), STD, out.data_ptr(), int(b["out_off"][i]))
            for i in range(b["n"].size)]
    return b, (raw_d, seeds_d), out, reqs


def _check_requests(oracle_mod, b, host, per_req, rng_seed):
    bits = np.unpackbits(host, bitorder="little")
    n, m = b["n"], b["m"]
    g = W.rng(rng_seed)
    rnd = g.integers(0, 1 << 62, size=(n.size, per_req), dtype=np.int64)

    def run(i0, i1):
        for i in range(i0, i1):
            mi, ni = int(m[i]), int(n[i])
            idx = np.unique(np.concatenate([np.arange(min(4, mi)), np.arange(max(0, mi - 4), mi), rnd[i] % mi]))
            seed = b["seeds"][b["seed_off"][i]:b["seed_off"][i] + b["seed_len"][i]]
            want = oracle_mod.toeplitz_bits(b["raw"], ni, mi, seed, STD, idx.astype(np.uint64),
                                            raw_off=int(b["raw_off"][i]))
            got = bits[int(b["out_off"][i]) + idx]
            if not np.array_equal(got, want):
                return i
        return None

    t = host_threads()
    step = max(1, -(-n.size // (8 * t)))
    with concurrent.futures.ThreadPoolExecutor(max_workers=t) as ex:
        for r in ex.map(lambda i0: run(i0, min(n.size, i0 + step)), range(0, n.size, step)):
            assert r is None, f"request {r} (n={n[r]}, m={m[r]}) differs from the oracle"


@pytest.mark.parametrize("route", ["auto", "ntt", "fft64", "fft32_seg", "direct"])
def test_full_uneven_batch_every_request(qlib, gpu, oracle_mod, batch, route):
    b, _keep, out, reqs = batch
    algo = {"auto": qlib.QRNG_ALGO_AUTO, "ntt": qlib.QRNG_ALGO_NTT, "fft64": qlib.QRNG_ALGO_FFT64,
            "fft32_seg": qlib.QRNG_ALGO_FFT32_SEG, "direct": qlib.QRNG_ALGO_DIRECT}[route]
    out.fill_(SENTINEL)
    qlib.qrng_reset_stats(gpu)
    qlib.qrng_extract_batch(gpu, reqs, algo=algo)
    qlib.qrng_synchronize(gpu)
    host = out.cpu().numpy()
    nbytes = (b["out_bits"] + 7) // 8
    assert np.all(host[nbytes:] == SENTINEL), "wrote past the batch output"
    tail = b["out_bits"] % 8
    if tail:  # pad bits of the last byte keep the sentinel's bits
        assert (host[nbytes - 1] >> tail) == (SENTINEL >> tail)
    _check_requests(oracle_mod, b, host[:nbytes], per_req=8, rng_seed=algo + 17)
    st = qlib.qrng_get_stats(gpu)
    assert sum(st["batch_requests"].values()) == b["n"].size
    if route in ("fft64", "fft32_seg"):
        assert 0.0 < st["worst_fft_round_err"] < 0.25
