"""The block-length sweep at full size, every algorithm against the oracle (Sec. III.E block
processing, Sec. III.D modified Toeplitz).

A fixed 2^30-bit Bernoulli(0.5) stream is cut into blocks of n = 2^10 .. 2^24 bits, m = 0.75 n,
one (n-1)-bit seed per n. Every algorithm the sweep times hashes the whole stream, and its output
is compared with the oracle on EVERY block: with the oracle's Freivalds check (64 random parity
tests per block, escape probability 2^-64) where its O(nm) preparation is affordable
(n m <= 2^31), otherwise on sampled output bits of every block, each computed by the oracle on its
own. The bytes around the output must stay untouched. Bar: bit-exact.
"""
import concurrent.futures

import numpy as np
import pytest

import workloads as W
from gpu_util import check_every_block

pytestmark = pytest.mark.gpu

MOD = 1
ALGOS = {"direct": 1, "gemm_tc": 2, "fft64": 3, "fft32_seg": 4, "ntt": 5, "gemm_fp4": 6, "gemm_fp4_pair": 7,
         "gemm_karatsuba": 8, "auto": 0}
SENTINEL = 0xC3


@pytest.fixture(scope="module")
def stream():
    import torch

    c = W.CFG3
    raw = W.random_bits(c["stream_bits"], c["raw_seed"])
    return raw, torch.from_numpy(raw).to("cuda")


@pytest.mark.parametrize("log2n", list(range(10, 25)))
def test_every_algorithm_every_block(qlib, gpu, oracle_mod, stream, log2n):
    import torch

    c = W.CFG3
    raw, raw_d = stream
    n = 1 << log2n
    m = int(n * c["ratio"])
    B = c["stream_bits"] // n
    seed = W.random_bits(n - 1, c["seed_seed"] + log2n)
    seed_d = torch.from_numpy(seed).to("cuda")
    nbytes = B * m // 8
    out = torch.full((nbytes + 64,), SENTINEL, dtype=torch.uint8, device="cuda")
    outs = {}
    for name, algo in ALGOS.items():
        out.fill_(SENTINEL)
        qlib.qrng_toeplitz_extract(gpu, raw_d, n, m, seed_d, MOD, algo, B, out)
        qlib.qrng_synchronize(gpu)
        host = out.cpu().numpy()
        assert np.all(host[nbytes:] == SENTINEL), f"{name}: wrote past the output"
        outs[name] = host[:nbytes].copy()

    def check(name):
        got = outs[name]
        if n * m <= (1 << 31):
            mism = oracle_mod.freivalds(raw, n, m, seed, MOD, B, got, rng_seed=log2n)
            assert not mism.any(), f"{name}: {np.count_nonzero(mism)} of {B} blocks fail the Freivalds check"
            return "freivalds"
        per_block = 8 if n <= (1 << 20) else 6
        check_every_block(oracle_mod, raw, n, m, seed, MOD, got, B, per_block=per_block,
                          rng_seed=1000 * log2n + ALGOS[name])
        return f"{per_block} bits x {B} blocks"

    if n * m <= (1 << 31):  # one Freivalds call per algorithm, side by side (each is single-threaded C)
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(outs)) as ex:
            checked = dict(zip(outs, ex.map(check, outs)))
    else:  # each check spreads over the cores itself
        checked = {name: check(name) for name in outs}
    assert len(checked) == len(ALGOS)
