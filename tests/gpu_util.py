"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and compare with the oracle."""
import numpy as np

import workloads as W


def to_dev(a: np.ndarray, offset: int = 0):
    """Copy a byte array to the GPU; with offset > 0 the returned address is that many bytes past
    a 256-byte aligned allocation (to exercise unaligned pointers)."""
    import torch

    buf = torch.zeros(a.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset:offset + a.size] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return buf, buf.data_ptr() + offset


def extract(q, ctx, raw: np.ndarray, n: int, m: int, seed: np.ndarray, form: int, algo: int, num_blocks: int,
            raw_off: int = 0, seed_off: int = 0, out_off: int = 0, sentinel: int = 0xA5):
    """Runs qrng_toeplitz_extract and returns the packed output bytes (and checks that the bytes
    past the output were not touched)."""
    import torch

    nbytes = (num_blocks * m + 7) // 8
    _keep_r, raw_p = to_dev(raw, raw_off)
    _keep_s, seed_p = to_dev(seed, seed_off)
    out = torch.full((nbytes + out_off + 64,), sentinel, dtype=torch.uint8, device="cuda")
    out_p = out.data_ptr() + out_off
    q.qrng_toeplitz_extract(ctx, raw_p, n, m, seed_p, form, algo, num_blocks, out_p)
    q.qrng_synchronize(ctx)  # raises if a kernel's bounded wait gave up
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    assert np.all(host[:out_off] == sentinel), "wrote before the output buffer"
    assert np.all(host[out_off + nbytes:] == sentinel), "wrote past the output buffer"
    return host[out_off:out_off + nbytes].copy()


def spot_check(oracle, raw, n, m, seed, form, out, blocks, per_block=256, rng_seed=0):
    """Exact oracle values of selected output bits (first/last 64 and random ones) of the given blocks."""
    g = W.rng(rng_seed)
    bits = np.unpackbits(out, bitorder="little")
    for b in blocks:
        idx = np.unique(np.concatenate([np.arange(min(64, m)), np.arange(max(0, m - 64), m),
                                        g.integers(0, m, per_block)])).astype(np.uint64)
        want = oracle.toeplitz_bits(raw, n, m, seed, form, idx, raw_off=b * n)
        got = bits[b * m + idx.astype(np.int64)]
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"block {b}: {bad.size} of {idx.size} sampled bits differ (first at k_{idx[bad[0]]})"


def host_threads() -> int:
    import os

    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def check_every_block(oracle, raw, n, m, seed, form, out, num_blocks, per_block=8, rng_seed=0, out_bit0=0,
                      raw_bit0=0, threads=None):
    """Exact oracle values of `per_block` output bits of EVERY block (the first and the last bit
    and random ones), each computed on its own in O(n), spread over the host's cores (the oracle
    is plain C called through ctypes, which releases the interpreter lock). Returns the number of
    bits checked; raises AssertionError naming the first block that differs."""
    import concurrent.futures

    g = W.rng(rng_seed)
    idx_all = g.integers(0, m, size=(num_blocks, max(0, per_block - 2)), dtype=np.int64)
    bits = np.unpackbits(out, bitorder="little")

    def run(b0, b1):
        for b in range(b0, b1):
            idx = np.unique(np.concatenate([[0, m - 1], idx_all[b]])).astype(np.uint64)
            want = oracle.toeplitz_bits(raw, n, m, seed, form, idx, raw_off=raw_bit0 + b * n)
            got = bits[out_bit0 + b * m + idx.astype(np.int64)]
            bad = np.nonzero(got != want)[0]
            if bad.size:
                return b, int(idx[bad[0]]), bad.size
        return None

    t = threads or host_threads()
    step = max(1, -(-num_blocks // (4 * t)))
    with concurrent.futures.ThreadPoolExecutor(max_workers=t) as ex:
        for r in ex.map(lambda b0: run(b0, min(num_blocks, b0 + step)), range(0, num_blocks, step)):
            assert r is None, f"block {r[0]}: {r[2]} sampled bits differ (first at k_{r[1]})"
    return num_blocks * per_block
