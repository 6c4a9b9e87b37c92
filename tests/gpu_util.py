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
