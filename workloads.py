"""Seeded synthetic inputs for the QRNG post-processing workloads.

This module only draws random numbers and packs bits; it holds none of the method's
arithmetic. Both the tests (oracle and CUDA sides) and the benchmark take their inputs from
here, so the two sides always see byte-identical data.

The paper's own inputs (a 10-Gbit laser-phase-noise stream and its seeds, Sec. III.E) are not
available; these generators stand in for them with the shapes and distributions the paper
describes: ADC samples of a Gaussian noise source (Sec. II.B), Bernoulli raw bits, uniform
random seeds, and independent n-bit blocks of one long stream (Sec. III.E).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def adc_samples(count: int, seed: int, mu: float = 128.0, sigma: float = 16.0, bits: int = 8) -> np.ndarray:
    """ADC codes of a Gaussian source: clip(round(N(mu, sigma^2)), 0, 2^bits - 1)."""
    g = rng(seed)
    out = np.empty(count, dtype=np.uint8 if bits <= 8 else np.uint16)
    hi = (1 << bits) - 1
    chunk = 1 << 24
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        x = np.rint(g.normal(mu, sigma, e - s))
        np.clip(x, 0, hi, out=x)
        out[s:e] = x.astype(out.dtype)
    return out


def random_bits(nbits: int, seed: int, p: float = 0.5) -> np.ndarray:
    """nbits Bernoulli(p) bits packed LSB-first into ceil(nbits/8) bytes; pad bits are zero
    (p is resolved to a multiple of 2^-16)."""
    g = rng(seed)
    nbytes = (nbits + 7) // 8
    if p == 0.5:
        out = g.integers(0, 256, size=nbytes, dtype=np.uint8)
    else:
        # P(bit = 1) = round(p * 2^16) / 2^16
        thr = int(round(p * 65536))
        out = np.empty(nbytes, dtype=np.uint8)
        chunk = 1 << 26
        for s in range(0, nbits, chunk):
            e = min(nbits, s + chunk)
            out[s // 8:(e + 7) // 8] = np.packbits(g.integers(0, 65536, e - s, dtype=np.uint16) < thr,
                                                   bitorder="little")
    if nbits % 8:
        out[-1] &= (1 << (nbits % 8)) - 1
    return out


def unpack_bits(buf: np.ndarray, nbits: int, off: int = 0) -> np.ndarray:
    """Bits [off, off+nbits) of an LSB-first packed buffer as a uint8 0/1 array."""
    return np.unpackbits(buf, bitorder="little")[off:off + nbits]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    return np.packbits(np.asarray(bits, dtype=np.uint8), bitorder="little")


def attack_voltages(count: int, seed: int, alpha0: float = 1.0, alpha_e: float = 0.99, beta_e: float = 2.0,
                    i_max: float = 5.0):
    """The photodiode-gain attack of Sec. II.B: intensity I ~ N(0,1), honest V = alpha0 I,
    attacked V' = alpha(I) I with alpha(I) = alpha_e (1 - I / (beta_e I_max))."""
    i = rng(seed).normal(0.0, 1.0, count)
    return alpha0 * i, alpha_e * (1.0 - i / (beta_e * i_max)) * i


def adc_quantise(v: np.ndarray, bits: int, lo: float, hi: float) -> np.ndarray:
    """Uniform ADC: 2^bits equal cells on [lo, hi], values outside clip to the end codes."""
    k = 1 << bits
    code = np.floor((v - lo) / (hi - lo) * k)
    return np.clip(code, 0, k - 1).astype(np.uint8 if bits <= 8 else np.uint16)


# ---------------------------------------------------------------------------------------------
# The five workloads (sizes and seeds fixed here).
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    description: str


CFG1 = dict(samples=65536, sample_seed=1, n=4096, m=2048, raw_seed=11, seed_seed=2, eps=1e-6)
CFG2 = dict(samples=1 << 26, sample_seed=3, n=1 << 16, seed_seed=4, eps=1e-6)
CFG3 = dict(stream_bits=1 << 30, raw_seed=5, seed_seed=6, n_list=[1 << k for k in range(10, 25)], ratio=0.75)
CFG4 = dict(m=6144, n=8192, blocks=4096, seed_seed=7, raw_seed=8)
CFG5 = dict(requests=10000, seed=9, log2n_lo=12, log2n_hi=22, rho_lo=0.5, rho_hi=0.9, p_lo=0.45, p_hi=0.55)


def uneven_requests(count: int, seed: int, log2n_lo: float = 12, log2n_hi: float = 22, rho_lo: float = 0.5,
                    rho_hi: float = 0.9, p_lo: float = 0.45, p_hi: float = 0.55):
    """Request shapes for the uneven batch: n log-uniform, m = floor(rho n) with rho uniform
    (clamped to [1, n-1]), and the Bernoulli parameter p of each request's raw bits."""
    g = rng(seed)
    n = np.floor(2.0 ** g.uniform(log2n_lo, log2n_hi, count)).astype(np.int64)
    rho = g.uniform(rho_lo, rho_hi, count)
    m = np.clip(np.floor(rho * n).astype(np.int64), 1, n - 1)
    p = g.uniform(p_lo, p_hi, count)
    return n, m, p


def uneven_batch(c: dict = CFG5, log2n_hi: float | None = None):
    """Host data of the uneven batch: request shapes from `uneven_requests`, every request's raw
    bits Bernoulli(p_r) at a 32-bit aligned offset of one stream, its own uniform seed of n+m-1
    bits at a byte offset of one seed buffer, and its m output bits back to back in one output
    stream. Returns a dict of the shapes (n, m, p), the offsets (raw_off and out_off in bits,
    seed_off in bytes) and the packed raw and seed buffers."""
    n, m, p = uneven_requests(c["requests"], c["seed"], c["log2n_lo"], c["log2n_hi"] if log2n_hi is None else log2n_hi,
                              c["rho_lo"], c["rho_hi"], c["p_lo"], c["p_hi"])
    raw_off = np.concatenate([[0], np.cumsum(((n + 31) // 32) * 32)[:-1]]).astype(np.int64)
    raw = np.zeros(int(raw_off[-1] + n[-1] + 64 + 7) // 8, dtype=np.uint8)
    for i in range(n.size):
        bits = random_bits(int(n[i]), 10_000 + i, float(p[i]))
        raw[raw_off[i] // 8:raw_off[i] // 8 + bits.size] = bits
    seed_len = (n + m - 1 + 7) // 8
    seed_off = np.concatenate([[0], np.cumsum(seed_len)[:-1]]).astype(np.int64)
    seeds = rng(c["seed"] + 7).integers(0, 256, int(seed_off[-1] + seed_len[-1]), dtype=np.uint8)
    out_off = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
    return dict(n=n, m=m, p=p, raw_off=raw_off, seed_off=seed_off, seed_len=seed_len, out_off=out_off, raw=raw,
                seeds=seeds, out_bits=int(out_off[-1] + m[-1]))
