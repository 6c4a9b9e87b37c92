"""CPU oracle for QRNG post-processing: ctypes wrapper around ``qrng_oracle.c``.

TEST INFRASTRUCTURE ONLY. Imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``; the product package never imports it. It shares no code with
the CUDA path: the C file is compiled on its own with gcc and loaded here.

Functions follow the paper:
  * ``toeplitz`` / ``toeplitz_blocks`` / ``toeplitz_bits`` -- Sec. III.B (standard matrix T) and
    Sec. III.D (modified matrix (A, I_m)), computed from the definition;
  * ``freivalds`` -- a probabilistic whole-output check built from the same definition;
  * ``histogram`` / ``minentropy`` / ``minentropy_from_hist`` -- Sec. II (H_min, Gaussian model,
    statistical distance, correction term);
  * ``output_length`` -- Sec. III.B (leftover-hash sizing).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qrng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STANDARD = 0
MODIFIED = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation flags, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class HminReport(ctypes.Structure):
    _fields_ = [
        ("h_modify", ctypes.c_double),
        ("h_emp", ctypes.c_double),
        ("h_model", ctypes.c_double),
        ("d_u", ctypes.c_double),
        ("d_u_peak", ctypes.c_double),
        ("delta_fs", ctypes.c_double),
        ("delta_hm", ctypes.c_double),
        ("mean", ctypes.c_double),
        ("var", ctypes.c_double),
        ("count", ctypes.c_uint64),
        ("max_count", ctypes.c_uint64),
        ("argmax", ctypes.c_uint32),
        ("bits", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u64 = ctypes.c_uint64
            lib.oracle_toeplitz.argtypes = [u8p, u64, u64, u64, u8p, ctypes.c_int, u8p, u64]
            lib.oracle_toeplitz_blocks.argtypes = [u8p, u64, u64, u8p, ctypes.c_int, u64, u8p]
            lib.oracle_toeplitz_bits.argtypes = [u8p, u64, u64, u64, u8p, ctypes.c_int, u64p, u64, u8p]
            lib.oracle_freivalds.argtypes = [u8p, u64, u64, u8p, ctypes.c_int, u64, u8p, u64p, u64p]
            lib.oracle_histogram.argtypes = [ctypes.c_void_p, u64, ctypes.c_int, u64p, u64p]
            lib.oracle_minentropy_from_hist.argtypes = [u64p, ctypes.c_int, ctypes.c_double,
                                                        ctypes.POINTER(HminReport)]
            lib.oracle_minentropy.argtypes = [ctypes.c_void_p, u64, ctypes.c_int, ctypes.c_double,
                                              ctypes.POINTER(HminReport)]
            lib.oracle_minentropy_quantum_from_hist.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_double,
                                                                ctypes.POINTER(HminReport),
                                                                ctypes.POINTER(ctypes.c_double)]
            lib.oracle_splitmix64.argtypes = [u64, u64]
            lib.oracle_splitmix64.restype = u64
            lib.oracle_histogram_sampled.argtypes = [ctypes.c_void_p, u64, ctypes.c_int, ctypes.c_double, u64, u64p,
                                                     u64p]
            lib.oracle_output_length.argtypes = [u64, ctypes.c_double, ctypes.c_int, ctypes.c_double]
            lib.oracle_output_length.restype = u64
            lib.oracle_seed_bits.argtypes = [u64, u64, ctypes.c_int]
            lib.oracle_seed_bits.restype = u64
            _lib = lib
    return _lib


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(status: int, what: str):
    if status != 0:
        raise ValueError(f"oracle {what} failed with status {status}")


def seed_bits(n: int, m: int, form: int) -> int:
    return int(_load().oracle_seed_bits(n, m, form))


def toeplitz(raw: np.ndarray, n: int, m: int, seed: np.ndarray, form: int, raw_off: int = 0) -> np.ndarray:
    """One block: packed output (ceil(m/8) bytes, pad bits zero)."""
    out = np.zeros((m + 7) // 8, dtype=np.uint8)
    _check(_load().oracle_toeplitz(_u8(raw), raw_off, n, m, _u8(seed), form, _u8(out), 0), "toeplitz")
    return out


def toeplitz_blocks(raw: np.ndarray, n: int, m: int, seed: np.ndarray, form: int, num_blocks: int) -> np.ndarray:
    """Every block of a bit-contiguous stream; packed output of num_blocks*m bits."""
    out = np.zeros((num_blocks * m + 7) // 8, dtype=np.uint8)
    _check(_load().oracle_toeplitz_blocks(_u8(raw), n, m, _u8(seed), form, num_blocks, _u8(out)), "blocks")
    return out


def toeplitz_bits(raw: np.ndarray, n: int, m: int, seed: np.ndarray, form: int, idx, raw_off: int = 0) -> np.ndarray:
    """Selected output bits k_idx of the block starting at raw bit raw_off (uint8 0/1 per index)."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    bits = np.zeros(idx.size, dtype=np.uint8)
    _check(_load().oracle_toeplitz_bits(_u8(raw), raw_off, n, m, _u8(seed), form, _u64(idx), idx.size, _u8(bits)),
           "toeplitz_bits")
    return bits


def freivalds(raw: np.ndarray, n: int, m: int, seed: np.ndarray, form: int, num_blocks: int, out: np.ndarray,
              rng_seed: int = 1234) -> np.ndarray:
    """Per-block mismatch words (0 = block consistent with the definition under 64 random tests)."""
    u = np.random.Generator(np.random.PCG64(rng_seed)).integers(0, 2**64, size=m, dtype=np.uint64)
    mism = np.zeros(num_blocks, dtype=np.uint64)
    _check(_load().oracle_freivalds(_u8(raw), n, m, _u8(seed), form, num_blocks, _u8(out), _u64(u), _u64(mism)),
           "freivalds")
    return mism


def histogram(samples: np.ndarray, bits: int):
    """Exact histogram (uint64[2^bits]) and the number of samples >= 2^bits."""
    samples = np.ascontiguousarray(samples)
    assert samples.dtype == (np.uint8 if bits <= 8 else np.uint16)
    hist = np.zeros(1 << bits, dtype=np.uint64)
    bad = np.zeros(1, dtype=np.uint64)
    _check(_load().oracle_histogram(samples.ctypes.data, samples.size, bits, _u64(hist), _u64(bad)), "histogram")
    return hist, int(bad[0])


def minentropy_from_hist(hist: np.ndarray, bits: int, eps: float) -> dict:
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    rep = HminReport()
    _check(_load().oracle_minentropy_from_hist(_u64(hist), bits, eps, ctypes.byref(rep)), "minentropy_from_hist")
    return rep.as_dict()


def minentropy(samples: np.ndarray, bits: int, eps: float) -> dict:
    samples = np.ascontiguousarray(samples)
    assert samples.dtype == (np.uint8 if bits <= 8 else np.uint16)
    rep = HminReport()
    _check(_load().oracle_minentropy(samples.ctypes.data, samples.size, bits, eps, ctypes.byref(rep)), "minentropy")
    return rep.as_dict()


def output_length(n: int, h_per_sample: float, bits: int, eps_lhl: float) -> int:
    return int(_load().oracle_output_length(n, h_per_sample, bits, eps_lhl))


def minentropy_quantum(samples_on: np.ndarray, samples_off: np.ndarray, bits: int, eps: float):
    """Classical-noise subtraction (Sec. II.B): (report of the quantum model, H^{q+c} - H'^c)."""
    h_on, bad_on = histogram(samples_on, bits)
    h_off, bad_off = histogram(samples_off, bits)
    if bad_on or bad_off:
        raise ValueError("sample >= 2^bits")
    rep = HminReport()
    hs = ctypes.c_double()
    _check(_load().oracle_minentropy_quantum_from_hist(_u64(h_on), _u64(h_off), bits, eps, ctypes.byref(rep),
                                                       ctypes.byref(hs)), "minentropy_quantum")
    return rep.as_dict(), hs.value


def splitmix64(x0: int, s: int) -> int:
    return int(_load().oracle_splitmix64(x0 & (2**64 - 1), s))


def histogram_sampled(samples: np.ndarray, bits: int, fraction: float, sel_seed: int):
    samples = np.ascontiguousarray(samples)
    hist = np.zeros(1 << bits, dtype=np.uint64)
    bad = np.zeros(1, dtype=np.uint64)
    _check(_load().oracle_histogram_sampled(samples.ctypes.data, samples.size, bits, fraction, sel_seed, _u64(hist),
                                            _u64(bad)), "histogram_sampled")
    return hist, int(bad[0])


def minentropy_sampled(samples: np.ndarray, bits: int, eps: float, fraction: float, sel_seed: int) -> dict:
    """Sec. II.C: the corrected entropy from a random subsample of the stream."""
    hist, bad = histogram_sampled(samples, bits, fraction, sel_seed)
    if bad:
        raise ValueError("sample >= 2^bits")
    return minentropy_from_hist(hist, bits, eps)
