"""Python binding of libqrng_gb300.so (the C ABI in include/qrng.h).

Argument marshalling only: every function forwards to the C entry point of the same name, and
every step of the computation runs in the library's CUDA kernels. Buffers are passed as torch
tensors (their data_ptr) or as integer addresses; streams as torch.cuda.Stream objects, raw
cudaStream_t integers, or None for torch's current stream. There is no CPU fallback: if the
shared library is missing, importing a function that needs it raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqrng_gb300.so")

QRNG_OK, QRNG_EINVAL, QRNG_ENOMEM, QRNG_ECUDA, QRNG_ETIMEOUT, QRNG_EPRECISION, QRNG_ENOTSUP = range(7)
QRNG_FORM_STANDARD, QRNG_FORM_MODIFIED = 0, 1
(QRNG_ALGO_AUTO, QRNG_ALGO_DIRECT, QRNG_ALGO_GEMM_TC, QRNG_ALGO_FFT64, QRNG_ALGO_FFT32_SEG, QRNG_ALGO_NTT,
 QRNG_ALGO_GEMM_FP4, QRNG_ALGO_GEMM_FP4_PAIR, QRNG_ALGO_GEMM_KARATSUBA) = range(9)
ALGO_NAMES = {QRNG_ALGO_AUTO: "auto", QRNG_ALGO_DIRECT: "direct", QRNG_ALGO_GEMM_TC: "gemm_tc",
              QRNG_ALGO_FFT64: "fft64", QRNG_ALGO_FFT32_SEG: "fft32_seg", QRNG_ALGO_NTT: "ntt",
              QRNG_ALGO_GEMM_FP4: "gemm_fp4", QRNG_ALGO_GEMM_FP4_PAIR: "gemm_fp4_pair",
              QRNG_ALGO_GEMM_KARATSUBA: "gemm_karatsuba"}

EXPORTED = ["qrng_create", "qrng_destroy", "qrng_last_error", "qrng_status_string", "qrng_minentropy",
            "qrng_output_length", "qrng_seed_bits", "qrng_toeplitz_extract", "qrng_postprocess", "qrng_postprocess_host",
            "qrng_postprocess_host_async", "qrng_postprocess_host_wait",
            "qrng_get_stats", "qrng_extract_stats", "qrng_reset_stats", "qrng_set_timing", "qrng_synchronize",
            "qrng_minentropy_noalloc", "qrng_extract_batch", "qrng_set_autotune", "qrng_inject_fault",
            "qrng_minentropy_sampled", "qrng_minentropy_quantum", "qrng_set_karatsuba", "qrng_karatsuba_plan",
            "qrng_set_fft32", "qrng_fft32_terms_bound"]
QRNG_FAULT_NONE, QRNG_FAULT_GEMM_NO_TMA = 0, 1


class QrngError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


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


class Request(ctypes.Structure):
    """qrng_request: one block with its own seed and shape (device pointers)."""
    _fields_ = [
        ("raw", ctypes.c_void_p),
        ("raw_bit_off", ctypes.c_uint64),
        ("n", ctypes.c_uint64),
        ("m", ctypes.c_uint64),
        ("seed", ctypes.c_void_p),
        ("form", ctypes.c_int),
        ("out", ctypes.c_void_p),
        ("out_bit_off", ctypes.c_uint64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("last_algo", ctypes.c_int),
        ("last_kernels", ctypes.c_uint32),
        ("kernels_launched", ctypes.c_uint64),
        ("worst_fft_round_err", ctypes.c_double),
        ("timed_launches", ctypes.c_uint64),
        ("timed_ms", ctypes.c_double),
        ("hist_timed_launches", ctypes.c_uint64),
        ("hist_timed_ms", ctypes.c_double),
        ("batch_graph_ms", ctypes.c_double),
        ("batch_requests", ctypes.c_uint64 * 4),
        ("batch_direct_bitmacs", ctypes.c_double),
        ("batch_transform_bytes", ctypes.c_double),
        ("batch_direct_ms", ctypes.c_double),
        ("batch_transform_ms", ctypes.c_double),
        ("worst_fft32_round_err", ctypes.c_double),
        ("fft32_recomputed", ctypes.c_uint64),
        ("last_fft32_segment", ctypes.c_uint64),
        ("kara_presplits", ctypes.c_uint64),
        ("kara_presplits_used", ctypes.c_uint64),
        ("autotune_runs", ctypes.c_uint64),
        ("speculative_hashes", ctypes.c_uint64),
        ("speculative_misses", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["batch_requests"] = dict(zip(("direct", "ntt", "fft64", "fft32_seg"), list(self.batch_requests)))
        return d


class KaratsubaPlan(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("block_bits", ctypes.c_uint64),
        ("products", ctypes.c_uint64),
        ("rows", ctypes.c_uint64),
        ("cols", ctypes.c_uint64),
        ("blocks_per_pass", ctypes.c_uint64),
        ("model_seconds", ctypes.c_double),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    lib.qrng_create.argtypes = [ctypes.POINTER(vp), i32]
    lib.qrng_destroy.argtypes = [vp]
    lib.qrng_destroy.restype = None
    lib.qrng_last_error.argtypes = [vp]
    lib.qrng_last_error.restype = ctypes.c_char_p
    lib.qrng_status_string.argtypes = [i32]
    lib.qrng_status_string.restype = ctypes.c_char_p
    lib.qrng_minentropy.argtypes = [vp, vp, u64, i32, dbl, ctypes.POINTER(HminReport), vp]
    lib.qrng_output_length.argtypes = [u64, dbl, i32, dbl]
    lib.qrng_output_length.restype = u64
    lib.qrng_seed_bits.argtypes = [u64, u64, i32]
    lib.qrng_seed_bits.restype = u64
    lib.qrng_toeplitz_extract.argtypes = [vp, vp, u64, u64, vp, i32, i32, u64, vp, vp]
    lib.qrng_postprocess.argtypes = [vp, vp, u64, i32, dbl, dbl, u64, vp, u64, i32, i32, vp, u64,
                                     ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(HminReport), vp]
    lib.qrng_postprocess_host.argtypes = [vp, vp, u64, i32, dbl, dbl, u64, vp, u64, i32, i32, vp, u64,
                                          ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(HminReport), vp]
    lib.qrng_postprocess_host_async.argtypes = [vp, vp, u64, i32, dbl, dbl, u64, vp, u64, i32, i32, vp, u64,
                                                ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(HminReport),
                                                vp]
    lib.qrng_postprocess_host_wait.argtypes = [vp, vp]
    lib.qrng_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.qrng_extract_stats.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.qrng_reset_stats.argtypes = [vp]
    lib.qrng_set_timing.argtypes = [vp, i32]
    lib.qrng_synchronize.argtypes = [vp, vp]
    lib.qrng_set_autotune.argtypes = [vp, i32]
    lib.qrng_set_karatsuba.argtypes = [vp, i32, u64, u64]
    lib.qrng_set_fft32.argtypes = [vp, u64, i32]
    lib.qrng_fft32_terms_bound.argtypes = [u64]
    lib.qrng_karatsuba_plan.argtypes = [vp, u64, u64, i32, u64, ctypes.POINTER(KaratsubaPlan)]
    lib.qrng_minentropy_sampled.argtypes = [vp, vp, u64, i32, dbl, dbl, u64, ctypes.POINTER(HminReport), vp]
    lib.qrng_minentropy_quantum.argtypes = [vp, vp, u64, vp, u64, i32, dbl, ctypes.POINTER(HminReport),
                                            ctypes.POINTER(dbl), vp]
    lib.qrng_inject_fault.argtypes = [vp, i32]
    lib.qrng_extract_batch.argtypes = [vp, ctypes.POINTER(Request), u64, i32, vp]
    lib.qrng_minentropy_noalloc.argtypes = [vp, u64, i32, dbl, ctypes.POINTER(HminReport), vp]
    _lib = lib
    return lib


def _status_name(status: int) -> str:
    try:
        return load_library().qrng_status_string(status).decode()
    except Exception:  # the library itself failed to load
        return f"status {status}"


def _ptr(x) -> int:
    """Address of a tensor / numpy array / integer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """Owns a qrng_ctx* (workspace, statistics) bound to one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        st = lib.qrng_create(ctypes.byref(h), device)
        if st != QRNG_OK:
            raise QrngError(st, f"qrng_create(device={device}) failed")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load_library().qrng_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def check(self, st: int, what: str):
        if st != QRNG_OK:
            msg = load_library().qrng_last_error(self.handle).decode()
            raise QrngError(st, f"{what}: {msg}")


def qrng_create(device: int = 0) -> Context:
    return Context(device)


def qrng_destroy(ctx: Context):
    ctx.close()


def qrng_last_error(ctx: Context) -> str:
    return load_library().qrng_last_error(ctx.handle).decode()


def qrng_status_string(status: int) -> str:
    return load_library().qrng_status_string(status).decode()


def qrng_minentropy(ctx: Context, samples, count: int | None = None, bits: int = 8, eps: float = 1e-6,
                    stream=None) -> dict:
    """Min-entropy report of device samples (uint8 for bits <= 8, uint16 otherwise)."""
    if count is None:
        count = samples.numel()
    rep = HminReport()
    st = load_library().qrng_minentropy(ctx.handle, _ptr(samples), count, bits, eps, ctypes.byref(rep),
                                        _stream(stream))
    ctx.check(st, "qrng_minentropy")
    return rep.as_dict()


def qrng_output_length(n: int, h_per_sample: float, bits: int, eps_lhl: float) -> int:
    return int(load_library().qrng_output_length(n, h_per_sample, bits, eps_lhl))


def qrng_seed_bits(n: int, m: int, form: int) -> int:
    return int(load_library().qrng_seed_bits(n, m, form))


def qrng_toeplitz_extract(ctx: Context, raw, n: int, m: int, seed, form: int, algo: int, num_blocks: int, out,
                          stream=None):
    """Hash num_blocks n-bit blocks of `raw` (device) with `seed` (device) into `out` (device)."""
    st = load_library().qrng_toeplitz_extract(ctx.handle, _ptr(raw), n, m, _ptr(seed), form, algo, num_blocks,
                                              _ptr(out), _stream(stream))
    ctx.check(st, "qrng_toeplitz_extract")
    return out


def qrng_postprocess(ctx: Context, samples, count: int, bits: int, eps: float, eps_lhl: float, n: int, seed,
                     seed_capacity_bits: int, form: int, algo: int, out, out_capacity_bytes: int, stream=None):
    """Whole pipeline on device buffers (the samples are also the raw stream); returns
    (m, num_blocks, report). The hash is left running on `stream`."""
    m = ctypes.c_uint64()
    nb = ctypes.c_uint64()
    rep = HminReport()
    st = load_library().qrng_postprocess(ctx.handle, _ptr(samples), count, bits, eps, eps_lhl, n, _ptr(seed),
                                         seed_capacity_bits, form, algo, _ptr(out), out_capacity_bytes,
                                         ctypes.byref(m), ctypes.byref(nb), ctypes.byref(rep), _stream(stream))
    ctx.check(st, "qrng_postprocess")
    return int(m.value), int(nb.value), rep.as_dict()


def qrng_postprocess_host_async(ctx: Context, samples, count: int, bits: int, eps: float, eps_lhl: float, n: int,
                                seed, seed_capacity_bits: int, form: int, algo: int, out, out_capacity_bytes: int,
                                stream=None):
    """Overlapped host pipeline: returns (m, num_blocks, report) once the call's hash and output
    download are enqueued; `out` is complete after a later qrng_postprocess_host_wait."""
    m = ctypes.c_uint64()
    nb = ctypes.c_uint64()
    rep = HminReport()
    st = load_library().qrng_postprocess_host_async(ctx.handle, _ptr(samples), count, bits, eps, eps_lhl, n,
                                                    _ptr(seed), seed_capacity_bits, form, algo, _ptr(out),
                                                    out_capacity_bytes, ctypes.byref(m), ctypes.byref(nb),
                                                    ctypes.byref(rep), _stream(stream))
    ctx.check(st, "qrng_postprocess_host_async")
    return int(m.value), int(nb.value), rep.as_dict()


def qrng_postprocess_host_wait(ctx: Context, stream=None):
    ctx.check(load_library().qrng_postprocess_host_wait(ctx.handle, _stream(stream)), "qrng_postprocess_host_wait")


def qrng_postprocess_host(ctx: Context, samples, count: int, bits: int, eps: float, eps_lhl: float, n: int, seed,
                          seed_capacity_bits: int, form: int, algo: int, out, out_capacity_bytes: int, stream=None):
    """Whole pipeline on host buffers; returns (m, num_blocks, report)."""
    m = ctypes.c_uint64()
    nb = ctypes.c_uint64()
    rep = HminReport()
    st = load_library().qrng_postprocess_host(ctx.handle, _ptr(samples), count, bits, eps, eps_lhl, n, _ptr(seed),
                                              seed_capacity_bits, form, algo, _ptr(out), out_capacity_bytes,
                                              ctypes.byref(m), ctypes.byref(nb), ctypes.byref(rep), _stream(stream))
    ctx.check(st, "qrng_postprocess_host")
    return int(m.value), int(nb.value), rep.as_dict()


def qrng_get_stats(ctx: Context) -> dict:
    s = Stats()
    ctx.check(load_library().qrng_get_stats(ctx.handle, ctypes.byref(s)), "qrng_get_stats")
    return s.as_dict()


def qrng_extract_stats(ctx: Context) -> float:
    """Worst |s - round(s)| of the FFT routes since the last reset."""
    w = ctypes.c_double()
    ctx.check(load_library().qrng_extract_stats(ctx.handle, ctypes.byref(w)), "qrng_extract_stats")
    return w.value


def qrng_reset_stats(ctx: Context):
    ctx.check(load_library().qrng_reset_stats(ctx.handle), "qrng_reset_stats")


def qrng_set_timing(ctx: Context, on: bool):
    ctx.check(load_library().qrng_set_timing(ctx.handle, 1 if on else 0), "qrng_set_timing")


def qrng_synchronize(ctx: Context, stream=None):
    """Wait for the stream; raises QrngError(QRNG_ETIMEOUT) if a kernel's bounded wait gave up."""
    ctx.check(load_library().qrng_synchronize(ctx.handle, _stream(stream)), "qrng_synchronize")


def qrng_minentropy_noalloc(samples, count: int | None = None, bits: int = 8, eps: float = 1e-6,
                            stream=None) -> dict:
    """qrng_minentropy without a context and without any device allocation (fixed scratch
    compiled into the library; see include/qrng.h). Runs on the current CUDA device."""
    if count is None:
        count = samples.numel()
    rep = HminReport()
    st = load_library().qrng_minentropy_noalloc(_ptr(samples), count, bits, eps, ctypes.byref(rep), _stream(stream))
    if st != QRNG_OK:
        raise QrngError(st, "qrng_minentropy_noalloc")
    return rep.as_dict()


def qrng_extract_batch(ctx: Context, requests, algo: int = QRNG_ALGO_AUTO, stream=None):
    """Hash a list of requests, each a dict or tuple (raw, raw_bit_off, n, m, seed, form, out, out_bit_off)
    with device addresses (tensors or ints), in one persistent launch."""
    arr = (Request * len(requests))()
    for i, r in enumerate(requests):
        if isinstance(r, dict):
            r = (r["raw"], r.get("raw_bit_off", 0), r["n"], r["m"], r["seed"], r.get("form", 0), r["out"],
                 r.get("out_bit_off", 0))
        raw, roff, n, m, seed, form, out, ooff = r
        arr[i] = Request(_ptr(raw), roff, n, m, _ptr(seed), form, _ptr(out), ooff)
    st = load_library().qrng_extract_batch(ctx.handle, arr, len(requests), algo, _stream(stream))
    ctx.check(st, "qrng_extract_batch")


def qrng_set_autotune(ctx: Context, on: bool):
    ctx.check(load_library().qrng_set_autotune(ctx.handle, 1 if on else 0), "qrng_set_autotune")


def qrng_set_karatsuba(ctx: Context, levels: int = 0, block_bits: int = 0, max_workspace: int = 0):
    """Block Karatsuba settings of QRNG_ALGO_GEMM_KARATSUBA (0 = chosen by the cost model)."""
    ctx.check(load_library().qrng_set_karatsuba(ctx.handle, levels, block_bits, max_workspace), "qrng_set_karatsuba")


def qrng_set_fft32(ctx: Context, segment_bits: int = 0, terms: int = 0):
    """FP32 segmented FFT settings (0 = chosen per shape / the proven bound)."""
    ctx.check(load_library().qrng_set_fft32(ctx.handle, segment_bits, terms), "qrng_set_fft32")


def qrng_fft32_terms_bound(segment_bits: int) -> int:
    return int(load_library().qrng_fft32_terms_bound(segment_bits))


def qrng_karatsuba_plan(ctx: Context, n: int, m: int, form: int, num_blocks: int) -> dict:
    """The block Karatsuba plan of QRNG_ALGO_GEMM_KARATSUBA for this shape (no GPU work)."""
    info = KaratsubaPlan()
    ctx.check(load_library().qrng_karatsuba_plan(ctx.handle, n, m, form, num_blocks, ctypes.byref(info)),
              "qrng_karatsuba_plan")
    return {"levels": info.levels, "h": info.block_bits, "groups": info.products, "mq": info.rows,
            "kq": info.cols, "blocks_per_pass": info.blocks_per_pass, "model_s": info.model_seconds}


def qrng_inject_fault(ctx: Context, fault: int):
    ctx.check(load_library().qrng_inject_fault(ctx.handle, fault), "qrng_inject_fault")


def qrng_minentropy_sampled(ctx: Context, samples, count: int | None = None, bits: int = 8, eps: float = 1e-6,
                            fraction: float = 1.0, sel_seed: int = 0, stream=None) -> dict:
    """Min-entropy report of a random subsample (splitmix64 selection) of device samples."""
    if count is None:
        count = samples.numel()
    rep = HminReport()
    st = load_library().qrng_minentropy_sampled(ctx.handle, _ptr(samples), count, bits, eps, fraction,
                                                sel_seed & (2**64 - 1), ctypes.byref(rep), _stream(stream))
    ctx.check(st, "qrng_minentropy_sampled")
    return rep.as_dict()


def qrng_minentropy_quantum(ctx: Context, samples_on, samples_off, count_on: int | None = None,
                            count_off: int | None = None, bits: int = 8, eps: float = 1e-6, stream=None):
    """Classical-noise subtraction: (report of the quantum model, H^{q+c} - H'^c)."""
    if count_on is None:
        count_on = samples_on.numel()
    if count_off is None:
        count_off = samples_off.numel()
    rep = HminReport()
    hs = ctypes.c_double()
    st = load_library().qrng_minentropy_quantum(ctx.handle, _ptr(samples_on), count_on, _ptr(samples_off), count_off,
                                                bits, eps, ctypes.byref(rep), ctypes.byref(hs), _stream(stream))
    ctx.check(st, "qrng_minentropy_quantum")
    return rep.as_dict(), hs.value
