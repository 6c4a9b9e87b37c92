"""Benchmark of the QRNG post-processing hot path on GB300.

Workload (the laser-phase-noise stream): 2^26 uint8 ADC samples ~ clip(round(N(128, 16^2))),
whose bytes are also the 2^29-bit raw stream; blocks of n = 2^16 bits; m = floor(n H_modify / 8)
from the corrected min-entropy (eps = 1e-6); one standard Toeplitz seed of n+m-1 bits shared by
every block. One step = one qrng_postprocess call: min-entropy estimate (histogram + FP64
finaliser, report read back) + extraction of all 8192 blocks. Metric: extracted output Gbit/s, bit-exact.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "extracted random Gbit/s on 1 GB300 (bit-exact), batched form vs plain per-block"
UNIT = "Gbit/s"
L2_FLUSH_BYTES = 256 << 20
# Integer-pipe rate of the direct kernel's LOP3: 64 results per clock per SM (the 32-bit bitwise
# throughput of the CUDA arithmetic-instruction table; a LOP3 throughput loop on this GB300 gave
# 1.888e13 LOP3/s at 1.99 GHz on 152 SMs = 62.4 per clock per SM), 32 bit-products per LOP3.
LOP3_PER_CLK_SM = 64
FP32_FMA_PER_CLK_SM = 128
FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (non-tensor) nominal


def device_caps(dev=0):
    """SM count of the device (read at run time) and the maximum SM clock (MEASURED_PEAKS.json,
    else GB300's 2070 MHz)."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return {"sms": sms, "sm_max_mhz": mhz}


def alu_peak_tbitmac(caps):
    return LOP3_PER_CLK_SM * 32 * caps["sms"] * caps["sm_max_mhz"] * 1e6 / 1e12


def fp32_peak_tflops(caps):
    return 2 * FP32_FMA_PER_CLK_SM * caps["sms"] * caps["sm_max_mhz"] * 1e6 / 1e12


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--algo", default="auto")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--blocks", type=int, default=0,
                   help="hash only the first BLOCKS blocks (a smaller case for profiler captures)")
    p.add_argument("--headline-only", action="store_true",
                   help="skip the per-configuration sub-records after the headline measurement")
    p.add_argument("--workload", default="laser",
                   choices=["laser", "single", "sweep", "tc", "uneven", "forms", "long", "hist"],
                   help="laser: the headline stream (default); single: one 4096-bit block; sweep: block-length "
                        "sweep on a 2^30-bit stream; tc: m=6144, n=8192, 4096 blocks; uneven: 10,000 requests; "
                        "long: 64 blocks of 2^22 bits (the transform route's profiling case)")
    p.add_argument("--sweep-algos", default="direct,gemm_tc,gemm_fp4,gemm_fp4_pair,gemm_karatsuba,ntt,fft64,fft32_seg",
                   help="algorithms timed at each block length of the sweep")
    p.add_argument("--uneven-max-log2n", type=float, default=22.0,
                   help="upper end of the log-uniform n range of the uneven requests")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_stream_seed(base: int, rank: int) -> int:
    """Weak scaling: every rank hashes its own stream of the same size (blocks are independent,
    Sec. III.E), so ranks only differ in the seed of their synthetic input."""
    return base + 1000 * rank


def reduce_max(value: float, world: int, device) -> float:
    """Largest value over the ranks (the timing rule: the job takes as long as its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, bits_per_rank: int, steps: int, t_ms: float) -> float:
    """Whole-job Gbit/s: output bits of all ranks over the slowest rank's time."""
    return world * bits_per_rank * steps / (t_ms / 1e3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the warm-up until
    after the timed region; `summary` keeps the samples whose host time falls in the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (host time, line)
        self.window = None

    def start(self):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                if line.strip():
                    self.samples.append((time.time(), line))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        time.sleep(0.3)  # let the first samples arrive before the timed region
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window if self.window else (float("-inf"), float("inf"))
        for ts, line in self.samples:
            if not (t0 <= ts <= t1 + 0.06):  # a sample is printed shortly after it is taken
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples_in_timed_region": len(sm)}


def run_ours(args, world, rank, local):
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    ctx = q.Context(local)
    algo = ALGOS[args.algo]

    c = W.CFG2
    n, eps, bits = c["n"], c["eps"], 8
    # weak scaling: every rank owns its own stream of the same size (independent blocks)
    samples_h = W.adc_samples(c["samples"], rank_stream_seed(c["sample_seed"], rank))
    samples = torch.from_numpy(samples_h).to(dev)
    seed_h = W.random_bits(2 * n - 1, c["seed_seed"])  # long enough for any m <= n
    seed = torch.from_numpy(seed_h).to(dev)
    num_blocks = samples_h.size * 8 // n
    if args.blocks:
        num_blocks = min(num_blocks, args.blocks)
    out = torch.empty((num_blocks * n + 7) // 8, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(a=algo):
        # the whole path in one call: estimate (read back to size m), then the hash of every block
        m, _, _ = q.qrng_postprocess(ctx, samples, num_blocks * n // 8, bits, eps, 1.0, n, seed, 2 * n - 1,
                                     q.QRNG_FORM_STANDARD, a, out, out.numel(), stream=stream)
        return m

    for _ in range(args.warmup):
        m = step()
    torch.cuda.synchronize()
    q.qrng_reset_stats(ctx)
    q.qrng_set_timing(ctx, True)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local).start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # evict the 64 MiB input from the 129 MB L2 between steps
        ev[i][0].record(stream)
        m = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(t_wall0, time.time())
    clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    stats = q.qrng_get_stats(ctx)
    q.qrng_set_timing(ctx, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = reduce_max(sum(step_ms), world, dev)
    out_bits = num_blocks * m
    value = job_throughput(world, out_bits, args.steps, t_total)
    kernel_ms = stats["timed_ms"] / max(1, stats["timed_launches"])
    used_algo = q.ALGO_NAMES.get(stats["last_algo"], str(stats["last_algo"]))
    caps = device_caps(local)

    # plain per-block direct kernel on the same inputs, same timing method
    plain = None
    if algo != q.QRNG_ALGO_DIRECT:
        q.qrng_reset_stats(ctx)
        q.qrng_set_timing(ctx, True)
        for i in range(max(3, args.steps // 2)):
            flush.fill_(i & 0xFF)
            q.qrng_toeplitz_extract(ctx, samples, n, m, seed, q.QRNG_FORM_STANDARD, q.QRNG_ALGO_DIRECT, num_blocks,
                                    out, stream=stream)
        s2 = q.qrng_get_stats(ctx)
        q.qrng_set_timing(ctx, False)
        pms = s2["timed_ms"] / max(1, s2["timed_launches"])
        plain = {"algo": "direct", "kernel_ms": pms, "gbps": out_bits / (pms / 1e3) / 1e9}
    # step again after the plain run so the final output is the measured algorithm's
    m = step()
    torch.cuda.synchronize()
    out_host = out[:(num_blocks * m + 7) // 8].cpu().numpy()

    plan = q.qrng_karatsuba_plan(ctx, n, m, q.QRNG_FORM_STANDARD, num_blocks) if used_algo == "gemm_karatsuba" else None
    roofline = roofline_for(used_algo, num_blocks, m, n, kernel_ms, plan, caps)

    # end to end through the host-buffer entry point (pinned host memory, copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        pin_samples = torch.from_numpy(samples_h).pin_memory()
        pin_seed = torch.from_numpy(seed_h).pin_memory()
        pin_out = [torch.empty(num_blocks * n // 8, dtype=torch.uint8).pin_memory() for _ in range(2)]

        # the overlapped host pipeline: every step uploads its samples and seed from pinned host
        # memory and downloads its output; a step's copies run beside its neighbours' hashing
        def e2e_steps(count):
            res = None
            for i in range(count):
                res = q.qrng_postprocess_host_async(ctx, pin_samples, samples_h.size, bits, eps, 1.0, n, pin_seed,
                                                    2 * n - 1, q.QRNG_FORM_STANDARD, algo, pin_out[i & 1],
                                                    pin_out[i & 1].numel(), stream=stream)
            q.qrng_postprocess_host_wait(ctx, stream=stream)
            return res

        e2e_steps(args.warmup)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m2, nb2, _ = e2e_steps(args.steps)
        b.record(stream)
        b.synchronize()
        et = reduce_max(a.elapsed_time(b), world, dev)
        e2e = {"value": job_throughput(world, nb2 * m2, args.steps, et), "unit": UNIT,
               "h2d_bytes_per_step": int(samples_h.nbytes + pin_seed.numel()),
               "d2h_bytes_per_step": int((nb2 * m2 + 7) // 8 + 112), "ms_per_step": et / args.steps,
               "api": "qrng_postprocess_host_async per step, qrng_postprocess_host_wait after the last (consecutive "
                      "steps overlap: one step's copies beside its neighbours' hashing)"}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES.get(used_algo, "u32 (bit-packed GF(2))"),
        "data": "synthetic",
        "config": {"workload": "laser-phase-noise stream: 2^26 uint8 ADC samples ~ round(N(128,16^2)) clipped, "
                               "2^29 raw bits, n=2^16, m=floor(n*H_modify/8), one shared standard seed",
                   "n": n, "m": m, "blocks_per_gpu": num_blocks, "eps": eps, "algo": used_algo,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"blocks sharded, {world} rank(s)"},
        "gpu_launches": int(stats["kernels_launched"]),
        "roofline": roofline,
        "plain_per_block": plain,
        "e2e": e2e,
        "clocks": clocks.summary(),
        "device": {"sms": caps["sms"], "sm_max_mhz": caps["sm_max_mhz"]},
    }
    if rank == 0 and not args.headline_only:
        result["configs"] = run_subrecords(q, ctx, local, caps, flush, (samples, seed, n, m, num_blocks, out))
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"], result["oracle_check"] = cpu_baseline(samples_h, seed_h, n, m, eps, out_host,
                                                                      num_blocks)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


DTYPES = {"gemm_tc": "e4m3 0/1 operands, f32 accumulate",
          "gemm_fp4": "e2m1 0/1 operands (ue8m0 scales 2^0), f32 accumulate",
          "gemm_fp4_pair": "e2m1 0/1 operands (ue8m0 scales 2^0), f32 accumulate",
          "gemm_karatsuba": "e2m1 0/1 operands (ue8m0 scales 2^0), f32 accumulate"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback"}


def captured_traffic(kernel: str, source: str, units: int):
    """DRAM bytes of one launch from the committed ncu capture, scaled to `units` blocks; None when
    the kernel's source changed since the capture."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, "paper_2011_04130_gb300", "csrc", source), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256") != sha:
        return None
    return int(rec["dram_bytes"] * units / rec["blocks"])


def hbm_record(bytes_moved, ms):
    pk = measured_peaks()
    gbs = bytes_moved / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
            "algorithmic_bytes": int(bytes_moved), "peak_source": "copy bandwidth " + pk["source"]}


def roofline_for(algo, num_blocks, m, n_t, kernel_ms, plan=None, caps=None, n=None):
    """Roofline of the dominant (extraction) kernel from its algorithmic work and live event time.
    n_t is the Toeplitz width (n, or n - m for the modified form); n the block length."""
    if caps is None and algo in ("direct", "fft32_seg"):
        caps = device_caps()
    n = n or n_t
    io_bytes = num_blocks * (n + m) / 8  # raw bits in, output bits out
    if algo == "direct":
        peak = alu_peak_tbitmac(caps)
        achieved = num_blocks * m * n_t / (kernel_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tbit-MAC/s", "frac": achieved / peak,
                "traffic": captured_traffic("direct_kernel", "k_direct.cu", num_blocks),
                "kernel": "direct_kernel<32>", "kernel_ms": kernel_ms,
                "peak_source": f"derived: {LOP3_PER_CLK_SM} LOP3/clk/SM x 32 bit-MACs x {caps['sms']} SMs x "
                               f"{caps['sm_max_mhz']:g} MHz"}
    if algo == "gemm_tc":
        pk = measured_peaks()
        peak = 2.0 * pk["bf16_tflops"]  # FP8 dense = bf16 measured x nominal ratio 4.5/2.25
        achieved = 2.0 * num_blocks * m * n_t / (kernel_ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": captured_traffic("gemm_tc_kernel", "k_gemm_tc.cu", num_blocks),
                "kernel": "gemm_tc_kernel (tcgen05 kind::f8f6f4)", "kernel_ms": kernel_ms,
                "peak_source": "FP8 = 2 x bf16 burst " + pk["source"]}
    if algo in ("gemm_fp4", "gemm_fp4_pair"):
        pk = measured_peaks()
        peak = 6.0 * pk["bf16_tflops"]  # FP4 dense = bf16 measured x nominal ratio 13.5/2.25
        achieved = 2.0 * num_blocks * m * n_t / (kernel_ms / 1e3) / 1e12
        pair = algo == "gemm_fp4_pair"
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (captured_traffic("gemm_pair_kernel", "k_gemm_pair.cu", num_blocks) if pair
                            else captured_traffic("gemm_fp4_kernel", "k_gemm_tc.cu", num_blocks)),
                "kernel": ("gemm_pair_kernel (tcgen05 cta_group::2 kind::mxf4, block scale 2^0)" if pair
                           else "gemm_tc_kernel<fp4> (tcgen05 kind::mxf4, block scale 2^0)"),
                "kernel_ms": kernel_ms, "peak_source": "FP4 = 6 x bf16 burst " + pk["source"]}
    if algo == "gemm_karatsuba":
        # the product kernel's own work: 3^L dense sub-products per block (the plan the library
        # ran, from qrng_karatsuba_plan), of kq columns and the rows it issues MMAs for: the
        # output tiles of 256 rows holding the ceil(m / span) h rows some output needs (mq pads
        # them to whole pairs of tiles; a pair's second tile past them gets no MMAs)
        pk = measured_peaks()
        peak = 6.0 * pk["bf16_tflops"]
        plan = plan or {}
        span = plan["h"] << plan["levels"]
        rows = min(plan["mq"], -(-(-(-m // span) * plan["h"]) // 256) * 256)
        flops = 2.0 * num_blocks * plan["groups"] * rows * plan["kq"]
        achieved = flops / (kernel_ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": captured_traffic("gemm_pair_kara_kernel", "k_gemm_pair.cu", num_blocks),
                "kernel": "gemm_pair_kernel<kKara> (tcgen05 cta_group::2 kind::mxf4 on the block-Karatsuba "
                          "sub-products)", "kernel_ms": kernel_ms,
                "plan": plan, "rows_issued": rows,
                "equivalent_plain_tflops": 2.0 * num_blocks * m * n_t / (kernel_ms / 1e3) / 1e12,
                "peak_source": "FP4 = 6 x bf16 burst " + pk["source"]}
    if algo == "fft64":
        # two P-point complex FP64 transforms per pair of blocks (5 P log2 P flops each) and the
        # spectrum product (6 P)
        P = 1 << max(1, (n_t + m - 2).bit_length())
        flops = (num_blocks + 1) // 2 * (2 * 5.0 * P * math.log2(P) + 6.0 * P)
        achieved = flops / (kernel_ms / 1e3) / 1e12
        return {"bound": "fp64", "achieved": achieved, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                "frac": achieved / FP64_TFLOPS_NOMINAL, "kernel": "stockham_pass4_kernel et al. (FP64)",
                "kernel_ms": kernel_ms, "hbm": hbm_record(io_bytes, kernel_ms),
                "peak_source": "GB300 FP64 nominal 1.25 TFLOP/s"}
    if algo == "fft32_seg":
        # per block: NS segment and (once per call) NQ + NS - 1 window transforms, NQ ceil(NS/T)
        # inverses (5 S log2 S flops each, S-point complex), NQ NS products of S bins (8 flops each)
        S = (plan or {}).get("segment") or 4096
        T = (plan or {}).get("terms") or 8
        NS, NQ = -(-n_t // S), -(-m // S)
        lg = S.bit_length() - 1
        flops = num_blocks * ((NS + NQ * -(-NS // T)) * 5.0 * S * lg + NQ * NS * S * 8.0) + \
            (NQ + NS - 1) * 5.0 * S * lg
        achieved = flops / (kernel_ms / 1e3) / 1e12
        peak = fp32_peak_tflops(caps)
        return {"bound": "fp32", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "segment": S, "terms": T, "kernel": "seg_spectra_kernel + seg_mac_kernel (FP32)",
                "kernel_ms": kernel_ms, "hbm": hbm_record(io_bytes, kernel_ms),
                "peak_source": f"derived: {FP32_FMA_PER_CLK_SM} FMA/clk/SM x 2 x {caps['sms']} SMs x "
                               f"{caps['sm_max_mhz']:g} MHz"}
    if algo == "ntt":
        r = hbm_record(io_bytes, kernel_ms)
        r.update({"kernel": "ntt_cols_kernel + ntt_rows_kernel (integer issue bound)", "kernel_ms": kernel_ms,
                  "traffic": None})
        return r
    return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
            "kernel_ms": kernel_ms}


def cpu_baseline(samples_h, seed_h, n, m, eps, out_host=None, num_blocks=0):
    """The oracle as it stands on the host's cores: min-entropy of the whole stream (one C call)
    plus the full Toeplitz hash of one block per core, the blocks on threads (the oracle is plain C
    called through ctypes, which releases the interpreter lock); and the same with one block on one
    thread. When the timed output is given, the oracle's Freivalds check of every block of it."""
    import concurrent.futures

    import oracle

    cores = host_cores()

    def sample(blocks, threads):
        t0 = time.perf_counter()
        rep = oracle.minentropy(samples_h, 8, eps)
        m_or = oracle.output_length(n, rep["h_modify"], 8, 1.0)
        seed_o = seed_h[: (n + m_or - 1 + 7) // 8].copy()

        def one(b):
            oracle.toeplitz(samples_h, n, m_or, seed_o, 0, raw_off=b * n)

        with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, range(blocks)))
        return m_or, time.perf_counter() - t0

    m1, dt1 = sample(1, 1)
    mall, dtall = sample(cores, cores)
    res = {"value": cores * mall / dtall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"min-entropy of all {samples_h.size} samples (one thread) + full hash of {cores} of the "
                     f"{samples_h.size * 8 // n} blocks, one per thread (n={n}, m={mall})", "seconds": dtall,
           "single_thread": {"value": m1 / dt1 / 1e9, "unit": UNIT, "cores": 1, "seconds": dt1,
                             "sample": "min-entropy of the whole stream + full hash of one block"}}
    check = None
    if out_host is not None:
        t0 = time.perf_counter()
        seed_o = seed_h[: (n + m - 1 + 7) // 8].copy()
        mism = oracle.freivalds(samples_h, n, m, seed_o, 0, num_blocks, out_host, rng_seed=2024)
        check = {"oracle_m": mall, "gpu_m": m, "m_equal": mall == m, "blocks": num_blocks,
                 "freivalds_failures": int(np.count_nonzero(mism)), "escape_probability_per_block": "2^-64",
                 "seconds": time.perf_counter() - t0}
    return res, check


def run_reference(args, world, rank):
    """The CPU oracle on the same workload on the host's cores, each step a bounded sample: the
    min-entropy of the full stream, then the full hash of one block per core (one thread each)."""
    if rank != 0:
        return None
    import concurrent.futures

    import oracle

    oracle.build()
    c = W.CFG2
    n, eps = c["n"], c["eps"]
    samples_h = W.adc_samples(c["samples"], c["sample_seed"])
    seed_h = W.random_bits(2 * n - 1, c["seed_seed"])
    cores = host_cores()
    nblk = samples_h.size * 8 // n
    times, bits_out = [], 0
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            rep = oracle.minentropy(samples_h, 8, eps)
            m = oracle.output_length(n, rep["h_modify"], 8, 1.0)
            seed_o = seed_h[: (n + m - 1 + 7) // 8].copy()
            blocks = [(i * cores + k) % nblk for k in range(cores)]
            list(ex.map(lambda b: oracle.toeplitz(samples_h, n, m, seed_o, 0, raw_off=b * n), blocks))
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt)
                bits_out += m * cores
    total = sum(times)
    value = bits_out / total / 1e9
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8 (one byte per bit)",
            "data": "synthetic",
            "config": {"workload": "laser-phase-noise stream: 2^26 uint8 ADC samples, n=2^16, one shared seed",
                       "n": n, "m": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: min-entropy of all 2^26 samples (one thread) + the full hash "
                                       f"of {cores} blocks, one per thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


ALGOS = {"auto": 0, "direct": 1, "gemm_tc": 2, "fft64": 3, "fft32_seg": 4, "ntt": 5, "gemm_fp4": 6,
         "gemm_fp4_pair": 7, "gemm_karatsuba": 8}


def _time_extract(q, ctx, raw, n, m, seed, form, algo, blocks, out, reps, warmup=1, flush=None):
    """Mean CUDA-event time (ms) of the main extraction kernel and of the whole call (L2 flushed
    before each call when `flush` is given; the flush is outside both timings)."""
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        q.qrng_toeplitz_extract(ctx, raw, n, m, seed, form, algo, blocks, out, stream=stream)
    torch.cuda.synchronize()
    q.qrng_reset_stats(ctx)
    q.qrng_set_timing(ctx, True)
    call_ms = 0.0
    for i in range(reps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        q.qrng_toeplitz_extract(ctx, raw, n, m, seed, form, algo, blocks, out, stream=stream)
        b.record(stream)
        b.synchronize()
        call_ms += a.elapsed_time(b)
    q.qrng_synchronize(ctx)
    st = q.qrng_get_stats(ctx)
    q.qrng_set_timing(ctx, False)
    return st["timed_ms"] / max(1, reps), call_ms / reps, st


def clocked(local, fn, *a, **kw):
    """Runs fn under the clock sampler; the record gets the clocks of its own region."""
    clocks = ClockSampler(local).start()
    t0 = time.time()
    res = fn(*a, **kw)
    clocks.mark(t0, time.time())
    clocks.stop()
    res["clocks"] = clocks.summary()
    return res


def fft32_plan(q, st):
    """Segment length and terms per inverse of the last FP32 segmented call (the proven bound)."""
    S = int(st.get("last_fft32_segment") or 0)
    return {"segment": S, "terms": q.qrng_fft32_terms_bound(S)} if S else None


def sub_single(q, ctx, caps, reps=20):
    """Config 1: one 4096-bit block, m = 2048, plus the min-entropy of 65,536 samples: latency."""
    import torch

    c = W.CFG1
    samples_h = W.adc_samples(c["samples"], c["sample_seed"])
    samples = torch.from_numpy(samples_h).cuda()
    n, m = c["n"], c["m"]
    raw = torch.from_numpy(W.random_bits(n, c["raw_seed"])).cuda()
    seed = torch.from_numpy(W.random_bits(n + m - 1, c["seed_seed"])).cuda()
    out = torch.empty(m // 8, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        q.qrng_minentropy(ctx, samples, bits=8, eps=c["eps"])
    q.qrng_reset_stats(ctx)
    q.qrng_set_timing(ctx, True)
    t0 = time.perf_counter()
    for _ in range(reps):
        q.qrng_minentropy(ctx, samples, bits=8, eps=c["eps"])
    ent_us = (time.perf_counter() - t0) / reps * 1e6
    st = q.qrng_get_stats(ctx)
    q.qrng_set_timing(ctx, False)
    hist_us = st["hist_timed_ms"] / max(1, st["hist_timed_launches"]) * 1e3
    kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, 0, ALGOS["direct"], 1, out, reps=reps, warmup=3)
    return {"workload": "65,536 uint8 samples + one block n=4096, m=2048, standard seed", "bound": "latency",
            "minentropy_call_us_host": ent_us, "histogram_kernel_us": hist_us, "extract_kernel_us": kms * 1e3,
            "extract_call_us": cms * 1e3, "gbps": m / (cms / 1e3) / 1e9,
            "roofline": roofline_for("direct", 1, m, n, kms, caps=caps)}


def sub_histogram(q, ctx, flush, reps=10):
    """The histogram kernel alone on the laser stream's 2^26 uint8 samples and on 2^26 uint16
    samples of a 16-bit ADC (clip(round(N(2^15, 4096^2)))): HBM bytes over kernel time."""
    import torch

    res = {"workload": "histogram kernel: 2^26 uint8 samples (8-bit ADC) and 2^26 uint16 samples (16-bit ADC)"}
    c = W.CFG2
    for bits, samples_h in ((8, W.adc_samples(c["samples"], c["sample_seed"])),
                            (16, W.adc_samples(c["samples"], 41, mu=32768.0, sigma=4096.0, bits=16))):
        samples = torch.from_numpy(samples_h.view(np.uint8)).cuda()
        for _ in range(3):
            q.qrng_minentropy(ctx, samples, count=samples_h.size, bits=bits, eps=1e-6)
        q.qrng_reset_stats(ctx)
        q.qrng_set_timing(ctx, True)
        for i in range(reps):
            flush.fill_(i & 0xFF)
            q.qrng_minentropy(ctx, samples, count=samples_h.size, bits=bits, eps=1e-6)
        st = q.qrng_get_stats(ctx)
        q.qrng_set_timing(ctx, False)
        ms = st["hist_timed_ms"] / max(1, st["hist_timed_launches"])
        r = hbm_record(samples_h.nbytes, ms)
        r["kernel_us"] = ms * 1e3
        r["kernel"] = "hist_u8_kernel" if bits <= 8 else "hist_u16 kernel"
        res[f"bits{bits}"] = r
    return res


def sub_sweep(q, ctx, caps, flush, reps=2):
    """Config 3: a fixed 2^30-bit Bernoulli(0.5) stream, n = 2^10 .. 2^24, m = 0.75 n, modified
    form, one (n-1)-bit seed per n: AUTO's choice per n against the plain per-block direct kernel."""
    import torch

    c = W.CFG3
    raw = torch.from_numpy(W.random_bits(c["stream_bits"], c["raw_seed"])).cuda()
    out = torch.empty(c["stream_bits"] // 8, dtype=torch.uint8, device="cuda")
    rows = []
    for n in c["n_list"]:
        m = int(n * c["ratio"])
        B = c["stream_bits"] // n
        seed = torch.from_numpy(W.random_bits(n - 1, c["seed_seed"] + n.bit_length() - 1)).cuda()
        kms, cms, st = _time_extract(q, ctx, raw, n, m, seed, 1, ALGOS["auto"], B, out, reps=reps, flush=flush)
        algo = q.ALGO_NAMES.get(st["last_algo"], str(st["last_algo"]))
        plan = q.qrng_karatsuba_plan(ctx, n, m, 1, B) if algo == "gemm_karatsuba" else None
        rl = roofline_for(algo, B, m, n - m, kms, plan, caps, n=n)
        row = {"n": n, "m": m, "blocks": B, "algo": algo, "call_ms": cms, "kernel_ms": kms,
               "gbps": B * m / (cms / 1e3) / 1e9, "frac": rl.get("frac"), "bound": rl.get("bound")}
        if n <= (1 << 20):
            dk, dc, _ = _time_extract(q, ctx, raw, n, m, seed, 1, ALGOS["direct"], B, out, reps=1, flush=flush)
            row["direct"] = {"call_ms": dc, "gbps": B * m / (dc / 1e3) / 1e9,
                             "frac": roofline_for("direct", B, m, n - m, dk, caps=caps)["frac"]}
            fk, fc, fs = _time_extract(q, ctx, raw, n, m, seed, 1, ALGOS["fft32_seg"], B, out, reps=1, flush=flush)
            frl = roofline_for("fft32_seg", B, m, n - m, fk, fft32_plan(q, fs), caps, n=n)
            row["fft32_seg"] = {"call_ms": fc, "gbps": B * m / (fc / 1e3) / 1e9, "frac": frl["frac"],
                                "segment": frl["segment"], "worst_round_err": fs["worst_fft_round_err"]}
        rows.append(row)
    return {"workload": "block-length sweep: 2^30-bit Bernoulli(0.5) stream, n = 2^10..2^24, m = 0.75n, modified "
                        "form, AUTO vs the plain per-block direct kernel (n <= 2^20)", "unit": UNIT, "rows": rows}


def sub_tc(q, ctx, caps, flush, reps=5):
    """Config 4: one standard seed, m = 6144, n = 8192, 4096 blocks: the tensor-core products."""
    import torch

    c = W.CFG4
    n, m, B = c["n"], c["m"], c["blocks"]
    raw = torch.from_numpy(W.random_bits(n * B, c["raw_seed"])).cuda()
    seed = torch.from_numpy(W.random_bits(n + m - 1, c["seed_seed"])).cuda()
    out = torch.empty(m * B // 8, dtype=torch.uint8, device="cuda")
    res = {"workload": "m=6144, n=8192, 4096 blocks, one standard seed (T 6144x8192 times X 8192x4096)",
           "unit": UNIT}
    for name in ("gemm_karatsuba", "gemm_fp4_pair", "gemm_fp4", "gemm_tc", "direct"):
        kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, 0, ALGOS[name], B, out, reps=reps, flush=flush)
        plan = q.qrng_karatsuba_plan(ctx, n, m, 0, B) if name == "gemm_karatsuba" else None
        rl = roofline_for(name, B, m, n, kms, plan, caps)
        res[name] = {"kernel_ms": kms, "call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9, "achieved": rl["achieved"],
                     "unit": rl["unit"], "frac": rl["frac"]}
    return res


def sub_fft_routes(q, ctx, caps, samples, seed, n, m, num_blocks, out, flush, reps=2):
    """The transform routes on the laser stream (the paper's FP64 circulant FFT, the FP32 segmented
    FFT and the exact number-theoretic transform) with their rounding evidence."""
    res = {"workload": "laser stream, n=2^16, standard form"}
    for name in ("ntt", "fft64", "fft32_seg"):
        kms, cms, st = _time_extract(q, ctx, samples, n, m, seed, 0, ALGOS[name], num_blocks, out, reps=reps,
                                     flush=flush)
        rl = roofline_for(name, num_blocks, m, n, kms, fft32_plan(q, st), caps=caps)
        res[name] = {"kernel_ms": kms, "call_ms": cms, "gbps": num_blocks * m / (cms / 1e3) / 1e9,
                     "worst_round_err": st["worst_fft_round_err"] if name != "ntt" else 0.0, "roofline": rl}
    return res


def sub_uneven(q, ctx, caps, routes=("auto", "fft32_seg", "fft64")):
    """Config 5: 10,000 uneven requests (n log-uniform in [2^12, 2^22], m/n uniform in [0.5, 0.9],
    per-request seeds, raw Bernoulli(p), p uniform in [0.45, 0.55]), one graph replay per call:
    AUTO's tuned schedule, and the FP32 segmented and FP64 transforms on every request."""
    import torch

    b = W.uneven_batch()
    raw = torch.from_numpy(b["raw"]).cuda()
    seeds = torch.from_numpy(b["seeds"]).cuda()
    out = torch.empty((b["out_bits"] + 7) // 8 + 8, dtype=torch.uint8, device="cuda")
    reqs = [(raw.data_ptr(), int(b["raw_off"][i]), int(b["n"][i]), int(b["m"][i]),
             seeds.data_ptr() + int(b["seed_off"][i]), 0, out.data_ptr(), int(b["out_off"][i]))
            for i in range(b["n"].size)]
    n, m = b["n"].astype(np.float64), b["m"].astype(np.float64)
    res = {"workload": f"{n.size} uneven requests, n log-uniform in [2^12, 2^22], m/n uniform in [0.5, 0.9], "
                       "per-request standard seeds, Bernoulli(p) raw bits", "unit": UNIT,
           "output_gbit": float(m.sum()) / 1e9, "bitmacs": float((m * n).sum())}
    stream = torch.cuda.current_stream()
    pk = measured_peaks()
    for route in routes:
        algo = ALGOS[route]
        q.qrng_extract_batch(ctx, reqs, algo=algo)  # plan (and for AUTO the class tuning), capture, first run
        q.qrng_synchronize(ctx)
        q.qrng_reset_stats(ctx)
        q.qrng_set_timing(ctx, True)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        q.qrng_extract_batch(ctx, reqs, algo=algo)  # one graph replay
        e.record(stream)
        e.synchronize()
        q.qrng_synchronize(ctx)
        st = q.qrng_get_stats(ctx)
        q.qrng_set_timing(ctx, False)
        ms = a.elapsed_time(e)
        r = {"ms": ms, "gbps": res["output_gbit"] / (ms / 1e3), "graph_ms": st["batch_graph_ms"],
             "kernels_per_call": st["last_kernels"], "requests": st["batch_requests"],
             "worst_round_err": st["worst_fft_round_err"],
             "direct_equivalent_tbitmac_per_s": res["bitmacs"] / (ms / 1e3) / 1e12}
        if st["batch_requests"]["direct"] and st["batch_direct_ms"] > 0:
            ach = st["batch_direct_bitmacs"] / (st["batch_direct_ms"] / 1e3) / 1e12
            r["direct_part"] = {"ms": st["batch_direct_ms"], "achieved": ach, "unit": "Tbit-MAC/s",
                                "frac": ach / alu_peak_tbitmac(caps), "bound": "alu"}
        if st["batch_transform_ms"] > 0:
            hb = hbm_record(st["batch_transform_bytes"], st["batch_transform_ms"])
            r["transform_part"] = {"ms": st["batch_transform_ms"], "hbm_achieved": hb["achieved"],
                                   "hbm_frac": hb["frac"], "unit": "GB/s"}
        res[route] = r
    return res


def run_subrecords(q, ctx, local, caps, flush, laser):
    subs = {}
    subs["single"] = clocked(local, sub_single, q, ctx, caps)
    subs["histogram"] = clocked(local, sub_histogram, q, ctx, flush)
    subs["fft_routes"] = clocked(local, sub_fft_routes, q, ctx, caps, *laser, flush)
    subs["tc"] = clocked(local, sub_tc, q, ctx, caps, flush)
    subs["sweep"] = clocked(local, sub_sweep, q, ctx, caps, flush)
    subs["uneven"] = clocked(local, sub_uneven, q, ctx, caps)
    return subs


def run_sweep(args):
    """Block-length sweep (the paper's Fig. 6 question on GB300): a fixed 2^30-bit Bernoulli(0.5)
    stream, n = 2^10 .. 2^24, m = 0.75 n, modified form, one (n-1)-bit seed per n; every algorithm
    of --sweep-algos at every n."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    caps = device_caps()
    c = W.CFG3
    raw = torch.from_numpy(W.random_bits(c["stream_bits"], c["raw_seed"])).cuda()
    out = torch.empty(c["stream_bits"] // 8, dtype=torch.uint8, device="cuda")
    rows = []
    for n in c["n_list"]:
        m = int(n * c["ratio"])
        B = c["stream_bits"] // n
        seed = torch.from_numpy(W.random_bits(n - 1, c["seed_seed"] + n.bit_length() - 1)).cuda()
        row = {"n": n, "m": m, "blocks": B}
        for name in args.sweep_algos.split(","):
            try:
                kms, cms, st = _time_extract(q, ctx, raw, n, m, seed, 1, ALGOS[name], B, out, reps=2)
                plan = (q.qrng_karatsuba_plan(ctx, n, m, 1, B) if name == "gemm_karatsuba"
                        else fft32_plan(q, st) if name == "fft32_seg" else None)
                rl = roofline_for(name, B, m, n - m, kms, plan, caps, n=n)
                row[name] = {"kernel_ms": kms, "call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9,
                             "frac": rl.get("frac"), "bound": rl.get("bound")}
                if name.startswith("fft"):
                    row[name]["worst_round_err"] = st["worst_fft_round_err"]
            except q.QrngError as e:
                row[name] = {"unsupported": str(e)}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr)
    ctx.close()
    return {"workload": "block-length sweep: 2^30-bit Bernoulli(0.5) stream, n = 2^10..2^24, m = 0.75n, "
                        "modified form", "unit": UNIT, "data": "synthetic", "rows": rows}


def run_forms(args):
    """Standard (n+m-1-bit seed) vs modified ((A, I_m), n-1-bit seed) Toeplitz hashing at equal n and
    m on the same 2^30-bit stream, for every algorithm: the comparison the paper leaves as future work."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    c = W.CFG3
    raw = torch.from_numpy(W.random_bits(c["stream_bits"], c["raw_seed"])).cuda()
    out = torch.empty(c["stream_bits"] // 8, dtype=torch.uint8, device="cuda")
    rows = []
    for n in (1 << 12, 1 << 16, 1 << 20):
        for ratio in (0.5, 0.75):
            m = int(n * ratio)
            B = c["stream_bits"] // n
            row = {"n": n, "m": m, "blocks": B}
            for form, fname in ((0, "standard"), (1, "modified")):
                L = n + m - 1 if form == 0 else n - 1
                seed = torch.from_numpy(W.random_bits(L, 99)).cuda()
                row[fname] = {"seed_bits": L}
                for name in ("direct", "gemm_tc", "gemm_fp4", "gemm_fp4_pair", "gemm_karatsuba", "ntt"):
                    kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, form, ALGOS[name], B, out, reps=2)
                    row[fname][name] = {"call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr)
    ctx.close()
    return {"workload": "standard vs modified Toeplitz on a 2^30-bit stream", "unit": UNIT, "rows": rows}


def run_long(args):
    """64 blocks of n = 2^22 raw bits, m = 0.75 n, modified form, one seed: a 2^28-bit stream on the
    long-block route (--algo, default ntt), small enough for a profiler capture."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    c = W.CFG3
    n, B = 1 << 22, 64
    m = int(n * c["ratio"])
    raw = torch.from_numpy(W.random_bits(n * B, c["raw_seed"])).cuda()
    seed = torch.from_numpy(W.random_bits(n - 1, c["seed_seed"] + 22)).cuda()
    out = torch.empty(m * B // 8, dtype=torch.uint8, device="cuda")
    name = "ntt" if args.algo == "auto" else args.algo
    kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, 1, ALGOS[name], B, out, reps=args.steps, warmup=args.warmup)
    ctx.close()
    return {"workload": "64 blocks of 2^22 bits, m = 0.75n, modified form", "algo": name, "unit": UNIT,
            "call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9, "data": "synthetic"}


def _standalone(fn):
    """One sub-record workload on its own (--workload single|tc|uneven|hist)."""
    def run(args):
        import torch

        import paper_2011_04130_gb300 as q

        torch.cuda.set_device(0)
        ctx = q.Context(0)
        caps = device_caps()
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        if fn is sub_uneven:
            routes = ("auto", "ntt", "fft64", "fft32_seg", "direct") if args.algo == "all" else (args.algo,)
            res = clocked(0, fn, q, ctx, caps, routes)
        elif fn is sub_histogram:
            res = clocked(0, fn, q, ctx, flush)
        else:
            res = clocked(0, fn, q, ctx, caps, flush) if fn is not sub_single else clocked(0, fn, q, ctx, caps)
        ctx.close()
        return res
    return run


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload != "laser":
        res = {"sweep": run_sweep, "forms": run_forms, "long": run_long, "single": _standalone(sub_single),
               "tc": _standalone(sub_tc), "uneven": _standalone(sub_uneven),
               "hist": _standalone(sub_histogram)}[args.workload](args)
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
