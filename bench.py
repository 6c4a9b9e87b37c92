"""Benchmark of the QRNG post-processing hot path on GB300.

Workload (the laser-phase-noise stream): 2^26 uint8 ADC samples ~ clip(round(N(128, 16^2))),
whose bytes are also the 2^29-bit raw stream; blocks of n = 2^16 bits; m = floor(n H_modify / 8)
from the corrected min-entropy (eps = 1e-6); one standard Toeplitz seed of n+m-1 bits shared by
every block. One step = min-entropy estimate (histogram + FP64 finaliser, report read back)
+ extraction of all 8192 blocks. Metric: extracted output Gbit/s, bit-exact.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
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
# integer-pipe peak of the direct kernel: 64 LOP3/clk/SM (measured on GB300), 32 bit-products per
# LOP3, 152 SMs, 2070 MHz maximum SM clock
LOP3_PER_CLK_SM = 64
SMS = 152
SM_MAX_MHZ = 2070.0
ALU_PEAK_TBITMAC = LOP3_PER_CLK_SM * 32 * SMS * SM_MAX_MHZ * 1e6 / 1e12


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
    p.add_argument("--workload", default="laser",
                   choices=["laser", "single", "sweep", "tc", "uneven", "forms", "long"],
                   help="laser: the headline stream (default); single: one 4096-bit block; sweep: block-length "
                        "sweep on a 2^30-bit stream; tc: m=6144, n=8192, 4096 blocks; uneven: 10,000 requests; "
                        "long: 64 blocks of 2^22 bits (the transform route's profiling case)")
    p.add_argument("--sweep-algos", default="direct,gemm_tc,gemm_fp4,gemm_fp4_pair,gemm_karatsuba,ntt,fft64",
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
        rep = q.qrng_minentropy(ctx, samples, bits=bits, eps=eps, stream=stream)
        m = q.qrng_output_length(n, rep["h_modify"], bits, 1.0)
        q.qrng_toeplitz_extract(ctx, samples, n, m, seed, q.QRNG_FORM_STANDARD, a, num_blocks, out, stream=stream)
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

    plan = q.qrng_karatsuba_plan(ctx, n, m, q.QRNG_FORM_STANDARD, num_blocks) if used_algo == "gemm_karatsuba" else None
    roofline = roofline_for(used_algo, num_blocks, m, n, kernel_ms, plan)

    # end to end through the host-buffer entry point (pinned host memory, copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        pin_samples = torch.from_numpy(samples_h).pin_memory()
        pin_seed = torch.from_numpy(seed_h).pin_memory()
        pin_out = torch.empty(num_blocks * n // 8, dtype=torch.uint8).pin_memory()
        e_ms = []
        for i in range(args.warmup + args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m2, nb2, _ = q.qrng_postprocess_host(ctx, pin_samples, samples_h.size, bits, eps, 1.0, n, pin_seed,
                                                 2 * n - 1, q.QRNG_FORM_STANDARD, algo, pin_out, pin_out.numel(),
                                                 stream=stream)
            b.record(stream)
            b.synchronize()
            if i >= args.warmup:
                e_ms.append(a.elapsed_time(b))
        et = reduce_max(sum(e_ms), world, dev)
        e2e = {"value": job_throughput(world, nb2 * m2, len(e_ms), et), "unit": UNIT,
               "h2d_bytes_per_step": int(samples_h.nbytes + (q.qrng_seed_bits(n, m2, 0) + 7) // 8),
               "d2h_bytes_per_step": int((nb2 * m2 + 7) // 8 + 112), "ms_per_step": et / len(e_ms)}

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
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(samples_h, seed_h, n, m, eps)
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


def roofline_for(algo, num_blocks, m, n, kernel_ms, plan=None):
    """Roofline of the dominant (extraction) kernel from its algorithmic work and live event time."""
    if algo == "direct":
        achieved = num_blocks * m * n / (kernel_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TBITMAC, "unit": "Tbit-MAC/s",
                "frac": achieved / ALU_PEAK_TBITMAC,
                "traffic": captured_traffic("direct_kernel", "k_direct.cu", num_blocks),
                "kernel": "direct_kernel<32>", "kernel_ms": kernel_ms,
                "peak_source": "derived: 64 LOP3/clk/SM x 32 bit-MACs x 152 SMs x 2070 MHz"}
    if algo == "gemm_tc":
        pk = measured_peaks()
        peak = 2.0 * pk["bf16_tflops"]  # FP8 dense = bf16 measured x nominal ratio 4.5/2.25
        achieved = 2.0 * num_blocks * m * n / (kernel_ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": captured_traffic("gemm_tc_kernel", "k_gemm_tc.cu", num_blocks),
                "kernel": "gemm_tc_kernel (tcgen05 kind::f8f6f4)", "kernel_ms": kernel_ms,
                "peak_source": "FP8 = 2 x bf16 burst " + pk["source"]}
    if algo in ("gemm_fp4", "gemm_fp4_pair"):
        pk = measured_peaks()
        peak = 6.0 * pk["bf16_tflops"]  # FP4 dense = bf16 measured x nominal ratio 13.5/2.25
        achieved = 2.0 * num_blocks * m * n / (kernel_ms / 1e3) / 1e12
        pair = algo == "gemm_fp4_pair"
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (captured_traffic("gemm_pair_kernel", "k_gemm_pair.cu", num_blocks) if pair
                            else captured_traffic("gemm_fp4_kernel", "k_gemm_tc.cu", num_blocks)),
                "kernel": ("gemm_pair_kernel (tcgen05 cta_group::2 kind::mxf4, block scale 2^0)" if pair
                           else "gemm_tc_kernel<fp4> (tcgen05 kind::mxf4, block scale 2^0)"),
                "kernel_ms": kernel_ms, "peak_source": "FP4 = 6 x bf16 burst " + pk["source"]}
    if algo == "gemm_karatsuba":
        # the product kernel's own work: 3^L dense sub-products of mq x kq per block (the plan the
        # library ran, from qrng_karatsuba_plan)
        pk = measured_peaks()
        peak = 6.0 * pk["bf16_tflops"]
        plan = plan or {}
        flops = 2.0 * num_blocks * plan["groups"] * plan["mq"] * plan["kq"]
        achieved = flops / (kernel_ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": captured_traffic("gemm_pair_kara_kernel", "k_gemm_pair.cu", num_blocks),
                "kernel": "gemm_pair_kernel<kKara> (tcgen05 cta_group::2 kind::mxf4 on the block-Karatsuba "
                          "sub-products)", "kernel_ms": kernel_ms,
                "plan": plan, "equivalent_plain_tflops": 2.0 * num_blocks * m * n / (kernel_ms / 1e3) / 1e12,
                "peak_source": "FP4 = 6 x bf16 burst " + pk["source"]}
    return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
            "kernel_ms": kernel_ms}


def cpu_baseline(samples_h, seed_h, n, m, eps, blocks=2):
    """The oracle as it stands, one thread: min-entropy of the whole stream plus the full
    Toeplitz hash of `blocks` blocks of it."""
    import oracle

    t0 = time.perf_counter()
    rep = oracle.minentropy(samples_h, 8, eps)
    m_or = oracle.output_length(n, rep["h_modify"], 8, 1.0)
    seed_o = seed_h[: (n + m_or - 1 + 7) // 8].copy()
    raw = samples_h[: blocks * n // 8].copy()
    oracle.toeplitz_blocks(raw, n, m_or, seed_o, 0, blocks)
    dt = time.perf_counter() - t0
    return {"value": blocks * m_or / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"min-entropy of all {samples_h.size} samples + full hash of {blocks} of "
                      f"{samples_h.size * 8 // n} blocks (n={n}, m={m_or})", "seconds": dt}


def run_reference(args, world, rank):
    """The CPU oracle on the same workload, each step a bounded sample (min-entropy of the full
    stream + one block's full hash)."""
    if rank != 0:
        return None
    import oracle

    oracle.build()
    c = W.CFG2
    n, eps = c["n"], c["eps"]
    samples_h = W.adc_samples(c["samples"], c["sample_seed"])
    seed_h = W.random_bits(2 * n - 1, c["seed_seed"])
    times, bits_out = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rep = oracle.minentropy(samples_h, 8, eps)
        m = oracle.output_length(n, rep["h_modify"], 8, 1.0)
        blk = i % (samples_h.size * 8 // n)
        raw = samples_h[blk * n // 8:(blk + 1) * n // 8].copy()
        oracle.toeplitz(raw, n, m, seed_h[: (n + m - 1 + 7) // 8].copy(), 0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            bits_out += m
    total = sum(times)
    value = bits_out / total / 1e9
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8 (one byte per bit)",
            "data": "synthetic",
            "config": {"workload": "laser-phase-noise stream: 2^26 uint8 ADC samples, n=2^16, one shared seed",
                       "n": n, "m": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: min-entropy of all 2^26 samples + the full hash of one block"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


ALGOS = {"auto": 0, "direct": 1, "gemm_tc": 2, "fft64": 3, "fft32_seg": 4, "ntt": 5, "gemm_fp4": 6,
         "gemm_fp4_pair": 7, "gemm_karatsuba": 8}


def _time_extract(q, ctx, raw, n, m, seed, form, algo, blocks, out, reps, warmup=1):
    """Mean CUDA-event time (ms) of the main extraction kernel and of the whole call."""
    import torch

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        q.qrng_toeplitz_extract(ctx, raw, n, m, seed, form, algo, blocks, out, stream=stream)
    torch.cuda.synchronize()
    q.qrng_reset_stats(ctx)
    q.qrng_set_timing(ctx, True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        q.qrng_toeplitz_extract(ctx, raw, n, m, seed, form, algo, blocks, out, stream=stream)
    b.record(stream)
    b.synchronize()
    q.qrng_synchronize(ctx)
    st = q.qrng_get_stats(ctx)
    q.qrng_set_timing(ctx, False)
    return st["timed_ms"] / max(1, st["timed_launches"]), a.elapsed_time(b) / reps, st


def run_sweep(args):
    """Block-length sweep (the paper's Fig. 6 question on GB300): a fixed 2^30-bit Bernoulli(0.5)
    stream, n = 2^10 .. 2^24, m = 0.75 n, modified form, one (n-1)-bit seed per n."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
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
                row[name] = {"kernel_ms": kms, "call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9}
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


def run_tc(args):
    """One standard seed, m = 6144, n = 8192, 4096 blocks: tensor-core product vs the direct kernel."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    c = W.CFG4
    n, m, B = c["n"], c["m"], c["blocks"]
    raw = torch.from_numpy(W.random_bits(n * B, c["raw_seed"])).cuda()
    seed = torch.from_numpy(W.random_bits(n + m - 1, c["seed_seed"])).cuda()
    out = torch.empty(m * B // 8, dtype=torch.uint8, device="cuda")
    res = {"workload": "m=6144, n=8192, 4096 blocks, one standard seed", "unit": UNIT, "data": "synthetic"}
    pk = measured_peaks()
    for name in ("gemm_karatsuba", "gemm_fp4_pair", "gemm_fp4", "gemm_tc", "direct"):
        kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, 0, ALGOS[name], B, out, reps=args.steps)
        res[name] = {"kernel_ms": kms, "call_ms": cms, "gbps": B * m / (cms / 1e3) / 1e9}
        if name == "gemm_karatsuba":
            plan = q.qrng_karatsuba_plan(ctx, n, m, 0, B)
            tf = 2.0 * plan["groups"] * plan["mq"] * plan["kq"] * B / (kms / 1e3) / 1e12
            res[name].update({"plan": plan, "tflops": tf, "frac_of_peak": tf / (6.0 * pk["bf16_tflops"]),
                              "peak_source": f"6 x bf16 burst {pk['source']}"})
        elif name.startswith("gemm"):
            tf = 2.0 * m * n * B / (kms / 1e3) / 1e12
            ratio = 6.0 if name.startswith("gemm_fp4") else 2.0  # nominal FP4 / FP8 dense rates over bf16
            res[name].update({"tflops": tf, "frac_of_peak": tf / (ratio * pk["bf16_tflops"]),
                              "peak_source": f"{ratio:g} x bf16 burst {pk['source']}"})
    ctx.close()
    return res


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


def run_single(args):
    """One 4096-bit block, m = 2048, plus the min-entropy of 65,536 samples: latency."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    c = W.CFG1
    samples = torch.from_numpy(W.adc_samples(c["samples"], c["sample_seed"])).cuda()
    n, m = c["n"], c["m"]
    raw = torch.from_numpy(W.random_bits(n, c["raw_seed"])).cuda()
    seed = torch.from_numpy(W.random_bits(n + m - 1, c["seed_seed"])).cuda()
    out = torch.empty(m // 8, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        q.qrng_minentropy(ctx, samples, bits=8, eps=c["eps"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q.qrng_minentropy(ctx, samples, bits=8, eps=c["eps"])
    ent_us = (time.perf_counter() - t0) / args.steps * 1e6
    kms, cms, _ = _time_extract(q, ctx, raw, n, m, seed, 0, ALGOS["direct"], 1, out, reps=args.steps)
    ctx.close()
    return {"workload": "65,536 samples + one block n=4096, m=2048", "minentropy_us_host": ent_us,
            "extract_kernel_us": kms * 1e3, "extract_call_us": cms * 1e3, "gbps": m / (cms / 1e3) / 1e9}


def run_uneven(args):
    """10,000 uneven requests (n log-uniform, m/n uniform in [0.5, 0.9], per-request seeds, raw
    Bernoulli(p), p uniform in [0.45, 0.55]) in one persistent launch under a CUDA graph."""
    import torch

    import paper_2011_04130_gb300 as q

    torch.cuda.set_device(0)
    ctx = q.Context(0)
    c = W.CFG5
    n, m, p = W.uneven_requests(c["requests"], c["seed"], c["log2n_lo"], args.uneven_max_log2n, c["rho_lo"],
                                c["rho_hi"], c["p_lo"], c["p_hi"])
    raw_off = np.concatenate([[0], np.cumsum(((n + 31) // 32) * 32)[:-1]])
    total_raw = int(raw_off[-1] + n[-1] + 64)
    seed_off = np.concatenate([[0], np.cumsum(((n + m + 7) // 8) * 8)[:-1]])  # byte-aligned seeds
    out_off = np.concatenate([[0], np.cumsum(m)[:-1]])
    g = W.rng(c["seed"] + 7)
    raw = torch.empty((total_raw + 7) // 8, dtype=torch.uint8, device="cuda")
    # raw bits per request are Bernoulli(p_r): fill in chunks of requests to bound host memory
    for i in range(len(n)):
        bits = W.random_bits(int(n[i]), 10_000 + i, float(p[i]))
        raw[raw_off[i] // 8:raw_off[i] // 8 + bits.size] = torch.from_numpy(bits).cuda()
    seeds = torch.from_numpy(g.integers(0, 256, int(seed_off[-1] + (n[-1] + m[-1] + 7) // 8), dtype=np.uint8)).cuda()
    out = torch.empty(int((out_off[-1] + m[-1] + 7) // 8 + 8), dtype=torch.uint8, device="cuda")
    table = (q.Request * len(n))()
    for i in range(len(n)):
        table[i] = q.Request(raw.data_ptr(), int(raw_off[i]), int(n[i]), int(m[i]),
                             seeds.data_ptr() + int(seed_off[i]) // 8, 0, out.data_ptr(), int(out_off[i]))
    lib = q.load_library()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def call():
        ctx.check(lib.qrng_extract_batch(ctx.handle, table, len(n), ALGOS[args.algo], sp), "qrng_extract_batch")

    call()  # capture + first run
    q.qrng_synchronize(ctx)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record(stream)
    for _ in range(max(1, args.steps)):
        call()  # graph replay (the request table is hashed on the host each call)
    b.record(stream)
    b.synchronize()
    host_ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    q.qrng_synchronize(ctx)
    ms = a.elapsed_time(b) / max(1, args.steps)
    bitmacs = float(np.sum(m.astype(np.float64) * n))
    st = q.qrng_get_stats(ctx)
    ctx.close()
    res = {"workload": f"{len(n)} uneven requests, n log-uniform in [2^12, 2^{args.uneven_max_log2n:g}], "
                       "m/n uniform in [0.5, 0.9], per-request seeds", "algo": args.algo, "ms": ms,
           "host_wall_ms": host_ms, "output_gbit": float(np.sum(m)) / 1e9,
           "gbps": float(np.sum(m)) / (ms / 1e3) / 1e9, "kernels_per_call": st["last_kernels"],
           "route": q.ALGO_NAMES.get(st["last_algo"], "mixed") if st["last_algo"] else "mixed (direct + ntt)",
           "direct_equivalent_tbitmac_per_s": bitmacs / (ms / 1e3) / 1e12}
    if st["last_algo"] == q.QRNG_ALGO_DIRECT:
        res["frac_of_lop3_peak"] = res["direct_equivalent_tbitmac_per_s"] / ALU_PEAK_TBITMAC
    return res


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload != "laser":
        res = {"sweep": run_sweep, "tc": run_tc, "single": run_single, "uneven": run_uneven,
               "forms": run_forms, "long": run_long}[args.workload](args)
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
