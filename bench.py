"""Benchmark: detector-samples/s of the TOD hot path on the 25-spaxel IFU workload.

One step = gateau_run over the whole 20-minute raster of the 25-spaxel IFU
(5x5 at 15", 347 channels, 3000 spectral points, 192 000 samples at 160 Hz,
1024^2 PWV screen, 128x128x3000 source cube): 1.666e9 detector samples, white
and pink noise on, output [t][pixel][channel] float32 (6.66 GB) in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs under torchrun: every rank simulates
its own independent copy of the workload (weak scaling, no collective on the data
path).  --impl reference times the FP64 oracle on the host cores instead.

    python bench.py --record-traffic RAW.csv --traffic-samples S

writes the fused kernel's DRAM traffic per full launch into the traffic record from
an ncu capture (`ncu -i report --page raw --csv`) of a run over the first S samples;
the bench line reports it only while the kernel source is the one captured.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_23305_b300 import workloads as W  # noqa: E402

METRIC = "detector-samples/s (pix·chan·t) split-BF16 vs plain FP32 GPU; serving p50/p99 latency"
UNIT = "detector-samples/s"
WORKLOAD = "ifu25_raster_20min: 25 spaxels (5x5, 15\"), 347 filterbank channels R=500, 3000 freq 220-440 GHz, " \
           "192000 samples @160 Hz, 1024^2 PWV screen, 128x128x3000 source cube, 6-stage cascade, white+pink noise"
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "fused_bf16x3_traffic.json")
FUSED_SRC = os.path.join(ROOT, "paper_2604_23305_b300", "csrc", "kernels_fused.cu")
FULL_SAMPLES = 192000        # samples of the ifu25 scan (one full launch)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["bf16_tflops"], p["hbm_gbs"], "measured"
    except Exception:
        return 1800.0, 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms from before the warm-up steps (the
    tool takes a moment to start) and kept for the timed region: mark(True) / mark(False) bracket it,
    and summary() uses the samples taken between the two marks (those within 0.3 s of the window when
    it holds none, e.g. a timed region shorter than one sampling period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.window = [None, None]

    def mark(self, start: bool):
        self.window[0 if start else 1] = time.monotonic()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        t0, t1 = self.window
        lines = []
        if t0 is not None and t1 is not None:
            for pad in (0.1, 0.3):                   # the window, then a sampling period or three around it
                lines = [ln for t, ln in self.lines if t0 - (pad - 0.1) <= t <= t1 + pad]
                if lines:
                    break
        if not lines:
            lines = [ln for _, ln in self.lines]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def fused_source_hash() -> str:
    return hashlib.sha256(open(FUSED_SRC, "rb").read()).hexdigest()[:16]


def traffic_from_record():
    """DRAM bytes per full launch of the fused kernel from the traffic record, or None when the
    record was taken on another kernel source (the counters no longer describe this kernel)."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
        if rec.get("kernel_source_sha256_16") == fused_source_hash():
            return float(rec["dram_bytes_per_full_launch"])
    except Exception:
        pass
    return None


def record_traffic(raw_csv: str, samples: int, command: str) -> dict:
    """Parse the raw page of an ncu capture (one row per launch) and write the traffic record:
    the fused launches' dram__bytes_read.sum + dram__bytes_write.sum, scaled from the captured
    samples to a full launch (the kernel's work is linear in the samples: tiles x channel groups)."""
    import csv
    with open(raw_csv, newline="") as f:
        rows = list(csv.reader(f))
    head = rows[0]
    col = {name: i for i, name in enumerate(head)}
    units = rows[1]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    tscale = {"nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0, "ns": 1e-9, "us": 1e-6, "ms": 1e-3}

    def val(r, name, table):
        return float(r[col[name]].replace(",", "")) * table.get(units[col[name]], 1.0)

    launches = [r for r in rows[2:] if "fused_bf16x3" in r[col["Kernel Name"]]]
    if not launches:
        raise SystemExit("no fused_bf16x3 launch in " + raw_csv)
    rd = [val(r, "dram__bytes_read.sum", scale) for r in launches]
    wr = [val(r, "dram__bytes_write.sum", scale) for r in launches]
    dur = [val(r, "gpu__time_duration.sum", tscale) for r in launches]
    per = (sum(rd) + sum(wr)) / len(launches)
    rec = {"kernel": "fused_bf16x3_kernel", "kernel_source_sha256_16": fused_source_hash(),
           "captured_samples": samples, "full_samples": FULL_SAMPLES, "launches": len(launches),
           "dram_read_bytes": sum(rd) / len(launches), "dram_write_bytes": sum(wr) / len(launches),
           "duration_s": sum(dur) / len(launches),
           "dram_bytes_per_full_launch": per * FULL_SAMPLES / samples, "command": command}
    with open(TRAFFIC_RECORD, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def oracle_rate(sc, nt_sample: int, white=True, pink=True):
    """FP64 oracle throughput (detector samples/s) on the first nt_sample samples, all spaxels."""
    from oracle import gateau_oracle as O
    t = time.perf_counter()
    O.simulate(sc, 0, nt_sample, white=white, pink=pink)
    dt = time.perf_counter() - t
    return W.detector_samples(sc, nt_sample) / dt, dt


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(sc, budget_s=12.0, workload="ifu25"):
    """The FP64 oracle as it stands on the host: once with numpy's default BLAS threads (only the
    matrix products of Eqs. 16-17 run on them; everything else runs on one core), once in a fresh
    process with BLAS held to one thread."""
    probe = 16
    r0, dt0 = oracle_rate(sc, probe)
    nt = max(probe, min(sc["nt_total"], int(probe * budget_s / max(dt0, 1e-3)) // 4 * 4))
    rate, dt = oracle_rate(sc, nt)
    nt1 = max(probe, nt // 2 // 4 * 4)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"from paper_2604_23305_b300 import workloads as W; "
            f"r, dt = bench.oracle_rate(W.scenario({workload!r}, **bench.replica_seeds(0)), {nt1}); print(r, dt)")
    try:
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        rate1, dt1 = (float(x) for x in res.stdout.split()[-2:])
        single = {"value": rate1, "unit": UNIT, "cores": 1,
                  "sample": f"first {nt1} samples, BLAS held to one thread (fresh process), {dt1:.1f} s"}
    except Exception as exc:                       # reported, not hidden
        single = {"error": repr(exc)}
    return {"value": rate, "unit": UNIT, "cores": blas_threads(), "nproc": os.cpu_count(), "kind": "oracle",
            "threads": "BLAS threads for the matrix products of Eqs. 16-17 (= cores); the rest on one core",
            "sample": f"first {nt} samples of the scan (all 25 spaxels x 347 channels, white+pink noise), "
                      f"FP64 numpy oracle, {dt:.1f} s",
            "single_thread": single}


def serving_leg(n_requests: int, seed: int = 2, budget_bytes: float = 120e9, max_active: int = 16,
                chunk_samples: int = 32768, max_chunk_bytes: int = 256 << 20, builders: int = 6,
                shared_launches: bool = False):
    """The serving workload: n_requests simulations (hexagonal IFUs of 1-61 spaxels, 100-347
    channels, 1000-6000 spectral points, 10 s - 10 min at 160 Hz) through the native server,
    admitted by a device-memory budget.  First all requests arrive at once (saturated: the
    server's capacity in requests/s), then Poisson arrivals at 0.75 x that capacity; latency =
    arrival -> last chunk of TOD on the host.  shared_launches: chunks in rounds whose
    contractions share persistent fused launches, instead of one launch sequence per request."""
    from paper_2604_23305_b300 import Plan
    from paper_2604_23305_b300.serve import Server, ServingInputs, build_requests, serving_requests

    shapes = serving_requests(n_requests, seed)
    scs, reqs = build_requests(shapes, ServingInputs(seed), chunk_samples)
    # tile autotuner: one plan per channel class (16-channel blocks) is tuned before the runs; every
    # request's plan then takes its class's choice from the cache when it is created
    t = time.perf_counter()
    classes, choices = {}, {}
    for i, r in enumerate(shapes):
        classes.setdefault((r["n_ch"] + 15) // 16, i)
    for c, i in sorted(classes.items()):
        p = Plan(scs[i], precision="bf16x3", device_inputs=False)
        ch = p.autotune(nt_sample=1024)
        choices[c] = (ch["n_groups"], ch["ring_b"])
        p.close()
    tune_s = time.perf_counter() - t

    def make(i):
        p = Plan(scs[i], precision="bf16x3", device_inputs=False)
        p.autotune(nt_sample=1024)                                  # from the cache
        return p
    srv = Server(int(budget_bytes), max_active=max_active, chunk_samples=chunk_samples,
                 max_chunk_bytes=max_chunk_bytes, n_streams=max_active, n_builders=builders,
                 shared_launches=shared_launches)
    srv.run(reqs[:4], make)                                       # warm-up (not reported)
    sat = srv.run(reqs, make)
    capacity = sat["n_done"] / sat["makespan_s"]
    rate = 0.75 * capacity
    rng = np.random.default_rng(seed + 1)
    arrivals = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0 / rate, n_requests - 1))])
    st = srv.run([dict(r, arrival_s=float(a)) for r, a in zip(reqs, arrivals)], make)
    srv.close()
    keys = ("p50_latency_s", "p99_latency_s", "mean_latency_s", "max_latency_s", "makespan_s", "throughput",
            "detector_samples", "peak_bytes", "peak_active", "overlap", "n_done", "n_failed", "rounds", "mean_round")
    out = {k: st[k] for k in keys}
    out.update(scheduler="shared persistent launches in rounds" if shared_launches else "a stream per request",
               autotune={"classes": len(classes), "seconds": tune_s,
                         "choices": {str(16 * c): list(v) for c, v in sorted(choices.items())}},
               requests=n_requests, budget_bytes=int(budget_bytes), max_active=max_active, plan_builders=builders,
               chunk_samples=chunk_samples, capacity_req_per_s=capacity, arrival_rate_req_per_s=rate,
               saturated={k: sat[k] for k in ("makespan_s", "throughput", "p50_latency_s", "p99_latency_s",
                                              "overlap")},
               throughput_unit="detector-samples/s", latency="arrival -> last chunk of TOD in host memory",
               workload="hex IFU R=0..4 (1-61 spaxels), 100-347 ch, 1000-6000 freq, 10 s-10 min at 160 Hz, "
                        "Poisson arrivals at 0.75 x measured capacity, seed 2")
    return out


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seeds(rank: int) -> dict:
    """Each rank simulates an independent copy of the workload: its own screen and noise seeds."""
    return dict(seed=rank, noise_seed=1 + rank)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the job's time); dist is torch.distributed or None."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, per_step: float, steps: int, elapsed_s: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * per_step * steps / elapsed_s


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    sc = W.scenario(args.workload)
    nt_step = args.ref_samples
    for _ in range(args.warmup):
        oracle_rate(sc, nt_step)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(sc, nt_step)
        times.append(dt)
    per_step = W.detector_samples(sc, nt_step)
    value = per_step * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"FP64 oracle on the first {nt_step} samples (all spaxels)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": blas_threads(),
                             "sample": f"first {nt_step} samples of the scan per step, all 25 spaxels x 347 channels"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ifu25")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp32-steps", type=int, default=1)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--ref-samples", type=int, default=48)
    ap.add_argument("--nt", type=int, default=None, help="shorter scan (profiling runs); default: the whole scan")
    ap.add_argument("--serving-requests", type=int, default=256)
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-kelvin", action="store_true")
    ap.add_argument("--skip-tk", action="store_true")
    ap.add_argument("--skip-prep", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default fused tiles")
    ap.add_argument("--skip-graph", action="store_true")
    ap.add_argument("--record-traffic", default=None, metavar="RAW_CSV")
    ap.add_argument("--traffic-samples", type=int, default=16384)
    ap.add_argument("--traffic-command", default="")
    args = ap.parse_args()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic, args.traffic_samples, args.traffic_command)))
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2604_23305_b300 import Plan

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def ranks_max(x: float) -> float:
        return max_over_ranks(x, dist, "cuda")

    sc = W.scenario(args.workload, nt_total=args.nt, **replica_seeds(rank))
    nt = sc["nt_total"]
    per_step = W.detector_samples(sc)
    # plan build, reported apart from the steps: inputs uploaded, then the FP64 plan (cascade collapse,
    # filter matrices, reference spectrum, operand tiling, pink design) on the host and the device
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    plan = Plan(sc, precision=args.precision, white=True, pink=True)
    plan.prepare()
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t_build)
    tune = plan.autotune(nt_sample=4096) if args.precision == "bf16x3" and not args.no_autotune else None
    out = torch.empty((nt, plan.n_pix, plan.n_ch), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    clk = ClockSampler(local).__enter__()          # running before the warm-up; the timed region is marked
    for _ in range(max(args.warmup, 3)):
        plan.run(0, nt, out)
    torch.cuda.synchronize()
    plan.status()
    plan.get_timing()
    plan.set_timing(True)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clk.mark(True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(0, nt, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk.mark(False)
    barrier()
    clk.__exit__(None, None, None)
    elapsed_s = ranks_max(ev0.elapsed_time(ev1) / 1e3)
    phase_ms, runs, launches = plan.get_timing()
    plan.set_timing(False)
    flags = plan.status()
    value = job_value(world, per_step, args.steps, elapsed_s)

    bf16_peak, hbm_peak, peak_kind = peaks()
    n_freq, n_ch = sc["n_freq"], plan.n_ch
    contract_ms = phase_ms[2] / max(runs, 1)
    alg_flops = 6.0 * n_freq * per_step                      # 3 contractions x 2 N_f per detector sample
    info = plan.info()
    n_groups = info.tile_groups if args.precision == "bf16x3" else (n_ch + 175) // 176
    n_half = info.tile_half if args.precision == "bf16x3" else ((n_ch + n_groups - 1) // n_groups + 15) // 16 * 16
    tiles = math.ceil(nt / 128) * plan.n_pix
    exec_flops = 5 * 2.0 * 128 * n_half * n_groups * info.n_freq_padded * tiles
    achieved = alg_flops / (contract_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak, "traffic": traffic_from_record(),
                "kernel": "fused_bf16x3_kernel" if args.precision == "bf16x3" else "psd_fp32+contract_fp32",
                "peak_source": f"{peak_kind} bf16 dense burst (MEASURED_PEAKS.json)",
                "algorithmic_flops_per_launch": alg_flops, "executed_mma_flops_per_launch": exec_flops,
                "executed_tflops": exec_flops / (contract_ms / 1e3) / 1e12,
                "kernel_ms_per_launch": contract_ms,
                "phase_ms_per_step": {"rows": phase_ms[0] / max(runs, 1), "contract": contract_ms,
                                      "pink": phase_ms[3] / max(runs, 1)}}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * elapsed_s / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16x3" else "f32",
              "data": "synthetic (seeded stand-ins for the paper's screens, ATM table and sources)",
              "config": {"workload": WORKLOAD, "n_pix": plan.n_pix, "n_ch": n_ch, "n_freq": n_freq, "nt": nt,
                         "detector_samples_per_step": per_step, "precision": args.precision,
                         "contraction": "split-BF16 hi/lo, 3 tcgen05 products, FP32 accumulate (noise: 1 product each)"
                         if args.precision == "bf16x3" else "FP32 SIMT",
                         "l2": "working set > L2: 197 MB source cube read and 6.66 GB output written per step",
                         "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
              "roofline": roofline, "gpu_launches": launches, "clocks": clk.summary(), "status_flags": flags,
              "autotune": None if tune is None else {
                  "choice": {"channel_groups": info.tile_groups, "channels_per_group": info.tile_half,
                             "ring_a": info.ring_a, "ring_b": info.ring_b},
                  "sample": "first 4096 samples of the scan", "ms": tune["ms"], "default_ms": tune["default_ms"],
                  "candidates": tune["candidates"]},
              "staged_inputs": info.staged_inputs,
              "plan_build": {"ms": build_ms, "device_bytes": int(info.device_bytes),
                             "what": "inputs uploaded (screen, opacity table, cube) + plan preparation: FP64 cascade "
                                     "collapse, filter matrices, reference spectrum, split-BF16 operand tiling, pink "
                                     "filter design; not in the steps, autotuning not included"}}

    # plain FP32 path on the same workload and GPU (the baseline the fused path is measured against)
    if not args.skip_fp32 and args.precision == "bf16x3":
        del out
        torch.cuda.empty_cache()
        p32 = Plan(sc, precision="fp32", white=True, pink=True)
        o32 = torch.empty((nt, p32.n_pix, p32.n_ch), dtype=torch.float32, device="cuda")
        p32.run(0, nt, o32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp32_steps):
            p32.run(0, nt, o32)
        e1.record(stream)
        torch.cuda.synchronize()
        t32 = ranks_max(e0.elapsed_time(e1) / 1e3)
        v32 = job_value(world, per_step, args.fp32_steps, t32)
        result["fp32_path"] = {"value": v32, "unit": UNIT, "ms_per_step": 1e3 * t32 / args.fp32_steps,
                               "speedup_of_bf16x3": value / v32}
        del o32, p32
        torch.cuda.empty_cache()
        out = None

    # brightness-temperature output (Sect. 2.7): the skydip fit runs once when the plan is prepared
    # (preparation timed beside the same plan's in W; the difference is within their noise), then
    # every step writes K instead of W
    if not args.skip_kelvin:
        torch.cuda.empty_cache()
        dip = (0.4, 2.4, 16)
        pw = Plan(sc, precision=args.precision, white=True, pink=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        pw.prepare()
        prep_w = time.perf_counter() - t
        del pw
        pk = Plan(dict(sc, output=dict(units="K", skydip=dip)), precision=args.precision, white=True, pink=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        pk.prepare()
        prep_k = time.perf_counter() - t
        ok = torch.empty((nt, pk.n_pix, pk.n_ch), dtype=torch.float32, device="cuda")
        pk.run(0, nt, ok)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pk.run(0, nt, ok)
        e1.record(stream)
        torch.cuda.synchronize()
        tk = e0.elapsed_time(e1)
        # downstream: common-mode reduction of the K TOD (Sect. 4.3, Eqs. 25-26), in place, off-source
        # spaxels beyond 25" (the outer ring of the 5 x 5 IFU)
        t = time.perf_counter()
        pwv_mean = pk.mean_zenith_pwv(nt)
        t_pwv = time.perf_counter() - t
        r_out = 25.0 * math.pi / (180 * 3600)
        pk.common_mode(0, ok, pwv_mean, r_out, out=ok)
        torch.cuda.synchronize()
        e0.record(stream)
        pk.common_mode(0, ok, pwv_mean, r_out, out=ok)
        e1.record(stream)
        torch.cuda.synchronize()
        t_cm = e0.elapsed_time(e1)
        cm_bytes = 2.0 * ok.numel() * 4 + nt * pk.n_pix * 32.0        # TOD in + out, row records
        result["common_mode"] = {"ms": t_cm, "mean_pwv_ms": 1e3 * t_pwv, "pwv_mean_mm": pwv_mean, "r_out_arcsec": 25.0,
                                 "algorithmic_bytes": cm_bytes, "achieved_gbs": cm_bytes / (t_cm / 1e3) / 1e9,
                                 "peak_gbs": hbm_peak, "frac": cm_bytes / (t_cm / 1e3) / 1e9 / hbm_peak,
                                 "kernels": "row_setup + band_transmission + common_mode", "status_flags": pk.status()}
        result["kelvin"] = {"skydip": {"pwv_mm": [dip[0], dip[1]], "n_pwv": dip[2], "elevation_rad": sc["scan"]["theta0"]},
                            "prepare_ms": 1e3 * prep_k, "prepare_ms_watts": 1e3 * prep_w, "ms_per_step": tk,
                            "step_overhead_vs_watts": tk / (1e3 * elapsed_s / args.steps) - 1.0,
                            "status_flags": pk.status()}
        del ok, pk
        torch.cuda.empty_cache()

    # exact pink noise (Sect. 2.6, Timmer & Koenig): the whole scan's realisation is drawn and
    # transformed when the plan is prepared (timed against preparing the filter plan); each step
    # then adds its samples instead of running the pole-zero filter scan
    if not args.skip_tk:
        torch.cuda.empty_cache()
        pt = Plan(dict(sc, noise=dict(sc["noise"], pink_tk=nt)), precision=args.precision, white=True, pink=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        pt.prepare()
        prep_t = time.perf_counter() - t
        ot = torch.empty((nt, pt.n_pix, pt.n_ch), dtype=torch.float32, device="cuda")
        pt.run(0, nt, ot)
        torch.cuda.synchronize()
        pt.get_timing()
        pt.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pt.run(0, nt, ot)
        e1.record(stream)
        torch.cuda.synchronize()
        ph, _, _ = pt.get_timing()
        pt.set_timing(False)
        info_t = pt.info()
        result["pink_tk"] = {"fft_length": 1 << (nt - 1).bit_length(), "prepare_ms": 1e3 * prep_t,
                             "ms_per_step": e0.elapsed_time(e1), "pink_phase_ms": ph[3],
                             "filter_pink_phase_ms": roofline["phase_ms_per_step"]["pink"],
                             "device_bytes": int(info_t.device_bytes), "status_flags": pt.status()}
        del ot, pt
        torch.cuda.empty_cache()

    # preprocessing on the device (Sect. 2.2, Eqs. 1-3): the workload's cube taken as a specific-
    # intensity cube and convolved with the far field of a 10 m dish (-10 dB edge taper) at all of its
    # frequencies, and the 1024^2 screen smoothed by the aperture footprint
    if not args.skip_prep and rank == 0:
        from paper_2604_23305_b300 import prep
        torch.cuda.empty_cache()
        src = sc["source"]
        cube = torch.from_numpy(np.ascontiguousarray(src["cube"], dtype=np.float32)).cuda()
        nu_grid = np.linspace(sc["f_lo"], sc["f_hi"], sc["n_freq"])
        scr = torch.from_numpy(np.ascontiguousarray(sc["atmosphere"]["screen"], dtype=np.float32)).cuda()
        prep.convolve_source(cube[:, :, :8].contiguous(), nu_grid[:8], src["el0"], src["daz"], src["del"], 5.0, -10.0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        pc = prep.convolve_source(cube, nu_grid, src["el0"], src["daz"], src["del"], 5.0, -10.0)
        torch.cuda.synchronize()
        t_conv = time.perf_counter() - t
        t = time.perf_counter()
        ps = prep.smooth_screen(scr, sc["atmosphere"]["pitch"], 5.0, -10.0)
        torch.cuda.synchronize()
        t_scr = time.perf_counter() - t
        n_az, n_el, n_f = cube.shape
        plane = 4 * n_az * n_el
        fft_flops = 4 * 5.0 * plane * math.log2(plane) * n_f        # 4 complex 2-D transforms per frequency
        result["preprocessing"] = {"cube": [int(n_az), int(n_el), int(n_f)], "convolve_source_ms": 1e3 * t_conv,
                                   "convolve_fft_gflops": fft_flops / t_conv / 1e9,
                                   "screen": list(scr.shape), "smooth_screen_ms": 1e3 * t_scr,
                                   "dish_m": 10.0, "edge_taper_db": -10.0}
        del cube, pc, scr, ps
        torch.cuda.empty_cache()

    # CUDA graphs where launches are the cost: a small request (1 spaxel, 64 channels, 512 points)
    # simulated in 64 chunks of 64 samples, launched one call at a time or replayed from one graph
    if rank == 0 and not args.skip_graph:
        gsc = W.scenario("single_pixel_small", nt_total=4096)
        gp = Plan(gsc, precision=args.precision, white=True, pink=True)
        gout = torch.empty((4096, gp.n_pix, gp.n_ch), dtype=torch.float32, device="cuda")
        gchunks = [(t, 64) for t in range(0, 4096, 64)]

        def gdirect():
            for t0, n in gchunks:
                gp.run(t0, n, gout[t0:t0 + n])
        gdirect()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            gdirect()
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            gdirect()
        e1.record(stream)
        torch.cuda.synchronize()
        t_direct = e0.elapsed_time(e1) / 5
        e0.record(stream)
        for _ in range(5):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        t_graph = e0.elapsed_time(e1) / 5
        result["cuda_graph"] = {"workload": "1 spaxel, 64 channels, 512 points: 64 chunks of 64 samples",
                                "kernels_per_chunk": 5, "direct_ms": t_direct, "graph_ms": t_graph,
                                "speedup": t_direct / t_graph}
        del graph, gout, gp
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: inputs uploaded from pinned host memory by
    # the setters and the TOD copied back by gateau_run_host, both inside the timed region
    if not args.skip_e2e:
        import ctypes
        pe = Plan(sc, precision=args.precision, white=True, pink=True, upload=False)
        pe.set_scan(sc["scan"], device=False)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        cube = pin(sc["source"]["cube"])
        screen = pin(sc["atmosphere"]["screen"])
        table = pin(sc["atmosphere"]["table"])
        host_out = torch.empty((nt, pe.n_pix, pe.n_ch), dtype=torch.float32, pin_memory=True).numpy()
        src = dict(sc["source"], cube=cube)
        atm = dict(sc["atmosphere"], screen=screen, table=table)

        def e2e_step():
            pe.set_source(src, device=False)
            pe.set_screen(atm, device=False)
            pe.set_table(atm, device=False)
            pe.run_host(0, nt, host_out)

        e2e_step()
        barrier()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        te = ranks_max(time.perf_counter() - t)
        result["e2e"] = {"value": job_value(world, per_step, args.e2e_steps, te), "unit": UNIT,
                         "h2d_bytes_per_step": int(cube.nbytes + screen.nbytes + table.nbytes),
                         "d2h_bytes_per_step": int(host_out.nbytes), "ms_per_step": 1e3 * te / args.e2e_steps}
        del pe, host_out

    if not args.skip_serving:
        torch.cuda.empty_cache()
        result["serving"] = serving_leg(args.serving_requests, seed=2 + 100 * rank)
        result["serving_shared_launches"] = serving_leg(args.serving_requests, seed=2 + 100 * rank,
                                                        shared_launches=True)
    if rank == 0 and world == 1 and not args.skip_cpu:
        result["cpu_baseline"] = cpu_baseline(sc, workload=args.workload)
    if rank == 0:
        print(json.dumps(result))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
