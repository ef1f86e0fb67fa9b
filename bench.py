#!/usr/bin/env python3
"""Throughput of the fast-bilateral-stereo path on GB300.

A step is one stereo pair through the whole path (cost volume, bilateral
aggregation of every disparity slice, WTA, Eq. (10) refinement) via the C ABI
entry point fbs_compute_disparity, with the pair already resident in HBM.
Three forms are timed on the same pair: plain FP32, and the tensor-core form
with BF16 and with FP16 operands (FP32 accumulation).  The headline value is
the BF16 form (--prec selects another); every form's Gtaps/s, fps and extra
bad-pixel rate (>1 px against the FP32 form on the whole frame, and against
the FP64 oracle on 300 sampled pixels) are in "forms".
The workload is the 640x480 RGB pair with D = 64, radius 7 (15x15 window),
sigma_s = 7, sigma_r = 12, rendered by the seeded synthetic scene generator
(fractal texture, slanted planes, occlusions).  The metric is aggregated
taps per second, Gtaps/s = H * W * D * (2 radius + 1)^2 / t, with fps and
Mde/s (Eq. (13)) beside it.

Timing: W untimed warm-up steps, then exactly K steps between a barrier and a
device synchronisation on both sides.  L2 is flushed (a 512 MiB write) before
every step, outside the CUDA-event pair that times the step; ms_per_step is
the mean of the per-step event times, max over ranks.  With --gpus N (under
torchrun) every rank runs an independent replica on its own pair: the path
does not shard, so there is no collective on the data path ("weak" scaling).

--impl reference times the FP64 CPU oracle on the host (bounded row bands of
the same workload) and prints the same JSON line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FBS aggregated Gtaps/s and fps; plain FP32 vs chosen form at fixed error"
UNIT = "Gtaps/s"
DEFAULT_WORKLOAD = "rgb640x480_d64_r7"
FLUSH_BYTES = 512 << 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128
SFU_EX2_PER_SM_CLK = 16   # special-function unit: exp2 results per SM per clock


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="bf16", choices=["f32", "bf16", "f16"],
                    help="the form reported as the headline value; all three forms are timed unless --only-form")
    ap.add_argument("--only-form", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--cost", default="ncc", choices=["ncc", "tad"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU baseline sample")
    ap.add_argument("--batched", action="store_true",
                    help="time the batched form on 64 uneven pairs (320..1024 x 240..768, D in {32,64,128,192}, "
                         "radius in {4,7,11}) instead of the single-pair workload")
    ap.add_argument("--batch-size", type=int, default=64)
    ap.add_argument("--band", action="store_true",
                    help="time the learned band form on the 1920x1080 RGB pair, D=256, radius 9 (network proposal "
                         "plus band-restricted path) against the plain full-range forms on the same pair")
    ap.add_argument("--sweep", action="store_true",
                    help="bad-pixel rate (e_PEP, Eq. (11)-(12), eps 2) per region against the scenes' ground truth "
                         "and runtime, over radius, gamma_d and gamma_r (640x480, D=64)")
    ap.add_argument("--lr", action="store_true",
                    help="time both views and the left-right consistency check (FP32) on the default workload")
    ap.add_argument("--band-shape", default=None,
                    help="WxH of the band workload's pair (default 1920x1080; smaller shapes are for profiling)")
    ap.add_argument("--band-threshold", type=float, default=None,
                    help="confidence threshold of the band form (default: the one shipped with the weights)")
    return ap.parse_args()


def _peaks():
    src = "measured"
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
    except (OSError, ValueError):
        p, src = dict(FALLBACK_PEAKS), "fallback"
    for k, v in FALLBACK_PEAKS.items():
        p.setdefault(k, v)
    return p, src


def _sm_count(torch, dev):
    """Streaming multiprocessors of the device (cudaDeviceProp), for the derived peaks."""
    return torch.cuda.get_device_properties(dev).multi_processor_count


def _taps(p):
    return p.H * p.W * p.D * (2 * p.radius + 1) ** 2


# ---------------------------------------------------------------------------
# clocks: nvidia-smi sampled during the run
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(index), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self, t0, t1):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        except OSError:
            return None
        if not rows:
            return None
        inwin = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        window = "timed region"
        if len(inwin) < 3:
            inwin = [r for r in rows if r[0] <= t1 + 0.05][-20:]
            window = "last samples up to the end of the timed region (timed region shorter than the sampling period)"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inwin for n, v in zip(names, r[3]) if v.lower().startswith("active")})
        mhz = sorted(r[1] for r in inwin)
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[2] for r in inwin), "reasons": reasons,
                "samples": len(inwin), "window": window}


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ---------------------------------------------------------------------------
def _oracle_band(p, y0, rows, mode):
    import oracle
    t = time.perf_counter()
    oracle.fbs(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, p.tau, mode=mode, rows=(y0, y0 + rows))
    return time.perf_counter() - t


def cpu_baseline(p, seconds, mode):
    """The oracle as it stands, single-threaded, on a row band sized to about
    ``seconds`` of work; Gtaps/s counts the taps of the rows it aggregated
    (its cost rows, including the 2*radius halo rows, are inside the time)."""
    probe = min(8, p.H)
    y0 = max(0, p.H // 2 - probe // 2)
    t = _oracle_band(p, y0, probe, mode)
    rows = int(max(probe, min(p.H, probe * seconds / max(t, 1e-6))))
    y0 = max(0, (p.H - rows) // 2)
    t = _oracle_band(p, y0, rows, mode)
    taps = rows * p.W * p.D * (2 * p.radius + 1) ** 2
    return {"value": taps / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"rows {y0}..{y0 + rows - 1} of the {p.W}x{p.H} frame ({rows} of {p.H} rows), "
                      f"single-threaded FP64 C oracle, {t:.1f} s"}


_POOL_PAIR = None


def _oracle_pool_init(name, seed):
    global _POOL_PAIR
    import oracle
    from synth import make_pair
    oracle.build()
    _POOL_PAIR = make_pair(name, seed)


def _oracle_rows_job(job):
    import oracle
    y0, rows, mode = job
    p = _POOL_PAIR
    oracle.fbs(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, p.tau, mode=mode, rows=(y0, y0 + rows))
    return rows


def cpu_baseline_all_cores(name, seed, p, seconds, mode):
    """The same oracle on every host core: row bands of the frame spread over a
    spawned process pool (one band per core, the pool's wall time measured)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    probe = min(4, p.H)
    t1 = _oracle_band(p, max(0, p.H // 2 - 2), probe, mode) / probe      # seconds per row on one core
    rows = int(max(1, min(p.H // cores, seconds / max(t1, 1e-6))))
    jobs = [(min(p.H - rows, i * rows), rows, mode) for i in range(cores)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                initializer=_oracle_pool_init, initargs=(name, seed)) as ex:
        list(ex.map(_oracle_rows_job, [(0, 1, mode)] * cores))   # every worker has rendered the pair
        t = time.perf_counter()
        list(ex.map(_oracle_rows_job, jobs))
        wall = time.perf_counter() - t
    taps = cores * rows * p.W * p.D * (2 * p.radius + 1) ** 2
    return {"value": taps / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} row bands of {rows} rows of the {p.W}x{p.H} frame, one per core "
                      f"(spawned process pool), single-threaded FP64 C oracle in each, {wall:.1f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from synth import make_pair
    oracle.build()
    p = make_pair(args.workload, args.seed)
    mode = 0 if args.cost == "ncc" else 1
    steps = args.steps if args.steps is not None else 5
    warmup = args.warmup if args.warmup is not None else 1
    # size each step's row band so the whole run stays near two minutes
    t8 = _oracle_band(p, p.H // 2 - 4, 8, mode) / 8
    rows = int(max(1, min(p.H, 120.0 / max(1, steps + warmup) / max(t8, 1e-6))))
    for i in range(warmup):
        _oracle_band(p, (i * rows) % max(1, p.H - rows + 1), rows, mode)
    total = 0.0
    for i in range(steps):
        total += _oracle_band(p, (i * rows) % max(1, p.H - rows + 1), rows, mode)
    taps = steps * rows * p.W * p.D * (2 * p.radius + 1) ** 2
    value = taps / total / 1e9
    sample = f"{rows} rows of the {p.W}x{p.H} frame per step, single-threaded FP64 C oracle"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(p, args, "ours"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _config(p, args, impl):
    return {"workload": args.workload, "H": p.H, "W": p.W, "C": p.C, "D": p.D, "radius": p.radius,
            "window": f"{2 * p.radius + 1}x{2 * p.radius + 1}", "sigma_s": p.sigma_s, "sigma_r": p.sigma_r,
            "tau": p.tau, "cost": args.cost, "precision": args.prec, "seed": args.seed,
            "pairs_per_step_per_gpu": 1, "parallelism": f"replicas x{args.gpus}",
            "l2": "512 MiB flush write before every step, outside the per-step CUDA-event timing",
            "inputs": "resident in HBM before the timed region"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def _traffic_for(kernel_file, kernel_name, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel and on this workload (else None).
    kernel_file is one path or a list of paths (the kernel's .cu and the
    headers holding its code), hashed in order."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    files = [kernel_file] if isinstance(kernel_file, str) else list(kernel_file)
    try:
        with open(path) as f:
            t = json.load(f)
        hs = hashlib.sha256()
        for fn in files:
            with open(fn, "rb") as f:
                hs.update(f.read())
        h = hs.hexdigest()[:16]
    except (OSError, ValueError):
        return None
    ent = t.get(kernel_name)
    if not ent or ent.get("source_sha256_16") != h or ent.get("workload") != workload:
        return None
    return ent.get("dram_bytes_per_launch_full_size")


FORM_PREC = {"f32": 0, "bf16": 1, "f16": 2}


def replica_env():
    """(world, rank, local rank) of a torchrun launch (1, 0, 0 otherwise).  The
    path does not shard: every rank runs an independent replica on its own
    pair (scene seed + rank), and only the step time is reduced."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, dist, device):
    """The largest per-rank value (the job's step time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, slowest_seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / slowest_seconds


def _time_form(fbs, torch, p, form, mode, dev, stream, dl, dr, flush, steps, warmup, dist):
    """Warm up, then time exactly `steps` steps of one form twice: first with
    per-step CUDA events on the launch stream only (the step time: the
    library's per-kernel events would serialise the programmatic launch of the
    tensor-core aggregation behind the cost kernel), then the same steps with
    the library's per-kernel events on (kernel times and launch counts).  The
    L2 flush is outside every event pair."""
    ctx = fbs.Context(dev.index, cost=mode, prec=FORM_PREC[form])
    di = torch.empty((p.H, p.W), dtype=torch.int32, device=dev)
    ds = torch.empty((p.H, p.W), dtype=torch.float32, device=dev)
    call = lambda: fbs.fbs_compute_disparity(ctx.ctx, dl, dr, p.H, p.W, p.C, p.D, p.radius, p.sigma_s, p.sigma_r,
                                             p.tau, di, ds, stream)

    def timed_pass():
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            call()
            b.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times = sorted(a.elapsed_time(b) for a, b in evs)
        return sum(times) / steps, times[len(times) // 2]

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.fill_(1)
            call()
        t0 = time.time()
        step_ms, step_ms_median = timed_pass()
        fbs.fbs_profile(ctx.ctx, 1)
        step_ms_profiled, _ = timed_pass()
        fbs.fbs_profile(ctx.ctx, 0)
        t1 = time.time()
    fbs.fbs_sync(ctx.ctx)
    step_ms = max_over_ranks(step_ms, dist, dev)
    kt = {fbs.KERNEL_NAMES[k]: fbs.fbs_profile_read(ctx.ctx, k) for k in range(fbs.FBS_KERNEL_KINDS)}
    return dict(ctx=ctx, di=di, ds=ds, step_ms=step_ms, step_ms_median=step_ms_median,
                step_ms_profiled=step_ms_profiled, kt=kt, t0=t0, t1=t1)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1807_02044_gb300 as fbs
    from synth import make_pair

    world, rank, local = replica_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    steps = args.steps if args.steps is not None else 3000
    warmup = max(3, args.warmup if args.warmup is not None else 20)

    p = make_pair(args.workload, args.seed + rank)
    mode = fbs.FBS_COST_NCC if args.cost == "ncc" else fbs.FBS_COST_TAD
    stream = torch.cuda.Stream(dev)
    dl = torch.from_numpy(p.left).to(dev)
    dr = torch.from_numpy(p.right).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    forms = [args.prec] if args.only_form else ["f32", "bf16", "f16"]
    if args.prec not in forms:
        forms.append(args.prec)
    sampler = None if args.no_clocks else ClockSampler(dev.index, os.path.join(ROOT, "_bench_clocks.csv"))
    res = {f: _time_form(fbs, torch, p, f, mode, dev, stream, dl, dr, flush, steps, warmup, dist) for f in forms}
    if sampler is not None:
        sampler.stop()

    taps = _taps(p)
    peaks, peak_src = _peaks()
    chosen = res[args.prec]
    # accuracy at fixed error: extra bad pixels (>1 px) against the FP32 form
    # on the whole frame, and against the FP64 oracle on sampled pixels
    ref = res.get("f32")
    rng = np.random.default_rng(1234)
    ns = 0 if args.no_oracle_check or rank != 0 else 300
    xs, ys = rng.integers(0, p.W, ns), rng.integers(0, p.H, ns)
    ref_ds = None
    if ns:
        import oracle
        oracle.build()
        _, ref_ds, _ = oracle.fbs_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys, tau=p.tau,
                                         mode=mode)
    form_out = {}
    for f, r in res.items():
        ds_np = r["ds"].cpu().numpy()
        ent = {"gtaps_per_s": world * taps / (r["step_ms"] * 1e-3) / 1e9, "ms_per_step": r["step_ms"],
               "fps": world * 1e3 / r["step_ms"], "ms_per_step_median": r["step_ms_median"],
               "ms_per_step_with_kernel_events": r["step_ms_profiled"],
               "kernel_ms_per_step": {k: v[0] / steps for k, v in r["kt"].items() if v[1]}}
        if ref is not None and f != "f32":
            ent["bad_px_vs_f32_pct"] = 100.0 * float(np.mean(np.abs(ds_np - ref["ds"].cpu().numpy()) > 1.0))
        if ref_ds is not None:
            ent["bad_px_vs_oracle_pct_sampled"] = 100.0 * float(np.mean(np.abs(ds_np[ys, xs] - ref_ds) > 1.0))
        form_out[f] = ent
    if ref_ds is not None and "f32" in form_out:
        for f, ent in form_out.items():
            ent["extra_bad_px_vs_oracle_pct"] = ent["bad_px_vs_oracle_pct_sampled"] - \
                form_out["f32"]["bad_px_vs_oracle_pct_sampled"]

    step_ms = chosen["step_ms"]
    value = job_rate(taps, world, step_ms * 1e-3) / 1e9
    kt = chosen["kt"]
    launches = sum(n for _, n in kt.values())
    clocks = sampler.summary(chosen["t0"], chosen["t1"]) if sampler is not None else None
    if sampler is not None:
        try:
            os.remove(sampler.path)
        except OSError:
            pass
    csrc = os.path.join(ROOT, "paper_1807_02044_gb300", "csrc")
    flops = 2.0 * taps
    sms = _sm_count(torch, dev)
    if args.prec == "f32":
        agg_ms, agg_n = kt["aggregate_f32"]
        agg_launch_ms = agg_ms / max(1, agg_n)
        fp32_peak = sms * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        roofline = {"kernel": "aggregate_f32_kernel", "bound": "alu",
                    "achieved": flops / (agg_launch_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                    "peak_source": f"derived: {sms} SMs (cudaDeviceProp) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                   f"{peaks['sm_max_mhz']:.0f} MHz (max SM clock, {peak_src})",
                    "traffic": _traffic_for(os.path.join(csrc, "fbs_aggregate_f32.cu"), "aggregate_f32_kernel",
                                           args.workload)}
    else:
        agg_ms, agg_n = kt["aggregate_tc"]
        agg_launch_ms = agg_ms / max(1, agg_n)
        # tensor peak: measured cuBLAS bf16 (burst); FP16 dense rate is the same on GB300
        rho8 = (p.radius + 7) // 8 * 8
        kw = (16 + rho8 + p.radius + 15) // 16 * 16
        n = (p.D + 15) // 16 * 16
        tiles = ((p.W + 15) // 16) * ((p.H + 7) // 8)
        issued = 2.0 * tiles * 128 * n * kw * (8 + 2 * p.radius)
        roofline = {"kernel": "aggregate_tc_kernel", "bound": "tensor",
                    "achieved": flops / (agg_launch_ms * 1e-3) / 1e12, "peak": peaks["bf16_tflops"],
                    "unit": "TFLOP/s", "peak_source": f"bf16_tflops burst ({peak_src}); FP16 dense equals BF16",
                    "issued_dense_tflops": issued / (agg_launch_ms * 1e-3) / 1e12,
                    "issued_over_algorithmic": issued / flops,
                    "traffic": _traffic_for([os.path.join(csrc, "fbs_aggregate_tc.cu"), os.path.join(csrc, "tc_aggregate.cuh")],
                                           "aggregate_tc_kernel", args.workload)}
    roofline.update({"algorithmic": "2 flop per tap (one multiply-add per window tap per disparity), "
                                    "H*W*D*(2r+1)^2 taps", "avg_launch_ms": agg_launch_ms, "launches": agg_n})
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    # weight generation (Eq. (7)-(8)), fused in the aggregation: one exp2 per
    # (pixel, window tap), reported against the derived exp2 rate of the SFUs
    weights = p.H * p.W * (2 * p.radius + 1) ** 2
    ex2_peak = sms * SFU_EX2_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6
    roofline["weight_generation"] = {
        "weights_per_launch": weights, "achieved_per_s": weights / (agg_launch_ms * 1e-3), "peak_per_s": ex2_peak,
        "peak_source": f"derived: {sms} SMs (cudaDeviceProp) x {SFU_EX2_PER_SM_CLK} exp2 per clock x "
                       f"{peaks['sm_max_mhz']:.0f} MHz",
        "frac": weights / (agg_launch_ms * 1e-3) / ex2_peak}
    cost_ms, cost_n = kt["cost_build"]
    cost_launch_ms = cost_ms / max(1, cost_n)
    ld = (p.D + 3) // 4 * 4
    vol = 4 * p.H * p.W * ld if args.prec == "f32" else 2 * p.H * p.D * ((p.W + 7) // 8 * 8)
    cost_bytes = 2 * p.H * p.W * p.C + vol
    cost_kernel = "cost_kernel" if args.prec == "f32" else "cost_xb_kernel"
    roofline_cost = {"kernel": "cost_kernel (+ grey_stats_kernel)" if args.prec == "f32" else
                     "cost_xb_kernel (statistics, costs, pad rows and guide in one launch)", "bound": "hbm",
                     "achieved": cost_bytes / (cost_launch_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "avg_launch_ms": cost_launch_ms, "launches": cost_n,
                     "algorithmic": "read both images once, write the cost volume once",
                     "traffic": _traffic_for(os.path.join(csrc, "fbs_cost.cu"), cost_kernel, args.workload)}
    roofline_cost["frac"] = roofline_cost["achieved"] / roofline_cost["peak"]

    e2e = None
    ctx = chosen["ctx"]
    if not args.no_e2e:
        n_e2e = min(steps, 200)
        hl = torch.from_numpy(p.left).pin_memory()
        hr = torch.from_numpy(p.right).pin_memory()
        hi = torch.empty((p.H, p.W), dtype=torch.int32).pin_memory()
        hs = torch.empty((p.H, p.W), dtype=torch.float32).pin_memory()
        host_call = lambda: fbs.fbs_compute_disparity_host(ctx.ctx, hl.data_ptr(), hr.data_ptr(), p.H, p.W, p.C, p.D,
                                                           p.radius, p.sigma_s, p.sigma_r, p.tau, hi.data_ptr(),
                                                           hs.data_ptr())
        for _ in range(3):
            host_call()
        tot = 0.0
        for _ in range(n_e2e):
            flush.fill_(1)
            torch.cuda.synchronize()
            t = time.perf_counter()
            host_call()
            tot += time.perf_counter() - t
        e2e_s = max_over_ranks(tot / n_e2e, dist, dev)
        assert np.array_equal(hi.numpy(), chosen["di"].cpu().numpy())
        e2e = {"value": job_rate(taps, world, e2e_s) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * p.H * p.W * p.C,
               "d2h_bytes_per_step": 8 * p.H * p.W, "steps": n_e2e,
               "call": "fbs_compute_disparity_host (pinned host buffers, transfers and sync inside the timed call; "
                       "the 16-bit forms read the images from and write the maps to the pinned host buffers "
                       "directly, without staging copies)"}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_seconds, mode)
        cpu_all = cpu_baseline_all_cores(args.workload, args.seed, p, args.cpu_seconds, mode)

    cfg = _config(p, args, "ours")
    cfg["forms_timed"] = forms
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
           "ms_per_step": step_ms, "ms_per_step_median": chosen["step_ms_median"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic", "config": cfg,
           "fps": world * 1e3 / step_ms, "mde_per_s": world * p.W * p.H * p.D / (step_ms * 1e-3) * 1e-6,
           "form": args.prec, "forms": form_out,
           "roofline": roofline, "roofline_cost_build": roofline_cost, "cpu_baseline": cpu,
           "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
           "gpu_launches": launches, "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items() if v[1]},
           "timing": "ms_per_step from per-step events only; kernel times, launches and the rooflines from a "
                     "second timed pass of the same steps with the library's per-kernel events "
                     f"({chosen['step_ms_profiled']:.4f} ms per step there)",
           "clocks": clocks, "wall_s_timed_region": chosen["t1"] - chosen["t0"]}
    if "f32" in form_out:
        # the paper-precision comparator: the plain FP32 form on the same inputs
        out["f32_gtaps_per_s"] = form_out["f32"]["gtaps_per_s"]
        out["f32_ms_per_step"] = form_out["f32"]["ms_per_step"]
    if rank == 0:
        print(json.dumps(out))
    for r in res.values():
        r["ctx"].close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _render_batch_member(spec):
    from synth import make_pair
    p = make_pair("rgb640x480_d64_r7", spec["seed"], H=spec["H"], W=spec["W"], D=spec["D"], radius=spec["radius"])
    return p.left, p.right


def _tc_plan_graph(plan):
    """What the batched graph of tensor-core plan `plan` holds."""
    if plan == 6:
        return ("per pair: one-kernel 16-bit cost build (2 concurrent branches); then one persistent tcgen05 "
                "aggregation over the tiles of every pair")
    return (f"per pair: one-kernel 16-bit cost build, tcgen05 aggregation; {[1, 2, 4][plan >> 1]} concurrent "
            f"branches, stage rows {'max' if plan % 2 == 0 else '<= 3'}")


def run_batched(args):
    """One step = one batch of uneven pairs through fbs_compute_disparity_batched
    (FP32, one CUDA graph; the autotuner's plan).  Beside it: the same
    pairs as sequential per-pair calls, FP32 and BF16 tensor-core form, and
    the BF16 batched form (one graph of every pair's tensor-core launches)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from synth import random_batch_specs
    specs = random_batch_specs(args.seed, args.batch_size)
    # render in worker processes started with spawn, before the first GPU call
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        imgs = list(ex.map(_render_batch_member, specs))
    import torch

    import paper_1807_02044_gb300 as fbs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    steps = args.steps if args.steps is not None else 10
    warmup = max(3, args.warmup if args.warmup is not None else 3)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    pairs = []
    for spec, (L, R) in zip(specs, imgs):
        H, W = spec["H"], spec["W"]
        pairs.append(dict(left=torch.from_numpy(L).to(dev), right=torch.from_numpy(R).to(dev), H=H, W=W, C=3,
                          D=spec["D"], radius=spec["radius"], sigma_s=spec["sigma_s"], sigma_r=spec["sigma_r"],
                          tau=spec["tau"], disp_int=torch.empty((H, W), dtype=torch.int32, device=dev),
                          disp_subpix=torch.empty((H, W), dtype=torch.float32, device=dev)))
    taps = sum(q["H"] * q["W"] * q["D"] * (2 * q["radius"] + 1) ** 2 for q in pairs)

    def timed(fn, ctx):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.fill_(1)
                fn()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.synchronize()
            fbs.fbs_profile(ctx.ctx, 1)
            for a, b in evs:
                flush.fill_(1)
                a.record(stream)
                fn()
                b.record(stream)
            torch.cuda.synchronize()
            fbs.fbs_profile(ctx.ctx, 0)
        fbs.fbs_sync(ctx.ctx)
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        launches = sum(fbs.fbs_profile_read(ctx.ctx, k)[1] for k in range(fbs.FBS_KERNEL_KINDS))
        return ms, launches

    arr = fbs.make_pairs(pairs)
    with fbs.Context(0) as ctx:
        t_batch, launches = timed(lambda: fbs.fbs_compute_disparity_batched(ctx.ctx, arr, stream), ctx)
        plan = fbs.fbs_batch_plan(ctx.ctx, arr)
        ref = [(q["disp_int"].clone(), q["disp_subpix"].clone()) for q in pairs]

        def seq():
            for q in pairs:
                fbs.fbs_compute_disparity(ctx.ctx, q["left"], q["right"], q["H"], q["W"], 3, q["D"], q["radius"],
                                          q["sigma_s"], q["sigma_r"], q["tau"], q["disp_int"], q["disp_subpix"],
                                          stream)
        t_seq, _ = timed(seq, ctx)
        torch.cuda.synchronize()
        identical = all(torch.equal(q["disp_int"], r[0]) and torch.equal(q["disp_subpix"], r[1])
                        for q, r in zip(pairs, ref))
    with fbs.Context(0, prec=fbs.FBS_PREC_BF16) as ctx16:
        def seq16():
            for q in pairs:
                fbs.fbs_compute_disparity(ctx16.ctx, q["left"], q["right"], q["H"], q["W"], 3, q["D"], q["radius"],
                                          q["sigma_s"], q["sigma_r"], q["tau"], q["disp_int"], q["disp_subpix"],
                                          stream)
        t_seq16, _ = timed(seq16, ctx16)
        torch.cuda.synchronize()
        ref16 = [(q["disp_int"].clone(), q["disp_subpix"].clone()) for q in pairs]
        t_b16, launches16 = timed(lambda: fbs.fbs_compute_disparity_batched(ctx16.ctx, arr, stream), ctx16)
        plan16 = fbs.fbs_batch_plan(ctx16.ctx, arr)
        torch.cuda.synchronize()
        identical16 = all(torch.equal(q["disp_int"], r[0]) and torch.equal(q["disp_subpix"], r[1])
                          for q, r in zip(pairs, ref16))
        # every tensor-core plan on the same batch (the autotuner keeps the fastest)
        plans16 = {}
        for pl in range(7):
            fbs.fbs_batch_set_plan(ctx16.ctx, arr, pl)
            ms, nl = timed(lambda: fbs.fbs_compute_disparity_batched(ctx16.ctx, arr, stream), ctx16)
            torch.cuda.synchronize()
            same = all(torch.equal(q["disp_int"], r[0]) and torch.equal(q["disp_subpix"], r[1])
                       for q, r in zip(pairs, ref16))
            plans16[str(pl)] = {"ms_per_batch": ms, "gpu_launches": nl, "equals_sequential_bf16_bitwise": same,
                                "graph": _tc_plan_graph(pl)}
        fbs.fbs_batch_set_plan(ctx16.ctx, arr, plan16)
    n = len(pairs)
    out = {"metric": METRIC, "value": taps / (t_batch * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batch{n}_uneven_320-1024x240-768_d32-192_r4-11", "pairs": n, "taps": taps,
                      "seed": args.seed, "plan": plan,
                      "graph": ("persistent launches: statistics, cost, aggregation" if plan < 4 else
                                f"per-pair launches in {[1, 2, 4][plan - 4]} concurrent branches"),
                      "l2": "512 MiB flush write before every step, outside the per-step CUDA-event timing"},
           "pairs_per_s": n / (t_batch * 1e-3), "gpu_launches": launches,
           "batched_equals_sequential_bitwise": identical,
           "sequential_f32": {"ms_per_batch": t_seq, "gtaps_per_s": taps / (t_seq * 1e-3) / 1e9},
           "sequential_bf16": {"ms_per_batch": t_seq16, "gtaps_per_s": taps / (t_seq16 * 1e-3) / 1e9},
           "batched_bf16": {"ms_per_batch": t_b16, "gtaps_per_s": taps / (t_b16 * 1e-3) / 1e9, "plan": plan16,
                            "gpu_launches": launches16, "equals_sequential_bf16_bitwise": identical16,
                            "graph": _tc_plan_graph(plan16), "plans": plans16},
           "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out))
    return 0


def _time_call(fbs, torch, ctx, call, stream, flush, steps, warmup):
    """Warm up, then time exactly `steps` calls with per-step CUDA events on the
    launch stream (the L2 flush outside them); per-kind kernel times from the
    library's accounting."""
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.fill_(1)
            call()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        fbs.fbs_profile(ctx.ctx, 1)
        t0 = time.time()
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            call()
            b.record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
        fbs.fbs_profile(ctx.ctx, 0)
    fbs.fbs_sync(ctx.ctx)
    kt = {fbs.KERNEL_NAMES[k]: fbs.fbs_profile_read(ctx.ctx, k) for k in range(fbs.FBS_KERNEL_KINDS)}
    return dict(step_ms=sum(a.elapsed_time(b) for a, b in evs) / steps, kt=kt, t0=t0, t1=t1)


BAND_WORKLOAD = "rgb1920x1080_d256_r9"
HALF_BAND = 8


def run_band(args):
    """One step = one 1920x1080 pair through fbs_compute_disparity_learned:
    quarter-resolution features, the six-layer network (tensor cores), the
    per-pixel bands, the band-restricted cost and aggregation with WTA and
    Eq. (10).  Beside it: the plain full-range FP32 and BF16 forms on the
    same pair.  Gtaps/s counts the full-range taps H*W*D*(2r+1)^2 that the
    step replaces (the band path computes only part of them; the fraction is
    in config.work_fraction)."""
    import numpy as np
    import torch

    import paper_1807_02044_gb300 as fbs
    from synth import make_pair

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    steps = args.steps if args.steps is not None else 200
    warmup = max(3, args.warmup if args.warmup is not None else 5)
    if args.band_shape:
        bw, bh = (int(v) for v in args.band_shape.lower().split("x"))
        p = make_pair(BAND_WORKLOAD, args.seed, H=bh, W=bw)
    else:
        p = make_pair(BAND_WORKLOAD, args.seed)
    stream = torch.cuda.Stream(dev)
    dl = torch.from_numpy(p.left).to(dev)
    dr = torch.from_numpy(p.right).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    H, W, D = p.H, p.W, p.D
    thr = args.band_threshold if args.band_threshold is not None else fbs.default_band_threshold()
    taps = _taps(p)
    outs = {k: (torch.empty((H, W), dtype=torch.int32, device=dev), torch.empty((H, W), device=dev))
            for k in ("band", "f32", "bf16")}
    sampler = None if args.no_clocks else ClockSampler(dev.index, os.path.join(ROOT, "_bench_clocks.csv"))
    ctx = fbs.Context(0)
    fbs.fbs_band_net_load(ctx.ctx, fbs.default_band_net_path())
    arr = fbs.make_pairs([dict(left=dl, right=dr, H=H, W=W, C=3, D=D, radius=p.radius, sigma_s=p.sigma_s,
                               sigma_r=p.sigma_r, tau=p.tau, disp_int=outs["band"][0], disp_subpix=outs["band"][1])])
    band = _time_call(fbs, torch, ctx, lambda: fbs.fbs_compute_disparity_learned(ctx.ctx, arr, HALF_BAND, thr, stream),
                      stream, flush, steps, warmup)
    plain = {}
    for form in ("f32", "bf16"):
        c = fbs.Context(0, prec=FORM_PREC[form])
        di, ds = outs[form]
        plain[form] = _time_call(fbs, torch, c, lambda: fbs.fbs_compute_disparity(
            c.ctx, dl, dr, H, W, 3, D, p.radius, p.sigma_s, p.sigma_r, p.tau, di, ds, stream),
            stream, flush, max(3, steps // 10), warmup)
        c.close()
    if sampler is not None:
        sampler.stop()
    # the bands of this pair and the work they leave
    centre = torch.empty((H, W), device=dev)
    conf = torch.empty((H, W), device=dev)
    fbs.fbs_band_net_forward(ctx.ctx, dl, dr, H, W, 3, D, None, centre, conf)
    lo = torch.empty((H, W), dtype=torch.int32, device=dev)
    hi = torch.empty((H, W), dtype=torch.int32, device=dev)
    fbs.fbs_band_limits(ctx.ctx, centre, conf, H * W, D, HALF_BAND, thr, lo, hi)
    torch.cuda.synchronize()
    work = float(((hi - lo + 1).double().sum() / (H * W * D)).item())
    fallback = float((conf < thr).float().mean().item())
    # the non-learned band source (feature points, Sec. V) at a few margin thresholds
    fp_rows = []
    fc = torch.empty((H, W), device=dev)
    fk = torch.empty((H, W), device=dev)
    fi = torch.empty((H, W), dtype=torch.int32, device=dev)
    fs = torch.empty((H, W), device=dev)
    farr = fbs.make_pairs([dict(left=dl, right=dr, H=H, W=W, C=3, D=D, radius=p.radius, sigma_s=p.sigma_s,
                                sigma_r=p.sigma_r, tau=p.tau, disp_int=fi, disp_subpix=fs)])
    for th_m in (0.02, 0.05, 0.1, 0.2):
        def fp_step():
            fbs.fbs_band_feature_points(ctx.ctx, dl, dr, H, W, 3, D, th_m, fc, fk, stream)
            fbs.fbs_compute_disparity_banded(ctx.ctx, farr, fc, fk, HALF_BAND, 0.5, stream)
        t = _time_call(fbs, torch, ctx, fp_step, stream, flush, max(3, steps // 10), 3)
        fbs.fbs_band_limits(ctx.ctx, fc, fk, H * W, D, HALF_BAND, 0.5, lo, hi, stream)
        torch.cuda.synchronize()
        fp_rows.append({"margin_threshold": th_m, "ms_per_step": t["step_ms"], "fps": 1e3 / t["step_ms"],
                        "fallback_pct": 100.0 * float((fk < 0.5).float().mean().item()),
                        "work_fraction": float(((hi - lo + 1).double().sum() / (H * W * D)).item()),
                        "bad_px_vs_f32_pct": 100.0 * float(((fs - outs["f32"][1]).abs() > 1.0).float().mean().item())})
    ds_f32 = outs["f32"][1].cpu().numpy()
    res = {}
    for k in ("band", "bf16"):
        res[k] = 100.0 * float(np.mean(np.abs(outs[k][1].cpu().numpy() - ds_f32) > 1.0))
    # against the FP64 oracle on sampled pixels (full range)
    ns = 0 if args.no_oracle_check else 100
    rng = np.random.default_rng(1234)
    xs, ys = rng.integers(0, W, ns), rng.integers(0, H, ns)
    vs_oracle = None
    if ns:
        import oracle
        oracle.build()
        _, ref_ds, _ = oracle.fbs_points(p.left, p.right, D, p.radius, p.sigma_s, p.sigma_r, xs, ys)
        vs_oracle = {k: 100.0 * float(np.mean(np.abs(outs[k][1].cpu().numpy()[ys, xs] - ref_ds) > 1.0))
                     for k in ("band", "f32", "bf16")}
    peaks, peak_src = _peaks()
    kt = band["kt"]
    agg_ms, agg_n = kt["aggregate_f32"]
    agg_launch_ms = agg_ms / max(1, agg_n)
    sms = _sm_count(torch, dev)
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    band_flops = 2.0 * taps * work
    roofline = {"kernel": "aggregate_band_kernel", "bound": "alu",
                "achieved": band_flops / (agg_launch_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "peak_source": f"derived: {sms} SMs (cudaDeviceProp) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                               f"{peaks['sm_max_mhz']:.0f} MHz (max SM clock, {peak_src})",
                "algorithmic": "2 flop per tap of each pixel's own band (sum of band widths x (2r+1)^2)",
                "avg_launch_ms": agg_launch_ms, "launches": agg_n, "traffic": None}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    clocks = sampler.summary(band["t0"], band["t1"]) if sampler is not None else None
    if sampler is not None:
        try:
            os.remove(sampler.path)
        except OSError:
            pass
    e2e = None
    if not args.no_e2e:
        hl = torch.from_numpy(p.left).pin_memory()
        hr = torch.from_numpy(p.right).pin_memory()
        hs = torch.empty((H, W), dtype=torch.float32).pin_memory()
        hd = torch.empty((H, W), dtype=torch.int32).pin_memory()

        def e2e_call():
            with torch.cuda.stream(stream):
                dl.copy_(hl, non_blocking=True)
                dr.copy_(hr, non_blocking=True)
                fbs.fbs_compute_disparity_learned(ctx.ctx, arr, HALF_BAND, thr, stream)
                hd.copy_(outs["band"][0], non_blocking=True)
                hs.copy_(outs["band"][1], non_blocking=True)
            stream.synchronize()
        for _ in range(3):
            e2e_call()
        n_e2e = min(steps, 50)
        tot = 0.0
        for _ in range(n_e2e):
            flush.fill_(1)
            torch.cuda.synchronize()
            t = time.perf_counter()
            e2e_call()
            tot += time.perf_counter() - t
        e2e = {"value": taps / (tot / n_e2e) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * H * W * 3,
               "d2h_bytes_per_step": 8 * H * W, "steps": n_e2e,
               "call": "pinned host images copied in, fbs_compute_disparity_learned, disparities copied out, "
                       "stream synchronised; all inside the timed region"}
    cpu = None if args.no_cpu_baseline else cpu_baseline(p, args.cpu_seconds, 0)
    step_ms = band["step_ms"]
    out = {"metric": METRIC, "value": taps / (step_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (network bf16)", "data": "synthetic",
           "config": {"workload": BAND_WORKLOAD if not args.band_shape else f"{BAND_WORKLOAD} at {W}x{H}",
                      "H": H, "W": W, "C": 3, "D": D, "radius": p.radius,
                      "half_band": HALF_BAND, "conf_threshold": thr, "seed": args.seed,
                      "weights": os.path.relpath(fbs.default_band_net_path(), ROOT),
                      "work_fraction": work, "fallback_pct": 100.0 * fallback,
                      "l2": "512 MiB flush write before every step, outside the per-step CUDA-event timing",
                      "inputs": "resident in HBM before the timed region"},
           "fps": 1e3 / step_ms, "form": "learned band",
           "forms": {"band": {"gtaps_per_s": taps / (step_ms * 1e-3) / 1e9, "fps": 1e3 / step_ms,
                              "bad_px_vs_f32_pct": res["band"],
                              "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items() if v[1]}},
                     **{f: {"gtaps_per_s": taps / (plain[f]["step_ms"] * 1e-3) / 1e9, "fps": 1e3 / plain[f]["step_ms"],
                            "ms_per_step": plain[f]["step_ms"]} for f in plain}},
           "bad_px_vs_oracle_pct_sampled": vs_oracle, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": sum(n for _, n in kt.values()), "clocks": clocks}
    out["forms"]["bf16"]["bad_px_vs_f32_pct"] = res["bf16"]
    out["feature_point_band"] = fp_rows
    print(json.dumps(out))
    ctx.close()
    return 0


def run_lr(args):
    """One step = both disparity maps and the LRC check (Eq. (9)) through
    fbs_compute_disparity_lr (FP32): one cost pass storing both volumes, two
    aggregations, the check.  Gtaps/s counts the taps of both views.  Beside it
    the same call in a BF16 context (both views on the tensor cores)."""
    import numpy as np
    import torch

    import paper_1807_02044_gb300 as fbs
    from synth import make_pair

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    steps = args.steps if args.steps is not None else 500
    warmup = max(3, args.warmup if args.warmup is not None else 10)
    p = make_pair(args.workload, args.seed)
    stream = torch.cuda.Stream(dev)
    dl = torch.from_numpy(p.left).to(dev)
    dr = torch.from_numpy(p.right).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    H, W, D = p.H, p.W, p.D
    li = torch.empty((H, W), dtype=torch.int32, device=dev)
    ls = torch.empty((H, W), device=dev)
    ri = torch.empty((H, W), dtype=torch.int32, device=dev)
    rs = torch.empty((H, W), device=dev)
    ctx = fbs.Context(0)
    res = _time_call(fbs, torch, ctx, lambda: fbs.fbs_compute_disparity_lr(
        ctx.ctx, dl, dr, H, W, p.C, D, p.radius, p.sigma_s, p.sigma_r, p.tau, li, ls, ri, rs, True, stream),
        stream, flush, steps, warmup)
    one = _time_call(fbs, torch, ctx, lambda: fbs.fbs_compute_disparity(
        ctx.ctx, dl, dr, H, W, p.C, D, p.radius, p.sigma_s, p.sigma_r, p.tau, ri, rs, stream),
        stream, flush, steps, warmup)
    rejected = float((li == -1).float().mean().item())
    gt_ok = torch.from_numpy(~p.occ).to(dev)
    occ_rejected = float(((li == -1) & ~gt_ok).float().sum().item() / max(1.0, float((~gt_ok).sum().item())))
    taps = 2 * _taps(p)
    kt = res["kt"]
    ctx.close()
    # the same step in a BF16 context: both views on the tensor cores
    ctx16 = fbs.Context(0, prec=fbs.FBS_PREC_BF16)
    li16 = torch.empty_like(li)
    ls16 = torch.empty_like(ls)
    res16 = _time_call(fbs, torch, ctx16, lambda: fbs.fbs_compute_disparity_lr(
        ctx16.ctx, dl, dr, H, W, p.C, D, p.radius, p.sigma_s, p.sigma_r, p.tau, li16, ls16, ri, rs, True, stream),
        stream, flush, steps, warmup)
    torch.cuda.synchronize()
    valid = (li != -1) & (li16 != -1)
    bf16 = {"ms_per_step": res16["step_ms"], "gtaps_per_s": taps / (res16["step_ms"] * 1e-3) / 1e9,
            "fps": 1e3 / res16["step_ms"], "lrc_rejected_pct": 100.0 * float((li16 == -1).float().mean().item()),
            "bad_px_vs_f32_pct": 100.0 * float(((ls16 - ls).abs() > 1.0)[valid].float().mean().item()),
            "kernel_ms_per_step": {k: v[0] / steps for k, v in res16["kt"].items() if v[1]},
            "gpu_launches": sum(n for _, n in res16["kt"].values())}
    ctx16.close()
    out = {"metric": METRIC, "value": taps / (res["step_ms"] * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
           "steps": steps, "warmup": warmup, "ms_per_step": res["step_ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "views": "left + right + LRC (Eq. 9)", "seed": args.seed,
                      "l2": "512 MiB flush write before every step, outside the per-step CUDA-event timing"},
           "fps": 1e3 / res["step_ms"], "left_only_ms": one["step_ms"],
           "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items() if v[1]},
           "lrc_rejected_pct": 100.0 * rejected, "occluded_px_rejected_pct": 100.0 * occ_rejected,
           "gpu_launches": sum(n for _, n in kt.values()), "bf16_both_views": bf16,
           "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out))
    return 0


def e_pep(estimate, truth, eps, mask):
    """Eq. (11)-(12): percentage of the pixels of mask whose |estimate - truth|
    exceeds eps (the tests check it against the oracle's e_pep)."""
    import numpy as np
    bad = np.abs(np.asarray(estimate, np.float64) - np.asarray(truth, np.float64)) > eps
    return 100.0 * float(np.count_nonzero(bad[mask])) / max(1, int(np.count_nonzero(mask)))


def run_sweep(args):
    """Accuracy against ground truth and runtime over the aggregation
    parameters: radius (sigma_s = radius), gamma_d at radius 7, gamma_r at
    radius 7 -- the synthetic counterparts of the paper's parameter studies.
    e_PEP = % of pixels of a region whose |d - gt| > 2 (Eq. (11)-(12))."""
    import numpy as np
    import torch

    import paper_1807_02044_gb300 as fbs
    from synth import make_pair, regions as scene_regions

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    seeds = [args.seed, args.seed + 1, args.seed + 2]
    pairs = [make_pair("rgb640x480_d64_r7", s) for s in seeds]
    regions = [scene_regions(p) for p in pairs]
    devs = [(torch.from_numpy(p.left).to(dev), torch.from_numpy(p.right).to(dev)) for p in pairs]
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ctxs = {"f32": fbs.Context(0), "bf16": fbs.Context(0, prec=fbs.FBS_PREC_BF16)}

    def point(radius, gd, gr):
        row = {"radius": radius, "gamma_d": gd, "gamma_r": gr}
        for form, ctx in ctxs.items():
            if form == "bf16" and radius > 24:
                continue
            peps = {k: [] for k in regions[0]}
            for p, reg, (dl, dr) in zip(pairs, regions, devs):
                di, ds = ctx.compute_disparity(dl, dr, p.D, radius, gd, gr, stream=stream)
                torch.cuda.synchronize()
                est = ds.cpu().numpy()
                for k, m in reg.items():
                    peps[k].append(e_pep(est, p.gt, 2.0, m))
            p, (dl, dr) = pairs[0], devs[0]
            di = torch.empty((p.H, p.W), dtype=torch.int32, device=dev)
            ds = torch.empty((p.H, p.W), device=dev)
            t = _time_call(fbs, torch, ctx, lambda: fbs.fbs_compute_disparity(
                ctx.ctx, dl, dr, p.H, p.W, p.C, p.D, radius, gd, gr, p.tau, di, ds, stream), stream, flush, 20, 3)
            row[form] = {"e_pep_pct": {k: round(float(np.mean(v)), 3) for k, v in peps.items()},
                         "ms_per_frame": round(t["step_ms"], 4),
                         "mde_per_s": round(p.W * p.H * p.D / (t["step_ms"] * 1e-3) * 1e-6, 1)}
        return row

    out = {"sweep": "e_PEP (eps 2) per region and runtime, 640x480 RGB, D=64, scenes " + str(seeds),
           "radius": [point(r, float(r), 12.0) for r in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 15)],
           "gamma_d": [point(7, gd, 12.0) for gd in (1.0, 2.0, 3.0, 5.0, 7.0, 10.0, 15.0, 25.0)],
           "gamma_r": [point(7, 7.0, gr) for gr in (2.0, 4.0, 8.0, 12.0, 16.0, 24.0, 32.0, 64.0)]}
    print(json.dumps(out))
    for c in ctxs.values():
        c.close()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
    if args.band:
        return run_band(args)
    if args.lr:
        return run_lr(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
