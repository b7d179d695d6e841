#!/usr/bin/env python
"""Round-trip spherical-harmonic transform benchmark on GB300.

One step = one inverse (spectral -> grid) plus one direct (grid -> spectral)
transform of every field of the workload, through the C ABI.  The headline
workload is T639 on the octahedral grid O640 (1280 Gaussian latitudes, row i
from either pole with 20 + 4 i points, 1 666 560 points per field) with
137 levels x 4 fields = 548 fields, spectra N(0,1) (n+1)^-1.5, Legendre
stage in BF16x3 split precision with FP32 accumulation.

Prints one JSON line (rank 0).  `value` is field-transforms/s (fields x
round trips / s) with inputs resident in HBM; `e2e` is the same with the
spectra copied host -> device and the result device -> host inside each step.
`--impl reference` times the FP64 CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("field-transforms/s round trip at T639 O1280 x137 lev, split-prec vs FP64 GPU @2e-5; "
          "p99 latency")

WORKLOADS = {
    # name: (T, grid, nlat, nlon, fields, spectral decay p, seed)
    "t639_o640_548": (639, "octahedral", 1280, 0, 548, 1.5, 1002),
    "t159_reg_411": (159, "regular", 160, 320, 411, 1.0, 1001),
    "t639_o640_64": (639, "octahedral", 1280, 0, 64, 1.5, 1002),
    "t639_o640_256": (639, "octahedral", 1280, 0, 256, 1.5, 1002),
    "t639_o640_128": (639, "octahedral", 1280, 0, 128, 1.5, 1002),
    "t31_reg_10": (31, "regular", 32, 64, 10, 1.0, 1000),
    # the operational resolution of the paper's test cases: TCO1279 on O1280
    # (2560 Gaussian latitudes, rows 20 + 4i up to 5140 points), 137 levels
    "t1279_o1280_137": (1279, "octahedral", 2560, 0, 137, 1.5, 1005),
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def parse_clock_lines(lines, t0=None, t1=None):
    """Median SM clock, maximum clock and active throttle reasons of the
    nvidia-smi samples (CLOCK_FIELDS, csv, no units) stamped inside the
    window [t0, t1] (datetime; None: every sample)."""
    import datetime
    sm, smax, reasons = [], None, set()
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
        except ValueError:
            ts = None
        if ts is not None and ((t0 is not None and ts < t0) or (t1 is not None and ts > t1)):
            continue
        try:
            sm.append(float(f[2]))
            smax = float(f[3])
        except ValueError:
            continue
        for n, v in zip(CLOCK_REASONS, f[6:10]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 20 ms; start() before the
    warm-up (the tool takes a while to produce its first sample), begin() and
    end() around the timed region, whose samples alone stop() reports."""

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            import shutil
            # line-buffered, so that no sample is still in the tool's buffer when it is stopped
            pre = ["stdbuf", "-oL"] if shutil.which("stdbuf") else []
            self.proc = subprocess.Popen(pre + ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={CLOCK_FIELDS}",
                                                "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t < 5.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def begin(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def end(self):
        import datetime
        time.sleep(0.05)  # the sample of the last timed step is printed after it
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        out = parse_clock_lines(self.lines, self.t0, self.t1)
        if self.t0 is not None and self.t1 is not None:
            out["window_ms"] = round((self.t1 - self.t0).total_seconds() * 1e3, 1)
        return out


def geometry(rows, T):
    """Per northern row: M_j; per m: first northern row keeping m."""
    nlat = len(rows)
    J = nlat // 2
    M = [min(T, (rows[j] - 1) // 2) for j in range(J)]
    max_m = max(M)
    j0 = []
    for m in range(T + 1):
        j0.append(next((j for j in range(J) if M[j] >= m), J))
    return J, M, max_m, j0


# FFT lengths of the library's compile-time FP32 plans (ST_FF_PLANS): a row of
# N points runs one FFT of length N when N is one of them, else Bluestein with
# two FFTs of the shortest length >= N + 2M.  FP64 plans use 5-smooth lengths.
FF_LENGTHS = [16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1280,
              1536, 2048, 2560, 3072, 4096, 5120, 6144, 8192]


def fft_flops(rows, T, F, prec):
    """FP32 flops of one FFT stage (one direction) as the library runs it,
    5 L log2 L per complex FFT of length L, row pairs as complex sequences."""
    import math
    J = len(rows) // 2
    tot = 0.0
    for j in range(J):
        N = int(rows[j])
        M = min(T, (N - 1) // 2)
        if N in FF_LENGTHS:
            tot += 5.0 * N * math.log2(N)
        else:
            L = min((x for x in FF_LENGTHS if x >= N + 2 * M), default=None)
            if L is None:
                return None
            tot += 2 * 5.0 * L * math.log2(L) + 6.0 * L
    return tot * F if prec != "fp64" else None


def algorithmic(T, rows, F, prec):
    """Algorithmic work of one launch of each kernel for F fields (the counts
    the roofline fractions divide by)."""
    rows = [int(r) for r in rows]
    J, M, max_m, j0 = geometry(rows, T)
    npts = sum(rows)
    nspec = (T + 1) * (T + 2) // 2
    C = 2 * F
    # useful Legendre multiply-adds per direction: columns j >= j0(m) (inverse
    # outputs / direct reduction), all n in [m, T], both parities
    macs = sum((T - m + 1) * (J - j0[m]) for m in range(max_m + 1)) * C
    flops = 2.0 * macs
    split = 3.0 if prec in ("bf16x3", "tf32x3") else 1.0
    fb_vals = sum(M[j] + 1 for j in range(J)) * 2 * 2 * F  # (E,O or S,A) x (re,im)
    el = 8 if prec == "fp64" else 4
    op = {"bf16x3": 4, "tf32x3": 8, "fp32": 4, "fp64": 8}[prec]
    # Legendre HBM bytes per direction: its tables (about half the plan's), the
    # operand read and the output written (row-trimmed Fourier-buffer values)
    return {
        "leg_inv_bytes": nspec * 2 * F * op + fb_vals * el,
        "leg_dir_bytes": fb_vals * op + nspec * 2 * F * el,
        "fft_flops": fft_flops(rows, T, F, prec),
        "leg_flops": flops, "leg_tensor_flops": flops * split,
        "fft_dir_bytes": npts * F * el + fb_vals * op,
        "fft_inv_bytes": fb_vals * el + npts * F * el,
        "pack_bytes": nspec * 2 * F * (el + op),
        "unpack_bytes": nspec * 2 * F * (el + el),
    }


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle leg

def oracle_round_trip(T, grid, nlat, nlon, spec):
    import oracle
    rows = oracle.grid_rows(grid, nlat, nlon)
    mu, w = oracle.gauss(nlat)
    t0 = time.perf_counter()
    g = oracle.inv_trans(T, rows, mu, spec)
    oracle.dir_trans(T, rows, mu, w, g)
    return time.perf_counter() - t0, oracle.max_threads()


def cpu_baseline(wl, sample_fields=24):
    from paper_1908_06096_gb300 import inputs
    T, grid, nlat, nlon, F, p, seed = WORKLOADS[wl]
    n = min(sample_fields, F)
    spec = inputs.spectra(T, n, seed=seed, p=p)
    dt, cores = oracle_round_trip(T, grid, nlat, nlon, spec)
    return {"value": n / dt, "unit": "field-transforms/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} of {F} fields of workload {wl}, one round trip (inverse + direct), "
                      f"{dt:.1f} s; rate per field"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1908_06096_gb300 import inputs
    wl = args.workload
    T, grid, nlat, nlon, F, p, seed = WORKLOADS[wl]
    n = min(args.ref_fields, F)
    spec = inputs.spectra(T, n, seed=seed, p=p)
    for _ in range(args.warmup):
        oracle_round_trip(T, grid, nlat, nlon, spec)
    times, cores = [], 1
    for _ in range(args.steps):
        dt, cores = oracle_round_trip(T, grid, nlat, nlon, spec)
        times.append(dt)
    total = sum(times)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "field-transforms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, "fp64-oracle"),
            "cpu_baseline": {"value": value, "unit": "field-transforms/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {n} of {F} fields of workload {wl}, one round trip"},
            "e2e": {"value": value, "unit": "field-transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def config_of(wl, prec):
    T, grid, nlat, nlon, F, p, seed = WORKLOADS[wl]
    desc = {"t639_o640_548": "T639 octahedral O640 (1280 Gaussian latitudes, rows 20+4i), 137 levels x 4 fields",
            "t159_reg_411": "T159 regular 160 x 320 Gaussian grid, 137 levels x 3 fields",
            "t639_o640_64": "T639 octahedral O640, 64 fields (profiling case)",
            "t639_o640_256": "T639 octahedral O640, 256 fields (profiling case of the Legendre GEMM)",
            "t639_o640_128": "T639 octahedral O640, 128 fields (profiling case of the Legendre GEMM, ~3 GB)",
            "t31_reg_10": "T31 regular 32 x 64 Gaussian grid, 10 fields",
            "t1279_o1280_137": "T1279 octahedral O1280 (2560 Gaussian latitudes, rows 20+4i), 137 levels x 1 field"}[wl]
    return {"workload": desc, "T": T, "grid": grid, "nlat": nlat, "nlon": nlon or None, "fields": F,
            "spectra": f"N(0,1) (n+1)^-{p}, seed {seed}", "precision": prec,
            "step": "inverse + direct transform of every field",
            "l2": "inputs larger than L2 (no flush needed)" if F >= 64 else "L2 not flushed (small case)"}


# ------------------------------------------------------------------ GPU leg

def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1908_06096_gb300 import inputs, st
    st.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = args.workload
    T, grid, nlat, nlon, F, pdec, seed = WORKLOADS[wl]
    prec = args.precision
    pk = peaks()

    a = inputs.spectra(T, F, seed=seed + 7919 * rank, p=pdec)
    plan = st.Plan(T, grid, nlat=nlat, nlon=nlon or None, precision=prec, max_fields=F)
    if not args.no_autotune:
        # plan-time launch-shape search (FFT variants and budgets, Legendre
        # tile width), before and outside the timed region
        plan.autotune(F)
    dt = plan.dtype
    spec = torch.from_numpy(a).to(dev, dt)
    g = torch.empty((F, plan.npts), dtype=dt, device=dev)
    s_out = torch.empty((F, plan.nspec, 2), dtype=dt, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.inv(spec, out=g)
        plan.dir(g, out=s_out)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    plan.sync()
    plan.reset_timings()
    plan.set_timing(True)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.begin()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier(ws)
    ck = clocks.stop()
    plan.set_timing(False)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ws, ms)
    plan.sync()
    ktimes = plan.timings()
    value = ws * F / (ms * 1e-3)

    # per-kernel roofline from the in-library events of the timed region
    rows = plan.row_lengths()
    alg = algorithmic(T, rows, F, prec)
    tensor_peak = pk["bf16_tflops_sustained"] * (0.5 if prec == "tf32x3" else 1.0)
    # FP32 pipe: 128 FMA lanes x 2 flops per SM per clock at the maximum SM clock
    props = torch.cuda.get_device_properties(local)
    fp32_peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    tab_dir = plan.info.table_bytes / 2.0
    kern = {}
    total_k = sum(v["total_ms"] for v in ktimes.values()) or 1.0
    for name, v in ktimes.items():
        per = v["total_ms"] / max(v["timed"], 1)
        # launches: kernels; calls: stage calls timed (ms_per_launch is per call)
        e = {"launches": v["launches"], "calls": v["timed"], "ms_per_launch": per,
             "share": v["total_ms"] / total_k}
        if name.startswith("legendre") and prec in ("bf16x3", "tf32x3"):
            e.update(bound="tensor", unit="TFLOP/s", achieved=alg["leg_tensor_flops"] / (per * 1e-3) / 1e12,
                     peak=tensor_peak)
        elif name.startswith("legendre"):
            e.update(bound="alu", unit="TFLOP/s", achieved=alg["leg_flops"] / (per * 1e-3) / 1e12, peak=None)
        else:
            key = {"fft_direct": "fft_dir_bytes", "fft_inverse": "fft_inv_bytes", "pack_spectra": "pack_bytes",
                   "unpack_spectra": "unpack_bytes"}.get(name)
            if key:
                e.update(bound="hbm", unit="GB/s", achieved=alg[key] / (per * 1e-3) / 1e9, peak=pk["hbm_gbs"])
        if e.get("peak"):
            e["frac"] = e["achieved"] / e["peak"]
        # the other side of each kernel's roofline, and which one binds
        if name.startswith("legendre"):
            b = tab_dir + alg["leg_inv_bytes" if "inverse" in name else "leg_dir_bytes"]
            e["hbm"] = {"bytes": b, "achieved_gbs": b / (per * 1e-3) / 1e9,
                        "frac": b / (per * 1e-3) / 1e9 / pk["hbm_gbs"]}
            t_hbm = b / (pk["hbm_gbs"] * 1e9)
            t_ten = alg["leg_tensor_flops"] / (tensor_peak * 1e12) if e.get("bound") == "tensor" else 0.0
            e["binding"] = "hbm" if t_hbm > t_ten else e.get("bound")
            e["frac_of_binding_bound"] = max(t_hbm, t_ten) / (per * 1e-3)
        if name.startswith("fft") and alg.get("fft_flops"):
            e["fp32_pipe"] = {"flops": alg["fft_flops"], "achieved_tflops": alg["fft_flops"] / (per * 1e-3) / 1e12,
                              "peak_tflops": fp32_peak,
                              "frac": alg["fft_flops"] / (per * 1e-3) / 1e12 / fp32_peak,
                              "model": "5 L log2 L flops per complex FFT of length L as run (Bluestein: two)"}
            t_alu = alg["fft_flops"] / (fp32_peak * 1e12)
            t_hbm = alg[key] / (pk["hbm_gbs"] * 1e9)
            e["binding"] = "alu" if t_alu > t_hbm else "hbm"
            e["frac_of_binding_bound"] = max(t_alu, t_hbm) / (per * 1e-3)
            if e["binding"] == "alu":
                # the FP32 pipe binds: report that side first, the HBM side beside it
                e["hbm"] = {"bytes": alg[key], "achieved_gbs": e["achieved"], "frac": e["frac"]}
                f = e.pop("fp32_pipe")
                e.update(bound="alu", unit="TFLOP/s", achieved=f["achieved_tflops"], peak=fp32_peak,
                         frac=f["frac"], flop_model=f["model"])
        kern[name] = e
    dom = max(kern, key=lambda k: kern[k]["share"])
    d = kern[dom]
    traffic = load_traffic(dom, wl, prec)
    roof = {"kernel": dom, "bound": d.get("bound"), "achieved": d.get("achieved"), "peak": d.get("peak"),
            "unit": d.get("unit"), "frac": d.get("frac"), "traffic": traffic,
            "peak_source": ("derived: SMs x 128 FP32 lanes x 2 flops x 2.07 GHz" if d.get("bound") == "alu" else
                            f"{pk['source']} ({'bf16 sustained' if d.get('unit') == 'TFLOP/s' else 'HBM copy'})")}
    if d.get("bound") != "hbm" and d.get("hbm"):
        roof["hbm_side"] = {"achieved_gbs": d["hbm"]["achieved_gbs"], "frac": d["hbm"]["frac"]}
    launches = sum(v["launches"] for v in ktimes.values())

    # end to end through the public API with host buffers: every step copies
    # its spectra in from pinned host memory and its result back out; the
    # copies run on one copy stream (host-device copies in both directions at
    # once were slower than in turn on this machine) with double device
    # buffers, so step k's transforms overlap the input copy of step k + 1
    # and the output copy of step k - 1, as a data loader would
    h_in = torch.from_numpy(a).to(dt).pin_memory()
    h_out = [torch.empty((F, plan.nspec, 2), dtype=dt).pin_memory() for _ in range(2)]
    spec_b = [torch.empty_like(spec) for _ in range(2)]
    out_b = [torch.empty_like(s_out) for _ in range(2)]
    s_h2d = torch.cuda.Stream(dev)
    s_d2h = s_h2d
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("h2d", "comp", "d2h")}

    def e2e_run(n, start_event=None):
        for q in (s_h2d, s_d2h):
            q.wait_stream(stream)
        with torch.cuda.stream(s_h2d):
            spec_b[0].copy_(h_in, non_blocking=True)
            ev["h2d"][0].record(s_h2d)
        for k in range(n):
            b = k % 2
            if k + 1 < n:
                nb_ = (k + 1) % 2
                with torch.cuda.stream(s_h2d):
                    if k >= 1:
                        s_h2d.wait_event(ev["comp"][nb_])  # step k-1 has read that buffer
                    spec_b[nb_].copy_(h_in, non_blocking=True)
                    ev["h2d"][nb_].record(s_h2d)
            stream.wait_event(ev["h2d"][b])
            if k >= 2:
                stream.wait_event(ev["d2h"][b])  # step k-2's result has left that buffer
            plan.inv(spec_b[b], out=g)
            plan.dir(g, out=out_b[b])
            ev["comp"][b].record(stream)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(ev["comp"][b])
                h_out[b].copy_(out_b[b], non_blocking=True)
                ev["d2h"][b].record(s_d2h)
        stream.wait_stream(s_d2h)
        stream.wait_stream(s_h2d)

    e2e_run(max(1, args.warmup))
    torch.cuda.synchronize()
    barrier(ws)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(ws, e0.elapsed_time(e1) / args.steps)
    nb = F * plan.nspec * 2 * (8 if dt == torch.float64 else 4)
    e2e = {"value": ws * F / (ms_e2e * 1e-3), "unit": "field-transforms/s", "h2d_bytes_per_step": nb,
           "d2h_bytes_per_step": nb, "ms_per_step": ms_e2e,
           "copies": "pinned host buffers; H2D and D2H on one copy stream, overlapping the "
                     "neighbouring steps' transforms (double device buffers)"}

    out = {"metric": METRIC, "value": value, "unit": "field-transforms/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"bf16x3": "bf16x3 (fp32 accumulate)", "tf32x3": "tf32x3 (fp32 accumulate)",
                                           "fp32": "f32", "fp64": "f64"}[prec],
           "data": "synthetic",
           "config": dict(config_of(wl, prec), launch_shape=dict(zip(
               ["fft_inv_variant", "fft_inv_kb", "fft_dir_variant", "fft_dir_kb", "legendre_inv_tile",
                "legendre_inv_tile_high_m"],
               plan.launch_shape())), autotuned=not args.no_autotune),
           "roofline": roof, "kernels": kern,
           "e2e": e2e, "gpu_launches": launches, "clocks": ck}

    # other precision forms and the split-precision error against the FP64 GPU form
    if not args.skip_forms and prec != "fp64":
        forms = {}
        res_split = s_out.double().cpu().numpy()
        del h_in, h_out, spec_b, out_b
        for other in (["tf32x3", "fp64"] if prec == "bf16x3" else ["fp64"]):
            p2 = st.Plan(T, grid, nlat=nlat, nlon=nlon or None, precision=other, max_fields=F)
            sp2 = torch.from_numpy(a).to(dev, p2.dtype)
            g2 = torch.empty((F, p2.npts), dtype=p2.dtype, device=dev)
            o2 = torch.empty((F, p2.nspec, 2), dtype=p2.dtype, device=dev)
            nsteps = 2 if other == "fp64" else max(2, args.steps // 2)
            p2.inv(sp2, out=g2)
            p2.dir(g2, out=o2)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(nsteps):
                p2.inv(sp2, out=g2)
                p2.dir(g2, out=o2)
            e1.record(stream)
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1) / nsteps
            forms[other] = {"value": F / (ms2 * 1e-3), "ms_per_step": ms2, "steps": nsteps}
            if other == "fp64":
                # errors of the inverse (grid) and the round trip, per field, normwise
                ref_s = o2.cpu().numpy()
                gs = g.double()
                g64 = g2
                err_grid = per_field(gs, g64)
                den = np.abs(ref_s).reshape(F, -1).max(axis=1)
                err_rt = float((np.abs(res_split - ref_s).reshape(F, -1).max(axis=1) / den).max())
                out["error_vs_fp64_gpu"] = {"grid_max_rel": err_grid, "round_trip_spec_max_rel": err_rt,
                                            "bar": 2e-5, "metric": "per field max|x - x64| / max|x64|, worst field"}
            del p2, sp2, g2, o2
            torch.cuda.empty_cache()
        forms[prec] = {"value": value, "ms_per_step": ms, "steps": args.steps}
        out["forms"] = forms

    plan.close()
    del spec, g, s_out
    torch.cuda.empty_cache()
    if not args.skip_batch:
        out["batch_mixed"] = mixed_batch(args, dev)
    if not args.skip_serving:
        sv = serving(args, dev)
        out["serving"] = sv
        out["latency_ms"] = {"p50": sv["rates"]["0.7"]["p50_ms"], "p99": sv["rates"]["0.7"]["p99_ms"],
                             "at": "0.7 x saturated request rate"}

    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        try:
            out["cpu_baseline"] = cpu_baseline(wl, args.cpu_fields)
        except Exception as ex:  # report, do not hide
            out["cpu_baseline"] = {"error": repr(ex)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def mixed_batch(args, dev):
    """The 48-request mixed batch: T uniform over {79,159,255,319,511,639},
    regular (T+1) x (2T+2) or octahedral O(T+1) grids, 1-256 fields each,
    BF16x3; one round trip per request, all requests in one batch: timed as
    one persistent launch and as one launch per stage replayed from a CUDA
    graph (the two must agree bit for bit)."""
    import torch

    from paper_1908_06096_gb300 import inputs, st
    reqs = inputs.mixed_requests(48, seed=1003)
    plans, items, keep = [], [], []
    fields = 0
    for r in reqs:
        p = st.Plan(r["T"], r["grid"], precision="bf16x3", max_fields=r["nfields"])
        spec = torch.from_numpy(inputs.spectra(r["T"], r["nfields"], seed=r["seed"])).to(dev, p.dtype)
        g = torch.empty((r["nfields"], p.npts), dtype=p.dtype, device=dev)
        out = torch.empty_like(spec)
        plans.append(p)
        items.append((p, "round", spec, g, out))
        fields += r["nfields"]
    batch = st.Batch(items)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, args.steps)

    def timed(**kw):
        for _ in range(max(3, args.warmup)):
            batch.run(**kw)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            batch.run(**kw)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms_graph = timed(graph=True)
    staged = [out.clone() for (_, _, _, _, out) in items]
    try:
        ms_pers = timed(persistent=True)
        same = max(float(((a - out).abs().max() / a.abs().max()).item())
                   for a, (_, _, _, _, out) in zip(staged, items))
        pers_note = None
    except st.STError as e:
        ms_pers, same, pers_note = None, None, str(e)
    del staged
    ms = min(x for x in (ms_graph, ms_pers) if x is not None)
    # the same requests one plan call after another, for comparison
    e0.record()
    for p, _, spec, g, out in items:
        p.inv(spec, out=g)
        p.dir(g, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    batch.close()
    for p in plans:
        p.close()
    del items, plans, batch
    torch.cuda.empty_cache()
    return {"requests": len(reqs), "fields": fields, "ms_per_batch": ms,
            "field_transforms_per_s": fields / (ms * 1e-3),
            "ms_per_batch_persistent": ms_pers, "ms_per_batch_staged_graph": ms_graph,
            "persistent_vs_staged_max_rel": same, "persistent_unavailable": pers_note,
            "kernel_launches_per_run": {"persistent": 1 if ms_pers is not None else None,
                                        "staged_graph": "one per stage and FFT plan group"},
            "ms_one_call_per_request": ms_seq,
            "mix": "T uniform over {79,159,255,319,511,639}, regular or octahedral, 1-256 fields, seed 1003",
            "precision": "bf16x3",
            "launch": ("one persistent cooperative launch for the whole batch (stages separated by grid barriers)"
                       if ms == ms_pers else "one launch per stage for all requests, CUDA-graph replay"),
            "modes": "ms_per_batch is the faster of the two modes; both are timed every run"}


def serving(args, dev):
    """Serving: T uniform over {63,127,255,511,1279} on regular grids, 1-137
    fields, inverse or direct with equal odds, Poisson arrivals; BF16x3,
    tables and 4 slots' workspaces resident, request payloads in a device
    arena; the device budget is resident + arena.  The saturated rate first
    (every request present at t = 0: a throughput, no latency), then arrivals
    at 0.5 / 0.7 / 0.9 of it (10 000 requests at 0.7)."""
    import torch

    from paper_1908_06096_gb300 import inputs, serve
    arena = args.serve_arena_gb << 30
    srv = serve.Server(inputs.SERVE_T, precision="bf16x3", slots=4, max_fields=137, arena_bytes=arena)
    payloads = {}
    for T, p in srv.base.items():
        payloads[(T, "inv")] = torch.from_numpy(inputs.spectra(T, 137, seed=T)).to(torch.float32).pin_memory()
        payloads[(T, "dir")] = torch.randn((137, p.npts), generator=torch.Generator().manual_seed(T)).pin_memory()
    n = args.serve_requests
    specs = inputs.serve_requests(max(n, 1), seed=1004, rate_hz=1e12)       # all at t = 0
    srv.run(serve.make_requests(specs[:min(200, n)], payloads))              # warm-up
    nsat = min(n, 3000)
    sat = srv.run(serve.make_requests(specs[:nsat], payloads))
    rate_sat = sat["requests_per_s"]
    out = {"saturated": {k: sat[k] for k in ("requests", "fields", "wall_s", "requests_per_s",
                                             "field_transforms_per_s", "peak_inflight_bytes")},
           "rates": {}}
    for frac in (0.5, 0.7, 0.9):
        nr = n if frac == 0.7 else min(n, 3000)
        sp = inputs.serve_requests(nr, seed=1004, rate_hz=frac * rate_sat)
        res = srv.run(serve.make_requests(sp, payloads))
        res["rate_hz"] = frac * rate_sat
        out["rates"][str(frac)] = res
    out["mix"] = ("T uniform over {63,127,255,511,1279} regular grids, 1-137 fields, inverse or direct 50/50, "
                  f"Poisson arrivals, {n} requests at 0.7 of saturation, {min(n, 3000)} at 0.5 and 0.9, seed 1004")
    peak = max([sat["peak_inflight_bytes"]] + [r["peak_inflight_bytes"] for r in out["rates"].values()])
    out["server"] = {"slots": 4, "max_fields_per_call": 137, "budget_bytes": srv.budget,
                     "resident_bytes": srv.resident_bytes, "arena_bytes": srv.budget - srv.resident_bytes,
                     "peak_inflight_bytes": peak,
                     "peak_inflight_plus_resident_le_budget": peak + srv.resident_bytes <= srv.budget}
    srv.close()
    torch.cuda.empty_cache()
    return out


def per_field(x, ref):
    import torch
    F = x.shape[0]
    d = (x - ref).abs().reshape(F, -1).amax(dim=1)
    r = ref.abs().reshape(F, -1).amax(dim=1)
    return float((d / r).max().item())


def load_traffic(kernel, wl, prec):
    """dram read+write bytes per launch of `kernel` from the committed ncu
    summary (profiles/traffic.txt), or None when there is none for this
    workload or it was taken on other kernel sources than the current ones."""
    from paper_1908_06096_gb300 import build
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        fp, vals = None, {}
        with open(path) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith("# source fingerprint:"):
                    fp = line.split(":", 1)[1].strip()
                elif line and not line.startswith("#"):
                    k, w, pr, v = line.split()[:4]
                    vals[(k, w, pr)] = float(v)
        if fp != build.source_fingerprint():
            return None
        return vals.get((kernel, wl, prec))
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the plan's default launch shapes instead of the autotuned ones")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="t639_o640_548", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp32", "fp64"])
    ap.add_argument("--skip-forms", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-fields", type=int, default=24)
    ap.add_argument("--ref-fields", type=int, default=2)
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-arena-gb", type=int, default=8,
                    help="device arena for request payloads; the serving budget is resident + arena")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
