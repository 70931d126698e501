#!/usr/bin/env python
"""Throughput benchmark of the GB300 MBIR hot path.

One step = one complete reconstruction of the full-size synthetic B-scan
(1024 A-scans x 2048 spectral pixels, complex64 image 1024 x 2048, 500 seeded
beads, half the A-scans measured, 25 dB noise): power iteration for the step
size, the relative lambda rule and 100 FISTA iterations with the 3-level db4
wavelet penalty, all through the C ABI (mbir_solve).  The metric is B-scans per
second for the whole job; Phi+Phi^H pairs per second are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank reconstructs its own
B-scans (independent problems, no data-path collective): weak scaling.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "bscan-1024x2048-db4-100it-half-ascans"
METRIC = "fista_bscans_per_sec"
UNIT = "B-scans/s"
ITERS = 100
POWER_ITERS = 30
TV_ITERS = 20           # dual steps per TV prox (the library's default)
LAMBDA_FRAC = 0.01
EVAL_N = 10             # golden-section evaluations of the lambda search
EVAL_LO, EVAL_HI = -5.0, -1.0   # its bracket of log10(relative lambda)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving comparison")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32 / FP64 comparison")
    ap.add_argument("--no-tv", action="store_true", help="skip the TV-penalty solve")
    ap.add_argument("--no-hilbert", action="store_true",
                    help="skip the Hilbert-form back-projection (Phi*) measurements")
    ap.add_argument("--no-shapes", action="store_true",
                    help="skip the lateral-width (Bluestein) and 3-D volume measurements")
    ap.add_argument("--no-eval", action="store_true",
                    help="skip the evaluation loop (interpolated ISAM, NCC, lambda search)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch choices (no mbir_plan_autotune before timing)")
    ap.add_argument("--tuning", default=None, metavar="TILE,ORDER,KIND",
                    help="fix the full-size plan's launch choices (lateral tile, radix order, adjoint "
                         "kernel) instead of tuning them, e.g. to reproduce a tuned run under a profiler")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ CPU oracle leg

def oracle_setup():
    """The full-size workload as the FP64 oracle sees it: geometry, mask, operators,
    the noisy measurements and the relative lambda of the db4 penalty."""
    import numpy as np
    from oracle import fista, isam, wavelet  # noqa: F401
    from paper_2108_01438_gb300 import workloads

    wl = workloads.full_workload()
    g = isam.make_geom(wl["geom"])
    mask = wl["mask"]
    h = wavelet.daubechies_lowpass(4)
    phi = lambda v: isam.phi_nufft(v, mask, g)
    phi_adj = lambda r: isam.phi_adj_nufft(r, mask, g)
    clean = phi(wl["x_true"])
    sig = float(np.sqrt(np.mean(clean[mask == 1] ** 2)))
    y = clean + sig * 10 ** (-wl["snr_db"] / 20) * wl["noise"] * mask
    return dict(g=g, mask=mask, h=h, phi=phi, phi_adj=phi_adj, y=y, x_true=wl["x_true"])


def oracle_pair_and_lambda(o: dict) -> tuple[float, float, float]:
    """Seconds for one Phi+Phi^H pair and for the lambda rule; the lambda."""
    import numpy as np
    from oracle import wavelet
    t0 = time.perf_counter()
    o["phi_adj"](o["phi"](o["x_true"]))
    t_pair = time.perf_counter() - t0
    t0 = time.perf_counter()
    lam = LAMBDA_FRAC * float(np.max(np.abs(wavelet.dwt2(o["phi_adj"](o["y"] * o["mask"]), o["h"], 3))))
    return t_pair, time.perf_counter() - t0, lam


def oracle_iterations(o: dict, lam: float, iters: int) -> float:
    """Seconds per FISTA db4 iteration of the oracle over `iters` iterations."""
    from oracle import fista
    t0 = time.perf_counter()
    fista.fista(o["phi"], o["phi_adj"], o["y"], o["mask"], lambda v, t: fista.prox_wavelet(v, t, o["h"]), lam,
                1e-4, iters, (o["g"].nx, o["g"].nz))
    return (time.perf_counter() - t0) / iters


def solve_seconds(t_pair: float, t_lambda: float, t_iter: float) -> float:
    """One full reconstruction from its parts: the power-iteration pairs, the lambda
    rule and the FISTA iterations."""
    return POWER_ITERS * t_pair + t_lambda + ITERS * t_iter


def oracle_timing(sample_iters: int = 5) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload: one Phi+Phi^H pair,
    the lambda rule and `sample_iters` FISTA iterations (db4) of the full-size
    B-scan, then extrapolate to one full reconstruction (30 power-iteration pairs,
    the lambda rule and 100 iterations)."""
    o = oracle_setup()
    t_pair, t_lambda, lam = oracle_pair_and_lambda(o)
    t_iter = oracle_iterations(o, lam, sample_iters)
    return dict(t_pair=t_pair, t_iter=t_iter, t_lambda=t_lambda, t_solve=solve_seconds(t_pair, t_lambda, t_iter),
                sample_iters=sample_iters)


def host_cpu() -> dict:
    """The host's logical core count, the threads the oracle uses and its CPU model."""
    from oracle import isam
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "threads": isam.WORKERS, "model": model}


def workload_config() -> dict:
    """The workload every arm runs (the same dict on every line)."""
    return {"workload": WORKLOAD, "nx": 1024, "nz": 2048, "m": 2048, "penalty": "db4", "iters": ITERS,
            "power_iters": POWER_ITERS, "mask": "50% of A-scans", "l2": "flushed between steps (256 MiB write)"}


def run_reference(args, rank: int, ws: int) -> None:
    """The FP64 oracle as the reference arm, on the host cores.  One step is one
    FISTA db4 iteration of the full-size B-scan; the power-iteration pair and the
    lambda rule are timed once before the steps; the value is the B-scans per
    second of a whole reconstruction built from those parts."""
    if rank != 0:
        return
    o = oracle_setup()
    t_pair, t_lambda, lam = oracle_pair_and_lambda(o)
    times = []
    for step in range(args.warmup + args.steps):
        t = oracle_iterations(o, lam, 1)
        if step >= args.warmup:
            times.append(t)
    t_iter = statistics.mean(times)
    value = 1.0 / solve_seconds(t_pair, t_lambda, t_iter)
    cpu = host_cpu()
    sample = (f"per step: 1 FP64 FISTA db4 iteration of the 1024x2048 B-scan ({t_iter:.2f} s); one Phi+Phi^H "
              f"pair ({t_pair:.2f} s) and the lambda rule ({t_lambda:.2f} s) timed once; a reconstruction = "
              f"{POWER_ITERS} pairs + lambda + {ITERS} iterations")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu["threads"], "kind": "oracle",
                         "sample": sample, "nproc": cpu["nproc"], "cpu_model": cpu["model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clocks sampler

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int | None):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.index is not None:
            cmd += ["-i", str(self.index)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def smi_index(local_rank: int) -> int | None:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
        return None
    return local_rank


# ------------------------------------------------------------ roofline helpers

def application_bytes(nx: int, nz: int, m: int) -> dict:
    """Algorithmic bytes of the path per unit of work (FP32 path): b_x = 8 nx nz
    (complex64 image), b_y = 4 nx m (float32 measurements), the mask counted
    bit-packed (nx m / 8).  One Phi or one Phi^H: b_x + b_y + mask; one fused FISTA
    iteration: 4 b_x + 5 b_y + 2 mask (read z^k; write Phi z^k and r; read
    Phi z^{k-1} and y; read r; read z^k, z^{k-1}; write z^{k+1})."""
    bx, by, mk = 8.0 * nx * nz, 4.0 * nx * m, nx * m / 8.0
    return {"operator": bx + by + mk, "iteration": 4 * bx + 5 * by + 2 * mk}


# the operator application each kernel class belongs to (its launch is counted
# against one application's algorithmic bytes)
CLASS_APPLICATION = {
    "lateral_forward": "Phi", "row_forward": "Phi", "lateral_inverse_real": "Phi", "lateral_mid": "Phi",
    "lateral_residual": "Phi^H", "row_adjoint": "Phi^H", "lateral_adjoint": "Phi^H",
}


def algorithmic_bytes(cls: str, nx: int, nz: int, m: int) -> float | None:
    """Bytes one launch of a kernel class moves through its own operands (FP32
    path), intermediates and the resampling table included."""
    nlh = nx // 2 + 1
    img, meas = nx * nz, nx * m
    table = nlh * m * 16
    return {
        "lateral_forward": 16.0 * img,                       # read x, write X
        "row_forward": 8.0 * img + table + 8.0 * meas,       # read X, table, write S
        "lateral_inverse_real": 25.0 * meas,                 # read S, mask, y, pz; write pz, r
        "lateral_mid": 29.0 * meas,                          # read S, mask, y, pz; write pz, R
        "lateral_residual": 12.0 * meas,                     # read r, write R
        "row_adjoint": 8.0 * meas + table + 8.0 * img,       # read R, table, write W
        "lateral_adjoint": 32.0 * img,                       # read W, z1, z2; write v or z
    }.get(cls)


# sources that define each kernel class's code (its counters stay valid while these are unchanged)
_OPERATOR_SOURCES = ["common.cuh", "fft.cuh", "operator.cuh", "operator.cu", "plan.cu"]
CLASS_SOURCES = {
    "row_forward": _OPERATOR_SOURCES, "row_adjoint": _OPERATOR_SOURCES, "lateral_forward": _OPERATOR_SOURCES,
    "lateral_mid": _OPERATOR_SOURCES, "lateral_adjoint": _OPERATOR_SOURCES, "lateral_inverse_real": _OPERATOR_SOURCES,
    "lateral_residual": _OPERATOR_SOURCES, "hilbert": ["common.cuh", "fft.cuh", "operator.cuh", "hilbert.cu", "plan.cu"],
}


def source_hash(cls: str | None = None) -> str:
    """Hash of the kernel sources of one class (every csrc file when the class is unknown)."""
    csrc = os.path.join(ROOT, "paper_2108_01438_gb300", "csrc")
    names = CLASS_SOURCES.get(cls) if cls else None
    files = sorted(os.path.join(csrc, n) for n in names) if names else sorted(glob.glob(os.path.join(csrc, "*")))
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def traffic_for(cls: str) -> float | None:
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(cls)
    if not e or e.get("source_hash") != source_hash(cls) or e.get("workload") != WORKLOAD:
        return None
    return float(e["dram_bytes_per_launch"])


# ------------------------------------------------------------ uneven batch

def tune_plans(plans, enabled: bool = True) -> dict:
    """Autotune the launch choices once per shape class (mbir_plan_autotune) and
    apply the result to the class's other plans; outside every timed region."""
    done = {}
    if not enabled:
        return done
    for p in plans:
        key = (p.nx, p.nz, p.m)
        if key in done:
            p.set_tuning(done[key]["tile_c"], done[key]["lateral_order"], done[key]["adjoint_kernel"])
        else:
            done[key] = p.autotune(reps=3)
    return done


def batch_comparison(dev, stream, count: int = 64, repeats: int = 2, autotune: bool = True) -> dict:
    """The uneven-batch workload (64 B-scans, widths 256-2048, depths 1024/2048,
    l1, 100 iterations, power iteration and relative lambda per scan): one batched,
    graph-captured solve (mbir_solve_batch) against the same scans solved one at a
    time with mbir_solve.  B-scans per second for both."""
    import numpy as np
    import torch

    from paper_2108_01438_gb300 import mbir, workloads

    wls = workloads.batch_workload(count)
    plans, ys, ms = [], [], []
    for wl in wls:
        p = mbir.Plan(wl["geom"])
        x = torch.from_numpy(wl["x_true"].astype(np.complex64)).to(dev)
        m = torch.from_numpy(wl["mask"]).to(dev)
        clean = p.forward(x, m)
        sig = torch.sqrt(torch.mean(clean[m == 1].double() ** 2)).item()
        noise = torch.from_numpy(wl["noise"].astype(np.float32)).to(dev)
        ys.append((clean + float(sig * 10 ** (-wl["snr_db"] / 20)) * noise * m).contiguous())
        plans.append(p)
        ms.append(m)
    tuned = tune_plans(plans, autotune)
    outs = [torch.empty((p.nx, p.nz), dtype=torch.complex64, device=dev) for p in plans]
    kw = dict(penalties="l1", lams=LAMBDA_FRAC, relative=True, iters=ITERS, power_iters=POWER_ITERS)

    def batched():
        with torch.cuda.stream(stream):
            mbir.solve_batch(plans, ys, ms, outs=outs, stream=stream, **kw)

    def sequential():
        with torch.cuda.stream(stream):
            for p, y, m, o in zip(plans, ys, ms, outs):
                p.solve(y, m, penalty="l1", lam=LAMBDA_FRAC, relative=True, iters=ITERS,
                        power_iters=POWER_ITERS, out=o, stream=stream)

    res = {}
    for name, fn in (("batched", batched), ("sequential", sequential)):
        fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(repeats):
            fn()
        e1.record(stream)
        stream.synchronize()
        res[name] = count * repeats / (e0.elapsed_time(e1) / 1e3)
    for p in plans:
        p.close()
    pix = sum(w["geom"]["nx"] * w["geom"]["nz"] for w in wls)
    return {"workload": f"{count} uneven B-scans, widths 256-2048, depths 1024/2048, l1, {ITERS} iterations",
            "image_megapixels": round(pix / 1e6, 2), "shape_classes_tuned": len(tuned),
            "batched_bscans_per_sec": res["batched"],
            "sequential_bscans_per_sec": res["sequential"], "speedup": res["batched"] / res["sequential"]}


# ------------------------------------------------------------ precision

def precision_comparison(dev, stream, repeats: int = 20) -> dict:
    """The 64 x 256 point-scatterer workload (l1, relative lambda, power iteration)
    solved with FP32, FP32 with compensated KB accumulation and FP64 plans: the
    relative L2 distance of the FP32 reconstructions to the FP64 one after 10 / 50 /
    100 iterations, and solves per second of each precision (throughput ratio
    FP32 / FP64)."""
    import numpy as np
    import torch

    from paper_2108_01438_gb300 import mbir, workloads

    wl = workloads.tiny_workload()
    out = {"workload": "64x256 point scatterers, l1, relative lambda 0.01, power iteration"}
    recon, rate = {}, {}
    for name, mode in (("fp32", mbir.FP32), ("fp32c", mbir.FP32_COMPENSATED), ("fp64", mbir.FP64)):
        plan = mbir.Plan(wl["geom"], precision=mode, stream=stream)
        cdt = torch.complex128 if mode == mbir.FP64 else torch.complex64
        x = torch.from_numpy(wl["x_true"]).to(cdt).to(dev)
        with torch.cuda.stream(stream):
            y = plan.forward(x, stream=stream)
            noise = torch.from_numpy(wl["noise"]).to(y.dtype).to(dev)
            y = (y + 0.01 * noise).contiguous()
            recon[name] = {}
            _, info = plan.solve(y, penalty="l1", lam=LAMBDA_FRAC, iters=1, stream=stream)
            for k in (10, 50, 100):
                z, _ = plan.solve(y, penalty="l1", lam=info["lambda_used"], relative=False, iters=k,
                                  step=info["step"], stream=stream)
                recon[name][k] = z.to(torch.complex128)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(repeats):
                plan.solve(y, penalty="l1", lam=LAMBDA_FRAC, iters=100, stream=stream)
            e1.record(stream)
        stream.synchronize()
        rate[name] = repeats / (e0.elapsed_time(e1) / 1e3)
        plan.close()
    for name in ("fp32", "fp32c"):
        out[f"{name}_vs_fp64_rel_l2"] = {str(k): float(torch.linalg.norm(recon[name][k] - recon["fp64"][k]) /
                                                       torch.linalg.norm(recon["fp64"][k])) for k in (10, 50, 100)}
    out["solves_per_sec"] = rate
    out["fp32_over_fp64_throughput"] = rate["fp32"] / rate["fp64"]
    return out


# ------------------------------------------------------------ serving

def serve_stream(srv, reqs, arrivals, outs, kw) -> tuple[dict, dict, float]:
    """Feed `reqs` to the server at their scheduled arrival times (seconds from the
    start), one batched iteration per tick; latency runs from a request's scheduled
    arrival to its completion.  Returns latencies, iteration counts, wall seconds."""
    n = len(reqs)
    lat, iters, t_submit, tickets = {}, {}, {}, {}
    nxt = 0
    t0 = time.perf_counter()
    while len(lat) < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            p, y, m, pen = reqs[nxt]
            tickets[nxt] = srv.submit(p, y, m, outs[nxt], penalty=pen, **kw)
            t_submit[nxt] = now
            nxt += 1
        if not tickets:
            time.sleep(max(0.0, arrivals[nxt] - now))
            continue
        srv.step()
        for i, t in list(tickets.items()):
            r = srv.poll(t)
            if r is not None:
                lat[i] = (t_submit[i] - arrivals[i]) + r[2]
                iters[i] = r[1]["iters"]
                del tickets[i]
    return lat, iters, time.perf_counter() - t0


def serve_comparison(dev, stream, n_req: int = 2000, rate_hz: float = 200.0, low_rate_hz: float = 30.0,
                     n_low: int = 400, budget_bytes: int = 150 * 10 ** 9, autotune: bool = True,
                     pool_size: int = 64) -> dict:
    """A seeded Poisson stream of single B-scan solves (widths from 12 of the 7-smooth
    multiples of 8 in [128, 2048], 1024 or 2048 spectral pixels, l1 / db4 half and
    half, relative-objective tolerance 1e-4 within 30-150 iterations) served with
    continuous batching under a 150 GB budget, after a warm-up of two requests per
    shape.  Requests draw their data from a pool of `pool_size` seeded B-scans.
    Two operating points: `n_req` requests at `rate_hz` (above the GPU's capacity:
    latency is mostly queueing) and `n_low` requests at `low_rate_hz` (below it:
    latency is service).  The first stream's requests are then solved one after
    another with mbir_solve for the sequential rate."""
    import numpy as np
    import torch

    from paper_2108_01438_gb300 import mbir, workloads

    rng = np.random.default_rng(workloads.BASE_SEED + 5)
    widths = sorted(rng.choice(workloads.smooth_widths(128, 2048), 12, replace=False).tolist())
    plans, pool = {}, []
    for j in range(pool_size):
        nx, nz = int(rng.choice(widths)), int(rng.choice([1024, 2048]))
        if (nx, nz) not in plans:
            plans[(nx, nz)] = mbir.Plan(workloads.geometry(nx, nz, nz))
        p = plans[(nx, nz)]
        x = torch.from_numpy(workloads.point_scatterers(nx, nz, 40, 10_000 + j).astype(np.complex64)).to(dev)
        m = torch.from_numpy(workloads.mask_bernoulli(nx, nz, 0.5, 20_000 + j)).to(dev)
        clean = p.forward(x, m)
        sig = torch.sqrt(torch.mean(clean[m == 1].double() ** 2)).item()
        noise = torch.from_numpy(workloads.unit_noise(nx, nz, 30_000 + j).astype(np.float32)).to(dev)
        y = (clean + float(sig * 10 ** (-30.0 / 20)) * noise * m).contiguous()
        pool.append((p, y, m, "l1" if j % 2 == 0 else "db4"))
    torch.cuda.synchronize()
    tune_plans(list(plans.values()), autotune)
    kw = dict(lam=LAMBDA_FRAC, relative=True, iters=150, min_iter=30, rel_tol=1e-4, power_iters=POWER_ITERS)

    def stream_of(n, rate, seed):
        r = np.random.default_rng(seed)
        arrivals = np.cumsum(r.exponential(1.0 / rate, n))
        reqs = [pool[int(k)] for k in r.integers(0, pool_size, n)]
        return reqs, arrivals

    srv = mbir.Server(budget_bytes, stream=stream)
    res = {}
    with torch.cuda.stream(stream):
        # warm-up: two requests of every shape, served and drained
        seen, wreqs = {}, []
        for q in pool:
            if seen.get(id(q[0]), 0) < 2:
                seen[id(q[0])] = seen.get(id(q[0]), 0) + 1
                wreqs.append(q)
        wouts = [torch.empty((q[0].nx, q[0].nz), dtype=torch.complex64, device=dev) for q in wreqs]
        serve_stream(srv, wreqs, np.zeros(len(wreqs)), wouts, kw)
        del wouts
        for name, (n, rate, seed) in (("overload", (n_req, rate_hz, 51)), ("underload", (n_low, low_rate_hz, 52))):
            reqs, arrivals = stream_of(n, rate, seed)
            outs = [torch.empty((q[0].nx, q[0].nz), dtype=torch.complex64, device=dev) for q in reqs]
            peak0 = srv.stats()["peak_bytes"]
            lat, iters, wall = serve_stream(srv, reqs, arrivals, outs, kw)
            L = np.array([lat[i] for i in range(n)])
            res[name] = {"requests": n, "rate_hz": rate,
                         "latency_s": {"p50": float(np.percentile(L, 50)), "p99": float(np.percentile(L, 99))},
                         "served_bscans_per_sec": n / (wall - arrivals[0]),
                         "mean_iters": float(np.mean(list(iters.values())))}
            if name == "overload":
                over_reqs, over_outs = reqs, outs
            else:
                del outs
    peak = srv.stats()["peak_bytes"]
    srv.close()

    t1 = time.perf_counter()
    with torch.cuda.stream(stream):
        for (p, y, m, pen), o in zip(over_reqs, over_outs):
            p.solve(y, m, penalty=pen, out=o, iters=150, min_iter=30, rel_tol=1e-4, lam=LAMBDA_FRAC,
                    relative=True, power_iters=POWER_ITERS, stream=stream)
    stream.synchronize()
    sequential = len(over_reqs) / (time.perf_counter() - t1)
    for p in plans.values():
        p.close()
    over = res["overload"]
    return {"workload": f"Poisson requests, widths 128-2048, depths 1024/2048, l1/db4, rel_tol 1e-4 in "
                        f"30-150 iterations, 150 GB budget, data from {pool_size} seeded B-scans, "
                        "warm-up of two requests per shape",
            "latency_s": over["latency_s"], "served_bscans_per_sec": over["served_bscans_per_sec"],
            "sequential_bscans_per_sec": sequential, "speedup": over["served_bscans_per_sec"] / sequential,
            "mean_iters": over["mean_iters"], "requests": over["requests"], "rate_hz": over["rate_hz"],
            "underload": res["underload"], "peak_bytes": int(peak)}


# ------------------------------------------------------------ our arm

# ------------------------------------------------------------ other shapes

def shapes_section(dev, stream, peak: float) -> dict:
    """Shapes beyond the B-scan workload, with the data of Sec. 3.1 in mind (1024 x 1024
    A-scans): a lateral width with a prime factor above 7, whose lateral transform runs
    in the Bluestein form (1021), beside the 7-smooth width next to it (1024), both at
    2048 depth pixels; and a 256 x 256 x 512 volume (a 2-D lateral transform).  Phi +
    Phi^H pairs per second, back to back, against the algorithmic bytes of a pair,
    2 (b_x + b_y + bit-packed mask); for the volume also an l1 FISTA solve."""
    import torch

    from paper_2108_01438_gb300 import mbir, workloads

    def pair_ms(plan, x, mask, yshape, n):
        y = torch.empty(yshape, dtype=plan.real_dtype, device=dev)
        xa = torch.empty_like(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(3):
                plan.forward(x, mask, out=y, stream=stream)
                plan.adjoint(y, mask, out=xa, stream=stream)
            e0.record(stream)
            for _ in range(n):
                plan.forward(x, mask, out=y, stream=stream)
                plan.adjoint(y, mask, out=xa, stream=stream)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / n

    def entry(ms, nvox, nmeas, extra):
        alg = 2 * (8 * nvox + 4 * nmeas + nmeas / 8)
        gbs = alg / (ms * 1e-3) / 1e9
        return dict(extra, pairs_per_sec=1e3 / ms, ms_per_pair=ms, alg_bytes_per_pair=alg, achieved_gbs=gbs,
                    frac=gbs / peak)

    gen = torch.Generator(device=dev)
    gen.manual_seed(2108)
    res = {}
    for nx in (1021, 1024):
        d = workloads.geometry(nx, 2048, 2048)
        plan = mbir.Plan(d)
        x = torch.randn((nx, 2048), dtype=torch.complex64, device=dev, generator=gen)
        mask = torch.from_numpy(workloads.mask_ascans(nx, 2048, 0.5, 7)).to(dev)
        ms = pair_ms(plan, x, mask, (nx, 2048), 100)
        res[f"bscan_{nx}x2048"] = entry(ms, nx * 2048, nx * 2048, {
            "lateral_transform": "Bluestein (chirp-z, length 2048)" if nx == 1021 else "mixed radix"})
        plan.close()
    nx, ny, nz = 256, 256, 512
    d = workloads.geometry(nx, nz, nz)
    vol = mbir.VolumePlan(d, ny)
    x = torch.randn((nx, ny, nz), dtype=torch.complex64, device=dev, generator=gen)
    mask = (torch.rand((nx, ny, nz), device=dev, generator=gen) < 0.5).to(torch.uint8)
    ms = pair_ms(vol, x, mask, (nx, ny, nz), 10)
    v = entry(ms, nx * ny * nz, nx * ny * nz, {"l2": "image 268 MB, larger than L2"})
    # l1 FISTA on a sparse volume: 2000 unit scatterers of random phase, half of the samples
    xt = torch.zeros((nx * ny * nz,), dtype=torch.complex64, device=dev)
    idx = torch.randperm(nx * ny * nz, device=dev, generator=gen)[:2000]
    ph = torch.rand((2000,), device=dev, generator=gen) * 6.283185307179586
    xt[idx] = torch.polar(torch.ones_like(ph), ph)
    y = vol.forward(xt.view(nx, ny, nz), mask)
    iters, power = 20, 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        vol.solve(y, mask, lam=0.01, relative=True, iters=2, power_iters=2, stream=stream)
        e0.record(stream)
        _, info = vol.solve(y, mask, lam=0.01, relative=True, iters=iters, power_iters=power, stream=stream)
        e1.record(stream)
    stream.synchronize()
    solve_ms = e0.elapsed_time(e1)
    v["fista_l1"] = {"iters": iters, "power_iters": power, "ms_per_solve": solve_ms,
                     "voxel_iterations_per_sec": nx * ny * nz * (iters + power) / (solve_ms * 1e-3),
                     "note": "each FISTA and power step is one volume Phi and one volume Phi^H"}
    res[f"volume_{nx}x{ny}x{nz}"] = v
    vol.close()
    return res


def run_ours(args, rank: int, ws: int, local: int) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2108_01438_gb300 import mbir, workloads

    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        from paper_2108_01438_gb300 import build
        build.build()
    if ws > 1:
        dist.barrier()
    mbir.lib()

    wl = workloads.full_workload(seed_offset=1 + rank)
    d = wl["geom"]
    nx, nz, m = d["nx"], d["nz"], d["m"]
    plan = mbir.Plan(d)
    # launch choices for this shape class, timed before anything else (not in the timed region)
    if args.tuning:
        t, o, k = (int(v) for v in args.tuning.split(","))
        plan.set_tuning(t, o, k)
        tuning = {"tile_c": t, "lateral_order": o, "adjoint_kernel": k}
    else:
        tuning = None if args.no_autotune else plan.autotune(reps=5)
    stream = torch.cuda.current_stream()
    x_true = torch.from_numpy(wl["x_true"].astype(np.complex64)).to(dev)
    mask = torch.from_numpy(wl["mask"]).to(dev)
    clean = plan.forward(x_true, mask)
    sig = torch.sqrt(torch.mean(clean[mask == 1].double() ** 2)).item()
    noise = torch.from_numpy(wl["noise"].astype(np.float32)).to(dev)
    y = (clean + float(sig * 10 ** (-wl["snr_db"] / 20)) * noise * mask).contiguous()
    out = torch.empty((nx, nz), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        plan.solve(y, mask, penalty="db4", lam=LAMBDA_FRAC, relative=True, iters=ITERS,
                   power_iters=POWER_ITERS, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-class launch times from one instrumented solve outside the timed region
    # (an event pair around every launch would slow the timed steps down)
    plan.profile_begin(1 << 16)
    step()
    prof = plan.profile_end()
    dom_cls = max(prof.items(), key=lambda kv: kv[1][1])[0]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(smi_index(local))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()                       # evict the previous step's data from L2
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # the same steps again with an event pair around each launch of the dominant
    # class only (events between launches would cut the programmatic-launch
    # overlap inside the timed steps above): its mean launch time
    plan.profile_begin(1 << 17)
    plan.profile_only(dom_cls)
    for i in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof_dom = plan.profile_end()
    # the mean FISTA iteration alone (fixed step and lambda): 100 minus 10 iterations
    _, info_ref = plan.solve(y, mask, penalty="db4", lam=LAMBDA_FRAC, relative=True, iters=1,
                             power_iters=POWER_ITERS, out=out)
    it_ms = {}
    for n_it in (10, ITERS):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for _ in range(3):
            plan.solve(y, mask, penalty="db4", lam=info_ref["lambda_used"], relative=False, iters=n_it,
                       step=info_ref["step"], out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        it_ms[n_it] = e0.elapsed_time(e1) / 3
    iter_ms = (it_ms[ITERS] - it_ms[10]) / (ITERS - 10)
    total_s = sum(step_ms) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_max = float(t.item())
    value = ws * args.steps / total_max

    # Phi + Phi^H pairs per second on the same B-scan (operators alone)
    xa = torch.empty_like(out)
    for _ in range(3):
        plan.forward(out, mask, out=y.new_empty(y.shape))
    pairs = 200
    yb = torch.empty_like(y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(pairs):
        plan.forward(out, mask, out=yb)
        plan.adjoint(yb, mask, out=xa)
    e1.record(stream)
    torch.cuda.synchronize()
    pair_ms = e0.elapsed_time(e1) / pairs

    # the isotropic TV penalty on the same B-scan (Sec. 2.2): a whole solve, and the
    # TV prox kernels against the HBM roof (they stream the dual fields)
    tv_res = None
    if not args.no_tv:
        tv_kw = dict(penalty="tv", lam=LAMBDA_FRAC, relative=True, iters=ITERS, power_iters=POWER_ITERS,
                     out=out, tv_iters=TV_ITERS)
        plan.solve(y, mask, **tv_kw)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(2):
            flush.zero_()
            plan.solve(y, mask, **tv_kw)
        t1.record(stream)
        torch.cuda.synchronize()
        tv_solve_ms = t0.elapsed_time(t1) / 2
        plan.profile_begin(1 << 14)
        plan.profile_only("tv_prox")
        plan.solve(y, mask, **tv_kw)
        torch.cuda.synchronize()
        n_launch, tv_total_ms = plan.profile_end()["tv_prox"]
        per_prox = TV_ITERS // 2 + TV_ITERS % 2 + 1      # two-step passes, an odd last step, the finish
        n_prox = n_launch / per_prox
        # bytes a prox must move per pixel (FP32): the first two-step pass reads v and
        # writes p_1, p_2 (40); later two-step passes read p_{k-1}, p_{k-2}, v and write
        # p_k, p_{k+1} (72); an odd last step reads p_{k-1}, p_{k-2}, v and writes p_k
        # (56); the finishing pass reads p and v and writes z (32)
        pairs = TV_ITERS // 2
        bpp = (40 + 72 * (pairs - 1) if pairs else 0) + (TV_ITERS % 2) * (56 if pairs else 24) + 32
        prox_ms = tv_total_ms / n_prox
        peak_gbs = measured_peak()[0]
        gbs = bpp * nx * nz / (prox_ms * 1e-3) / 1e9
        tv_res = {"workload": f"bscan-1024x2048-tv-{ITERS}it-half-ascans, {TV_ITERS} dual steps per prox",
                  "bscans_per_sec": 1e3 / tv_solve_ms, "ms_per_solve": tv_solve_ms,
                  "prox_ms": prox_ms, "prox_launches": per_prox,
                  "roofline": {"bound": "hbm", "kernel": "tv_prox", "achieved": gbs, "peak": peak_gbs,
                               "unit": "GB/s", "frac": gbs / peak_gbs, "alg_bytes_per_prox": bpp * nx * nz}}

    # the paper's back-projection Phi* = B^H A(s .) (Eq. back_model) on the same B-scan:
    # Phi + Phi* pairs, a db4 solve with Phi* in the gradient, the Hilbert kernel
    # against the HBM roof, and how far Phi* is from 2 Phi^H on these measurements
    hil_res = None
    if not args.no_hilbert:
        xh = torch.empty_like(out)
        plan.adjoint_hilbert(y, mask, out=xh)
        e0.record(stream)
        for _ in range(pairs):
            plan.forward(out, mask, out=yb)
            plan.adjoint_hilbert(yb, mask, out=xh)
        e1.record(stream)
        torch.cuda.synchronize()
        hpair_ms = e0.elapsed_time(e1) / pairs
        plan.profile_begin(4096)
        plan.profile_only("hilbert")
        for _ in range(20):
            plan.adjoint_hilbert(yb, mask, out=xh)
        torch.cuda.synchronize()
        n_h, h_ms = plan.profile_end()["hilbert"]
        h_avg = h_ms / n_h
        # y (4 B) and the mask (1 B) in, A(s y) (8 B) out, per sample
        h_bytes = 13.0 * nx * m
        peak_gbs = measured_peak()[0]
        h_gbs = h_bytes / (h_avg * 1e-3) / 1e9
        hil_kw = dict(penalty="db4", lam=LAMBDA_FRAC, relative=True, iters=ITERS, power_iters=POWER_ITERS,
                      out=out, backprojection="hilbert")
        plan.solve(y, mask, **hil_kw)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        t0.record(stream)
        for _ in range(2):
            plan.solve(y, mask, **hil_kw)
        t1.record(stream)
        torch.cuda.synchronize()
        hsolve_ms = t0.elapsed_time(t1) / 2
        plan.adjoint_hilbert(clean, mask, out=xh)
        plan.adjoint(clean, mask, out=xa)
        gap = (torch.linalg.vector_norm(xh - 2 * xa) / torch.linalg.vector_norm(2 * xa)).item()
        hil_res = {"workload": f"bscan-1024x2048-db4-{ITERS}it-half-ascans, Phi* in the gradient",
                   "bscans_per_sec": 1e3 / hsolve_ms, "ms_per_solve": hsolve_ms,
                   "pairs_per_sec": 1e3 / hpair_ms, "hilbert_ms": h_avg,
                   "rel_gap_to_twice_transpose": gap,
                   "roofline": {"bound": "hbm", "kernel": "hilbert", "achieved": h_gbs, "peak": peak_gbs,
                                "unit": "GB/s", "frac": h_gbs / peak_gbs, "alg_bytes": h_bytes,
                                "traffic": traffic_for("hilbert")}}

    # the evaluation loop of Sec. 3 on the same phantom with the paper's three
    # sub-sampling schemes (half of the spectrometer samples each): the
    # interpolated-ISAM baseline, and MBIR (db4, TV) at the lambda a golden-section
    # search finds best, as in the paper's NCC table
    # The phantom is the 500 beads without the random-phase background: a background
    # whose phase changes from pixel to pixel is white across the whole band, which
    # the band-limited, sub-sampled system cannot represent, and its speckle then
    # dominates every magnitude NCC and flattens the search.
    eval_res = None
    if not args.no_eval:
        eval_res = {"workload": "bscan-1024x2048, 500 beads on a zero background, 25 dB, half of the "
                                "spectrometer samples per scheme",
                    "search": {"log10_bracket": [EVAL_LO, EVAL_HI], "evaluations": EVAL_N, "iters": ITERS}}
        x_eval = torch.from_numpy(workloads.beads(nx, nz, 500, workloads.BASE_SEED + 1, background=0.0)
                                  .astype(np.complex64)).to(dev)
        schemes = {"random": workloads.mask_bernoulli(nx, m, 0.5, 4242),
                   "equispaced": workloads.mask_equispaced(nx, m), "partial": workloads.mask_partial(nx, m)}
        for scheme, mk in schemes.items():
            mask_r = torch.from_numpy(mk).to(dev)
            clean_r = plan.forward(x_eval, mask_r)
            sig_r = torch.sqrt(torch.mean(clean_r[mask_r == 1].double() ** 2)).item()
            y_r = (clean_r + float(sig_r * 10 ** (-wl["snr_db"] / 20)) * noise * mask_r).contiguous()
            base = plan.isam_interpolated(y_r, mask_r)
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(10):
                plan.isam_interpolated(y_r, mask_r, out=base)
            t1.record(stream)
            torch.cuda.synchronize()
            row = {"isam_interpolated": {"ncc": plan.ncc(base, x_eval), "ms": t0.elapsed_time(t1) / 10}}
            for pen in ("db4", "tv"):
                t_start = time.perf_counter()
                _, info = plan.lambda_search(y_r, mask_r, x_eval, lo=EVAL_LO, hi=EVAL_HI, n_eval=EVAL_N,
                                             penalty=pen, iters=ITERS, power_iters=POWER_ITERS, tv_iters=TV_ITERS)
                row["mbir_" + pen] = {"ncc": info["ncc"], "lambda_rel": info["lambda_rel"],
                                      "search_s": time.perf_counter() - t_start,
                                      "trace_ncc": [round(v, 5) for v in info["trace_ncc"].tolist()]}
            eval_res[scheme] = row

    # end to end through host buffers: pinned inputs in, reconstruction out, each step
    y_host = y.cpu().pin_memory()
    m_host = mask.cpu().pin_memory()
    x_host = torch.empty((nx, nz), dtype=torch.complex64).pin_memory()
    y_dev, m_dev = torch.empty_like(y), torch.empty_like(mask)
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        e_ev[i][0].record(stream)
        y_dev.copy_(y_host, non_blocking=True)
        m_dev.copy_(m_host, non_blocking=True)
        plan.solve(y_dev, m_dev, penalty="db4", lam=LAMBDA_FRAC, relative=True, iters=ITERS,
                   power_iters=POWER_ITERS, out=out)
        x_host.copy_(out, non_blocking=True)
        e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_s = sum(a.elapsed_time(b) for a, b in e_ev) / 1e3
    t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = ws * args.steps / float(t.item())

    # every step runs the same launches as the instrumented solve
    launches = args.steps * sum(v[0] for v in prof.values())
    dom_n, dom_ms = prof_dom[dom_cls]
    avg_ms = dom_ms / dom_n
    app = application_bytes(nx, nz, m)
    operand = algorithmic_bytes(dom_cls, nx, nz, m)
    peak, peak_kind = measured_peak()
    roofline = None
    if dom_cls in CLASS_APPLICATION:
        # one launch of the dominant class against the algorithmic bytes of the one
        # operator application it is part of
        alg = app["operator"]
        achieved = alg / (avg_ms * 1e-3) / 1e9
        traffic = traffic_for(dom_cls)
        it_gbs = app["iteration"] / (iter_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom_cls, "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                    "alg_bytes": alg,
                    "alg_bytes_basis": f"one {CLASS_APPLICATION[dom_cls]}: b_x + b_y + bit-packed mask",
                    "avg_launch_ms": avg_ms, "launches_timed": dom_n,
                    "operand_bytes": operand,
                    "operand_frac": None if operand is None else operand / (avg_ms * 1e-3) / 1e9 / peak,
                    "dram_frac": None if traffic is None else traffic / (avg_ms * 1e-3) / 1e9 / peak,
                    "iteration": {"alg_bytes": app["iteration"], "ms": iter_ms, "achieved": it_gbs,
                                  "frac": it_gbs / peak,
                                  "basis": "4 b_x + 5 b_y + 2 bit-packed masks per FISTA iteration"}}

    batch = None
    if not args.no_batch:
        batch = batch_comparison(dev, torch.cuda.Stream(device=dev), autotune=not args.no_autotune)
    precision = None
    if not args.no_precision:
        precision = precision_comparison(dev, torch.cuda.Stream(device=dev))
    serve = None
    if not args.no_serve:
        serve = serve_comparison(dev, torch.cuda.Stream(device=dev), n_req=args.serve_requests,
                                 autotune=not args.no_autotune)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ot = oracle_timing(sample_iters=5)
        hc = host_cpu()
        cpu = {"value": 1.0 / ot["t_solve"], "unit": UNIT, "cores": hc["threads"], "kind": "oracle",
               "sample": ("one FP64 Phi+Phi^H pair, the lambda rule and %d FISTA db4 iterations of the "
                          "1024x2048 B-scan (%.1f s), extrapolated to %d pairs + lambda + %d iterations"
                          % (ot["sample_iters"], ot["t_pair"] + ot["t_lambda"] + ot["sample_iters"] * ot["t_iter"],
                             POWER_ITERS, ITERS)),
               "pairs_per_sec": 1.0 / ot["t_pair"], "nproc": hc["nproc"], "cpu_model": hc["model"]}

    shapes = None
    if rank == 0 and not args.no_shapes:
        # last: these sizes run nowhere else in the bench
        try:
            shapes = shapes_section(dev, torch.cuda.Stream(device=dev), peak)
        except Exception as exc:   # report, keep the line
            shapes = {"error": str(exc)[:300]}

    if rank == 0:
        step_sorted = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_max * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(),
            "launch_tuning": None if tuning is None else
            {k: tuning[k] for k in ("tile_c", "lateral_order", "adjoint_kernel")},
            "pairs_per_sec": ws * 1e3 / pair_ms,
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))]},
            "kernels_ms_per_launch": {k: v[1] / v[0] for k, v in prof.items()},
            "batch": batch,
            "serve": serve,
            "precision": precision,
            "tv": tv_res,
            "hilbert": hil_res,
            "evaluation": eval_res,
            "shapes": shapes,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": y.numel() * 4 + mask.numel(),
                    "d2h_bytes_per_step": out.numel() * 8},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    run_ours(args, rank, ws, local)


if __name__ == "__main__":
    main()
