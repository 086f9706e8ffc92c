"""Throughput of the fused phase-field LBM step on GB300, one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--form F] [--storage fp32|fp16|bf16]

Metric: GLUPS = (lattice nodes x time steps) / second, one coupled f + h
update per node and step.  A step is one pass of the whole hot path: one
fused kernel launch (moments, central-scheme derivatives, interfacial force,
collision and streaming of both D2Q9 populations) over the workload's grid.

Default workload: the plain-FP32 capillary-wave / rising-bubble configuration
at scale, 512 x 1024 nodes, walls at bottom and top, rising bubble R = 64,
W = 5, sigma = 1e-3, M = 0.05, g = 1e-6, seeded 1e-3 noise on phi0 (density
ratio 10 with equal kinematic viscosities: the stated ratio 1000 diverges).
Its state (84 MB double-buffered) fits in the 129 MB L2, so L2 is flushed
before every timed step: a 256 MB buffer is written (evicting the state), then
another 256 MB buffer is read, so that the step starts with none of its data
in L2 and no dirty line of the flush left for it to write back.  Each step is
timed with CUDA events on the domain's stream around its single kernel
launch.

The line also carries "l2_exceeding": the same physics on 2048 x 4096 nodes
(1.34 GB of state per step, larger than L2), timed over consecutive steps,
and "cpu_baseline" times the FP64 oracle on all host cores and on one.

Multi-GPU (torchrun, one rank per GPU): every rank advances its own replica
of the workload, no data-path collective (the instances are independent);
value = all ranks' node-steps / max over ranks of the time ("scaling":
"weak").

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the host cores, on a bounded sample of the same workload.
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

from paper_2012_14729_gb300 import workloads as wl  # noqa: E402

BYTES_PER_LUP = {"fp32": 160, "fp16": 92, "bf16": 92}
L2_FLUSH_BYTES = 256 << 20


class ColdL2:
    """Flush L2 before a timed step: write one buffer larger than L2, then
    read another, which replaces the written (dirty) lines by clean ones."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.int64, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()


def make_case(name: str, form: str):
    if name == "bubble_512x1024":
        return wl.capillary_bubble("bubble", form=form)
    if name == "wave_512x1024":
        return wl.capillary_bubble("wave", form=form)
    if name == "bubble_4096x2048":
        # same physics as the default at 16x the nodes (state 1.3 GB > L2)
        return wl.capillary_bubble("bubble", form=form, nx=2048, ny=4096, R=256.0)
    if name == "bubble_2048x1024":
        # 4x the default's nodes, state 0.34 GB per buffer (> L2): DRAM traffic capture
        return wl.capillary_bubble("bubble", form=form, nx=1024, ny=2048, R=128.0)
    if name == "rising_bubble_120x240":
        # Sec. 5.4 geometry: free-slip side walls, no-slip top and bottom
        return wl.rising_bubble(form=form, nx=120)
    if name == "rising_bubble_2048x4096":
        # the same geometry at 8.4 M nodes (state 1.34 GB per step, > L2)
        return wl.rising_bubble(form=form, nx=2048)
    if name == "drop_64x64":
        return wl.stationary_drop(form)
    if name == "merging_256x128":
        return wl.merging_drops(form)
    raise SystemExit(f"unknown workload {name}")


def walls_name(case) -> str:
    w = ["x free-slip"] if case.meta.get("wall_x", False) else []
    if case.wall_y:
        w.append("y")
    return "+".join(w) if w else "none"


def time_bubble_diagnostics(dom, case, calls=20):
    """Wall time of one pflbm_bubble_diagnostics call (field staging, the
    FP64 reduction over nodes and cells, the read-back of 8 sums; it
    synchronises), mean over `calls`, with the quantities in SI units."""
    dom.bubble_diagnostics()
    t0 = time.perf_counter()
    for _ in range(calls):
        g = dom.bubble_diagnostics()
    ms = (time.perf_counter() - t0) / calls * 1e3
    m = case.meta
    return {"ms_per_call": ms, "calls": calls, "status": g["status"],
            "yc_m": (g["yc2"] + 0.5) * m["m_per_node"], "vc_mps": g["vc2"] * m["mps_per_lattice"],
            "circularity": g["circularity"]}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# the step kernel each stage mode launches (the dominant kernel of a step)
KERNEL_OF_STAGE = {"boxes": "k_step_boxes", "gather": "k_step_gather", "march": "k_step_march",
                   "gather8": "k_step_gather"}


# the sources the step kernels are compiled from
KERNEL_SOURCES = ("step_kernel.cuh", "lattice.cuh", "march_kernel.cuh")


def kernel_sha() -> str:
    """Hash (16 hex digits) of the step kernels' sources."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2012_14729_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(workload: str, storage: str, stage: str):
    """DRAM bytes per node and step of the step kernel from the committed ncu
    summary of this workload, valid only while the kernel sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        sha = kernel_sha()
        r = rec.get(f"{workload}/{storage}/{stage}")
        if r and r.get("kernel_sha") == sha:
            return float(r["dram_bytes_per_lup"])
    except (OSError, ValueError):
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[4:8]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """The job's value of a per-rank time: its maximum over the ranks (an
    all-reduce on the initialised process group; the value itself on one)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int, device) -> float:
    """Sum of a per-rank count over the ranks (the value itself on one)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n: int, rank: int, ws: int):
    """The contiguous share [lo, hi) of n independent items (the instances of
    a batch) that rank `rank` of `ws` advances: sizes differ by at most one,
    the shares are disjoint and cover [0, n)."""
    return n * rank // ws, n * (rank + 1) // ws


def job_glups(ws: int, n_nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of ws independent replicas of n_nodes nodes that
    each advanced `steps` steps in `seconds` (the slowest rank's time)."""
    return ws * n_nodes * steps / seconds / 1e9


def cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu on Arm)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def oracle_sample(case, seconds=10.0, max_steps=400, min_steps=2, threads=None, fields=False):
    """Oracle steps on the full grid of the workload (from the float32 phi0
    the GPU receives) until `seconds` of CPU work on `threads` OpenMP threads
    (all host cores by default): returns (GLUPS, steps, threads), and with
    fields=True also the oracle's fields after its 1 + steps steps."""
    import oracle
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    s = oracle.Sim(case.nx, case.ny, case.wall_y, oracle.Params(**case.params),
                   case.phi0.astype(np.float32).astype(np.float64),
                   wall_x=case.meta.get("wall_x", False))
    s.step(1)  # first step separately (first-step flag), untimed
    t0 = time.perf_counter()
    n = 0
    while n < min_steps or (time.perf_counter() - t0 < seconds and n < max_steps):
        s.step(1)
        n += 1
    dt = time.perf_counter() - t0
    out = (case.nx * case.ny * n / dt / 1e9, n, threads)
    return out + (s.macro(),) if fields else out


def pressure_jump(fields, case):
    """Mean p_h within R/2 of the bubble or drop centre minus its mean beyond
    R + 3W (the Laplace measurement of Sec. 5.1; distances wrap only across
    periodic sides)."""
    m = case.meta
    xc, yc, R, W = m["xc"], m["yc"], m["R"], case.params["W"]
    ny, nx = fields["phi"].shape
    dx = np.abs(np.arange(nx)[None, :] - xc)
    if not m.get("wall_x", False):
        dx = np.minimum(dx, nx - dx)
    dy = np.abs(np.arange(ny)[:, None] - yc)
    if not case.wall_y:
        dy = np.minimum(dy, ny - dy)
    r = np.hypot(dx, dy)
    ph = np.asarray(fields["p_h"], dtype=np.float64)
    return float(ph[r <= R / 2].mean() - ph[r >= R + 3 * W].mean())


def storage_parity(case, dev, steps, ref):
    """Errors of the GPU step after `steps` steps from the workload's phi0,
    with float32, FP16 and BF16 population storage, against the FP64 oracle's
    fields `ref` after the same steps: max |phi| and |u| errors and the error
    of the pressure jump relative to the Laplace jump sigma / R."""
    from paper_2012_14729_gb300 import pflbm
    out = {"steps": steps}
    lap = case.params["sigma"] / case.meta["R"]
    dp_ref = pressure_jump(ref, case)
    for st in ("fp32", "fp16", "bf16"):
        d = pflbm.Domain(case.nx, case.ny, wall_y=case.wall_y,
                         wall_x=case.meta.get("wall_x", False), storage=st, device=dev)
        d.set_params(**case.params).init_phi(case.phi0.astype(np.float32))
        d.step(steps)
        g = d.fields()
        out[st] = {"phi": float(np.abs(g["phi"] - ref["phi"]).max()),
                   "u": float(max(np.abs(g["ux"] - ref["ux"]).max(), np.abs(g["uy"] - ref["uy"]).max())),
                   "dp_over_laplace": abs(pressure_jump(g, case) - dp_ref) / lap}
    return out


def run_reference(args, case):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    s = oracle.Sim(case.nx, case.ny, case.wall_y, oracle.Params(**case.params), case.phi0,
                   wall_x=case.meta.get("wall_x", False))
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    value = case.nx * case.ny * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": "GLUPS (coupled f+h step)", "value": value,
        "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nx": case.nx, "ny": case.ny,
                   "form": args.form, "walls": walls_name(case)},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{args.warmup}+{args.steps} full-grid oracle steps"},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, case):
    import torch
    from paper_2012_14729_gb300 import build, pflbm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    pflbm.load()

    n_nodes = case.nx * case.ny
    wall_x = case.meta.get("wall_x", False)
    dom = pflbm.Domain(case.nx, case.ny, wall_y=case.wall_y, wall_x=wall_x, storage=args.storage,
                       device=dev)
    dom.set_params(**case.params)
    dom.init_phi(case.phi0.astype(np.float32))
    if args.stage == "auto":
        stage = dom.autotune(10)   # untimed; leaves the state unchanged
    else:
        stage = args.stage
        dom.stage_mode(stage)
    stream = dom.stream
    flush = ColdL2(dev)

    clk = ClockSampler(torch.cuda.current_device())
    clk.__enter__()
    # warm-up: at least `warmup` steps and at least ~1 s of load, so that the
    # clock sampler (50 ms period) sees the GPU under load around the timed
    # region, which itself can be shorter than one sample
    t_w = time.perf_counter()
    k = 0
    with torch.cuda.stream(stream):
        while time.perf_counter() - t_w < args.load_seconds:
            flush()
            dom.step(1)
            k += 1
            if k % 64 == 0:
                stream.synchronize()
    stream.synchronize()
    # restart the run from phi0 so that the timed steps follow the workload's
    # initial condition (the warm-up load above can run for thousands of steps)
    dom.init_phi(case.phi0.astype(np.float32))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush()
            dom.step(1)
    stream.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush()                # cold, clean L2 for every timed step
            e0.record(stream)
            dom.step(1)            # one fused kernel launch
            e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    time.sleep(0.15)  # one more clock sample after the timed region
    clk.__exit__(None, None, None)
    per_step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    t_ms = max_over_ranks(sum(per_step_ms), ws, dev)
    ms_per_step = t_ms / args.steps
    value = job_glups(ws, n_nodes, args.steps, t_ms * 1e-3)

    # stability check of the state that was timed (not timed)
    diag = dom.diagnostics()

    # end to end through the public API with host buffers: phi0 from pinned
    # host memory, K steps, all fields back to pinned host memory
    phi_host = torch.from_numpy(case.phi0.astype(np.float32)).pin_memory()
    out_host = torch.empty((len(pflbm.FIELDS), case.ny, case.nx), dtype=torch.float32,
                           pin_memory=True)
    e2e_dom = pflbm.Domain(case.nx, case.ny, wall_y=case.wall_y, wall_x=wall_x,
                           storage=args.storage, device=dev, stream=stream)
    e2e_dom.set_params(**case.params)
    e2e_dom.stage_mode(stage)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pflbm.pflbm_init_phi(e2e_dom.h, phi_host)
    pflbm.pflbm_step(e2e_dom.h, args.steps)
    pflbm.pflbm_read_fields(e2e_dom.h, out_host)
    stream.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    e2e = {"value": job_glups(ws, n_nodes, args.steps, e2e_s), "unit": "GLUPS",
           "steps": args.steps,  # the copies below are amortised over these steps
           "h2d_bytes_per_step": n_nodes * 4 / args.steps,
           "d2h_bytes_per_step": len(pflbm.FIELDS) * n_nodes * 4 / args.steps}

    peak, peak_kind = measured_peaks()
    bpl = BYTES_PER_LUP[args.storage]
    launch_ms = statistics.mean(per_step_ms)
    achieved = bpl * n_nodes / (launch_ms * 1e-3) / 1e9
    tr = traffic_record(args.workload, args.storage, stage)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None if tr is None else tr * n_nodes,
                "algorithmic_bytes": bpl * n_nodes,
                "kernel": KERNEL_OF_STAGE[stage]}

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        v, n, thr, ref = oracle_sample(case, seconds=0.75 * args.cpu_seconds, fields=True)
        v1, n1, _ = oracle_sample(case, seconds=0.25 * args.cpu_seconds, min_steps=1, threads=1)
        cpu = {"value": v, "unit": "GLUPS", "cores": thr, "kind": "oracle",
               "sample": f"{n} full-grid FP64 oracle steps of {args.workload}",
               "value_1thread": v1, "sample_1thread": f"{n1} steps on one thread",
               "cpu_model": cpu_model()}
        if "R" in case.meta and "xc" in case.meta:
            # the GPU path against the oracle's final state of that sample
            cpu["parity_vs_gpu"] = storage_parity(case, dev, 1 + n, ref)

    # the same physics on a grid whose state exceeds L2 (8.4 M nodes, 1.34 GB
    # per step), timed over consecutive steps without flushing
    l2x = (measure_l2_exceeding(args, dev, wall_x=wall_x)
           if ws == 1 and not args.no_l2x and case.nx * case.ny < (1 << 23) else None)
    # the patterns against this plain FP32 line (default workload, one GPU)
    patterns = (measure_patterns(args, case, dev, value, l2x)
                if ws == 1 and not args.no_patterns and args.storage == "fp32" and not wall_x
                else None)

    line = {
        "metric": "GLUPS (coupled f+h step)", "value": value, "unit": "GLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "nx": case.nx, "ny": case.ny,
                   "walls": walls_name(case), "form": args.form,
                   "storage": args.storage, "stage": stage,
                   "l2": "flushed before every timed step (256 MB written, then 256 MB "
                         "read: no line of the state and no dirty line left in L2)",
                   "parallelism": f"replicas{ws}", "state_status": diag["status"]},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if l2x is not None:
        line["l2_exceeding"] = l2x
    if patterns is not None:
        line["patterns"] = patterns
    if wall_x:
        line["bubble_diagnostics"] = time_bubble_diagnostics(dom, case)
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_l2_exceeding(args, dev, steps=30, wall_x=False):
    """GLUPS and roofline fraction of the step on the 2048 x 4096 rising
    bubble (same physics as the default workload, state larger than L2);
    with free-slip side walls when the timed workload has them."""
    import torch
    from paper_2012_14729_gb300 import pflbm
    name = "rising_bubble_2048x4096" if wall_x else "bubble_4096x2048"
    case = make_case(name, args.form)
    n = case.nx * case.ny
    dom = pflbm.Domain(case.nx, case.ny, wall_y=case.wall_y, wall_x=wall_x, storage=args.storage,
                       device=dev)
    dom.set_params(**case.params)
    dom.init_phi(case.phi0.astype(np.float32))
    stage = dom.autotune(5)
    dom.step(max(3, args.warmup))
    stream = dom.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    dom.step(steps)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peak, _ = measured_peaks()
    bpl = BYTES_PER_LUP[args.storage]
    return {"workload": name, "nx": case.nx, "ny": case.ny, "value": n / (ms * 1e-3) / 1e9,
            "unit": "GLUPS", "ms_per_step": ms, "steps": steps, "stage": stage,
            "roofline_frac": bpl * n / (ms * 1e-3) / 1e9 / peak,
            "l2": f"state {bpl * n / 1e9:.2f} GB per step, larger than L2: consecutive steps",
            "state_status": dom.diagnostics()["status"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="bubble_512x1024")
    ap.add_argument("--form", default="STF1")
    ap.add_argument("--storage", default="fp32", choices=("fp32", "fp16", "bf16"))
    ap.add_argument("--stage", default="auto", choices=("auto", "boxes", "gather", "march", "gather8"))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--load-seconds", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the 16-bit, batch and adjoint measurements of the default line")
    ap.add_argument("--ckpt-every", type=int, default=200,
                    help="adjoint workloads: checkpoint interval of the gradient run")
    ap.add_argument("--batch-config", default=None,
                    help="batch workloads: MODE:CTAS_PER_SM:ROWS instead of the autotuner's "
                         "choice, e.g. gather:4:16")
    ap.add_argument("--no-l2x", action="store_true",
                    help="skip the extra 2048 x 4096 (larger than L2) measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload.startswith("batch") and args.workload[5:].isdigit():
        if args.impl == "reference":
            raise SystemExit("the batched workload has no reference arm of its own")
        run_batch(args)
        return
    if args.workload.startswith("adjoint_shear"):
        if args.impl == "reference":
            raise SystemExit("the adjoint workload has no reference arm of its own")
        run_adjoint(args)
        return
    case = make_case(args.workload, args.form)
    if args.impl == "reference":
        run_reference(args, case)
    else:
        run_ours(args, case)


def run_adjoint(args):
    print(json.dumps(measure_adjoint(args)), flush=True)


def measure_adjoint(args, consistency=True):
    """Adjoint pattern on the drop-in-shear workload (512 x 256, walls at
    -/+0.01, drop R = 40, Re = 1, Ca = 0.2, W = 4, M = 0.05, form --form):
    `--steps` forward steps, then the full gradient run (forward with a
    checkpoint every `--ckpt-every` steps, 200 by default, recomputation of
    each segment, reverse sweep; --ckpt-every >= --steps keeps the whole tape
    of one segment taped in the forward run, with no recomputation).  Reported: GLUPS of the forward, time of the gradient run over the
    time of the forward, and the relative change of the gradients between
    checkpoint intervals 200 and 50 (a consistency figure)."""
    import torch
    from paper_2012_14729_gb300 import build, pflbm

    build.build()
    pflbm.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    # adjoint_shear: the 512 x 256 configuration; adjoint_shear_x<s>: the same
    # drop-in-shear physics on an s-times larger grid in each direction (drop
    # radius and wall speed scaled to keep Re and Ca)
    s = int(args.workload.rsplit("_x", 1)[1]) if "_x" in args.workload else 1
    c = wl.shear_drop(args.form, nx=512 * s, ny=256 * s, R=40.0 * s, U=0.01)
    T, every = args.steps, min(args.ckpt_every, args.steps)
    stream = torch.cuda.Stream(dev)
    d = pflbm.Domain(c.nx, c.ny, wall_y=True, stream=stream, device=dev).set_params(**c.params)
    phi0 = torch.from_numpy(c.phi0.astype(np.float32)).to(dev)
    target = torch.from_numpy(wl.ellipse(c.nx, c.ny, c.meta["R"], 4.0, 0.2).astype(np.float32)).to(dev)
    d.stage_mode("gather")
    d.graphs(True)  # the forward, alone and inside the gradient run, replays graphs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # forward alone
    d.init_phi(phi0)
    d.step(args.warmup)
    d.init_phi(phi0)
    stream.synchronize()
    e0.record(stream)
    d.step(T)
    e1.record(stream)
    stream.synchronize()
    t_fwd = e0.elapsed_time(e1)
    phiT = d.fields(device=True)["phi"]
    g = (2 * (phiT - target)).contiguous()
    scratch = torch.empty(pflbm.pflbm_adjoint_scratch_bytes(d.h, T, every), dtype=torch.uint8,
                          device=dev)
    dphi0 = torch.empty_like(phi0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ds, dm = pflbm.pflbm_adjoint_run(d.h, phi0, T, every, g, dphi0, scratch)
    t_adj = (time.perf_counter() - t0) * 1e3
    del scratch
    every2 = max(1, every // 4)
    rel = None
    if consistency:
        scratch2 = torch.empty(pflbm.pflbm_adjoint_scratch_bytes(d.h, T, every2),
                               dtype=torch.uint8, device=dev)
        dphi0b = torch.empty_like(phi0)
        ds2, dm2 = pflbm.pflbm_adjoint_run(d.h, phi0, T, every2, g, dphi0b, scratch2)
        rel = max(abs(ds2 / ds - 1), abs(dm2 / dm - 1))
    nodes = c.nx * c.ny
    line = {
        "metric": "GLUPS (coupled f+h step)", "value": nodes * T / (t_fwd * 1e-3) / 1e9,
        "unit": "GLUPS", "n_gpus": 1, "steps": T, "warmup": args.warmup,
        "ms_per_step": t_fwd / T, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "nx": c.nx, "ny": c.ny, "form": args.form,
                   "ckpt_every": every},
        "adjoint": {"gradient_run_ms": t_adj, "forward_ms": t_fwd,
                    "cost_over_forward": t_adj / t_fwd,
                    "dJ_dsigma": ds, "dJ_dM": dm},
    }
    if rel is not None:
        line["adjoint"]["rel_change_ckpt_every_%d" % every2] = rel
    return line


def run_batch(args):
    """Batched workload; under torchrun each rank advances its own share of
    the batch's instances (they are independent problems: no data-path
    collective), the job's time is the slowest rank's."""
    ws, rank, local = dist_env()
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    line = measure_batch(args, ws=ws, rank=rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def measure_batch(args, clocks=True, ws=1, rank=0):
    """Batched pattern, workload batchN (batch256 is the configuration): N
    drop instances (L from {64, 128, 256, 512}, R in [0.15, 0.35] L, sigma
    log-uniform in [1e-4, 1e-2], force family cycling STF, CPF, PF, CSF),
    FP32, one persistent launch per step replayed from a CUDA graph,
    autotuned; for N = 256 about 24 M nodes (3.6 GiB of state per step,
    larger than L2).  Also timed: the same instances stepped one launch
    each."""
    import torch
    from paper_2012_14729_gb300 import build, pflbm

    build.build()
    pflbm.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    all_cases = wl.batch_instances(int(args.workload[5:]), seed=0)
    lo, hi = shard(len(all_cases), rank, ws)
    cases = all_cases[lo:hi]
    stream = torch.cuda.Stream(dev)
    doms = []
    for c in cases:
        d = pflbm.Domain(c.nx, c.ny, wall_y=c.wall_y, stream=stream, device=dev)
        d.set_params(**c.params)
        d.init_phi(c.phi0.astype(np.float32))
        doms.append(d)
    nodes = sum(c.nx * c.ny for c in cases)
    b = pflbm.Batch(doms, stream=stream)
    b.step(1)
    if getattr(args, "batch_config", None):
        # a fixed configuration (e.g. to profile what the autotuner picks in a plain run)
        m, c_, r_ = args.batch_config.split(":")
        b.config(m, int(c_), int(r_))
        mode, cps, rows = m, int(c_), int(r_)
    else:
        mode, cps, rows = b.autotune(3)
    b.graphs(True)
    b.step(args.warmup)
    b.synchronize()

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(k)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    if clocks:
        clk = ClockSampler(torch.cuda.current_device())
        clk.__enter__()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_ms = timed(b.step, args.steps)
    torch.cuda.synchronize()
    t_ms = max_over_ranks(t_ms, ws, dev)
    if clocks:
        time.sleep(0.15)
        clk.__exit__(None, None, None)
    diag = doms[0].diagnostics()

    # the same instances, one launch per instance and step (autotuned each)
    for d in doms:
        d.autotune(2)

    def solo(k):
        for _ in range(k):
            for d in doms:
                d.step(1)
    solo(2)
    stream.synchronize()
    k_solo = max(3, args.steps // 10)
    t_solo = max_over_ranks(timed(solo, k_solo), ws, dev)

    nodes = int(sum_over_ranks(nodes, ws, dev))  # the whole job's nodes
    ms_per_step = t_ms / args.steps
    value = nodes * args.steps / (t_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    achieved = 160 * nodes / (ms_per_step * 1e-3) / 1e9
    line = {
        "metric": "GLUPS (coupled f+h step)", "value": value, "unit": "GLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        # the batch's instances are split over the ranks: fixed total work
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(all_cases), "nodes": nodes,
                   "parallelism": f"instances sharded over {ws} rank(s)",
                   "stage": mode, "ctas_per_sm": cps, "tile": f"32x{rows}", "graphs": True,
                   "l2": f"state {160 * nodes / 2**30:.2f} GiB per step (L2 is 129 MB)",
                   "state_status": diag["status"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes": 160 * nodes, "kernel": "k_step_batch"},
        "per_instance_launches": {"value": nodes * k_solo / (t_solo * 1e-3) / 1e9,
                                  "unit": "GLUPS", "launches_per_step": len(doms)},
        "gpu_launches": args.steps,
    }
    if clocks:
        line["clocks"] = clk.summary()
    return line


def measure_storage(args, case, dev, storage, steps):
    """GLUPS of the timed workload with another population storage, timed
    like the main line (L2 flushed before every step, CUDA events per step)."""
    import torch
    from paper_2012_14729_gb300 import pflbm
    dom = pflbm.Domain(case.nx, case.ny, wall_y=case.wall_y,
                       wall_x=case.meta.get("wall_x", False), storage=storage, device=dev)
    dom.set_params(**case.params)
    dom.init_phi(case.phi0.astype(np.float32))
    stage = dom.autotune(10)
    flush = ColdL2(dev)
    stream = dom.stream
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            flush()
            dom.step(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    stream.synchronize()
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush()
            e0.record(stream)
            dom.step(1)
            e1.record(stream)
    stream.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps
    n = case.nx * case.ny
    peak, _ = measured_peaks()
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GLUPS", "ms_per_step": ms,
            "stage": stage, "roofline_frac": BYTES_PER_LUP[storage] * n / (ms * 1e-3) / 1e9 / peak,
            "state_status": dom.diagnostics()["status"]}


def measure_patterns(args, case, dev, plain_value, l2x=None):
    """The three patterns against the plain FP32 step, measured in this run:
    16-bit storage on the timed workload (and, when the line has its
    L2-exceeding point, on that 2048 x 4096 grid against the FP32 point), the
    256-instance batch against the same instances launched one by one, and
    the adjoint of the 512 x 256 drop in shear (4000 steps, checkpoint every
    200) against its forward."""
    import argparse as _ap
    out = {"plain_fp32": {"value": plain_value, "unit": "GLUPS"}}

    def guarded(name, fn):
        # a failing side measurement is reported in its entry, never fails the line
        try:
            out[name] = fn()
        except Exception as exc:  # noqa: BLE001
            out[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    def storage(st):
        r = measure_storage(args, case, dev, st, args.steps)
        r["vs_plain"] = r["value"] / plain_value
        if l2x is not None:
            big = measure_l2_exceeding(_ap.Namespace(**{**vars(args), "storage": st}), dev)
            r["l2_exceeding"] = {"workload": big["workload"], "value": big["value"],
                                 "unit": "GLUPS", "stage": big["stage"],
                                 "roofline_frac": big["roofline_frac"],
                                 "vs_plain": big["value"] / l2x["value"],
                                 "state_status": big["state_status"]}
        return r

    def batch():
        b = measure_batch(_ap.Namespace(workload="batch256", steps=20, warmup=5), clocks=False)
        return {"value": b["value"], "unit": "GLUPS", "config": b["config"],
                "per_instance_launches": b["per_instance_launches"]["value"],
                "vs_per_instance_launches": b["value"] / b["per_instance_launches"]["value"]}

    def adjoint():
        a = measure_adjoint(_ap.Namespace(workload="adjoint_shear", steps=4000, warmup=10,
                                          form="STF1", ckpt_every=200), consistency=False)
        return {"cost_over_forward": a["adjoint"]["cost_over_forward"],
                "forward_glups": a["value"], "steps": 4000, "ckpt_every": 200, "form": "STF1"}

    guarded("fp16", lambda: storage("fp16"))
    guarded("bf16", lambda: storage("bf16"))
    guarded("batch256", batch)
    guarded("adjoint_shear", adjoint)
    return out


if __name__ == "__main__":
    main()
