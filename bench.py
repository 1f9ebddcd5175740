#!/usr/bin/env python
"""Throughput of the KFVM-WENO hot path on one GB300 (or N replicas under torchrun).

Metric: cell-updates/s per RK stage (cells x RK stages / time) of SSP-RK3 steps.
The default workload is the 3D Euler problem on 512^3 cells at radius 3: the
learned gate + mixed-precision path (FP32 Riemann states, the contraction on
the tcgen05 tensor cores, float64 accumulation) against the plain FP64 GPU
path, 512 seeded Voronoi regions each carrying the smooth sine-advection state
or a random constant (seed 5), outflow boundaries, CFL 0.4.  The plain FP64
comparison runs on the first 16 z-planes of the same state (that path takes
seconds per stage at full size).  ``matched_l1`` reports the accuracy side of
the metric on the smooth-translation check of the same dimension and radius:
the gated path's L1 density error against the exact solution over the plain
FP64 WENO-AO path's.  ``--workload`` selects the other synthetic workloads
(2D 1024^2 Voronoi; 3D 256^3 half smooth / half Voronoi at radius 2; 2D
2048^2 mixed smooth/constant regions; 3D 64^3 radius 3).

One printed JSON line (rank 0).  A "step" is one SSP-RK3 step: the CFL
reduction and three RK stages (Riemann states, face fluxes, update), all in the
library's kernels.  ``value`` is the headline path with inputs resident in
HBM; ``fp64_plain`` is the plain FP64 GPU path on the same workload; ``e2e``
is the headline path through the C ABI with the state copied host->device
before and device->host after every step; ``cpu_baseline`` is the oracle on
the host cores (all of them, OpenMP build, and one thread).  ``--impl reference``
times the oracle instead (the reference arm of this repository).
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
sys.path.insert(0, ROOT)

CFL = 0.4
METRIC = "cell-updates/s per RK stage"
GATE_THRESHOLD = 0.8
TRACED_STEPS = 5  # steps of the second, traced pass that gives each kernel's device time


class Workload:
    def __init__(self, name, dims, R, n, bc, desc, make, gate=None, fp64_planes=None, cpu_crop=None):
        self.name, self.dims, self.R, self.n, self.bc, self.desc = name, dims, R, n, bc, desc
        self.make = make                  # device -> float64 state
        self.gate = gate                  # trained gate parameters (.npy) or None
        self.fp64_planes = fp64_planes    # 3D: time the plain FP64 path on this many z-planes
        self.cpu_crop = cpu_crop          # edge of the cube / square the oracle times

    @property
    def ncell(self):
        c = 1
        for v in self.n:
            c *= v
        return c

    def gate_path(self):
        return os.path.join(ROOT, "paper_2401_16543_gb300", self.gate) if self.gate else None

    def has_gate(self):
        return self.gate is not None and os.path.exists(self.gate_path())


def _workloads():
    import workloads as wl
    return {
        "voronoi2d-1024": Workload(
            "voronoi2d-1024", 2, 2, [1024, 1024], "outflow",
            "2D Euler 1024x1024, radius-2 KFVM-WENO-AO (linearized primitive variables), HLLC + Batten, positivity "
            "limiter, outflow, 64 seeded Voronoi regions (rho,p~U[0.1,1], u,v~U[-1,1], seed 2), SSP-RK3 at CFL 0.4",
            lambda dev, crop=None: wl.voronoi_2d(1024, k=64, seed=2, device=dev, crop=crop), gate="gate_params_2d.npy",
            cpu_crop=128),
        "halfsine3d-256": Workload(
            "halfsine3d-256", 3, 2, [256, 256, 256], "periodic",
            "3D Euler 256^3 periodic, radius 2: x<1/2 smooth sine advection, x>=1/2 128 seeded Voronoi regions "
            "(seed 3), FP32 mixed path vs plain FP64, SSP-RK3 at CFL 0.4",
            lambda dev, crop=None: wl.half_sine_voronoi_3d(256, k=128, seed=3, device=dev, crop=crop), gate=None,
            cpu_crop=24),
        "mixed2d-2048": Workload(
            "mixed2d-2048", 2, 2, [2048, 2048], "outflow",
            "2D Euler 2048x2048, radius 2, learned gate: 256 seeded Voronoi regions (seed 4), each smooth sine or a "
            "constant (coin 1/2), outflow, SSP-RK3 at CFL 0.4",
            lambda dev, crop=None: wl.mixed_voronoi(2, 2048, 256, seed=4, device=dev, crop=crop),
            gate="gate_params_2d.npy", cpu_crop=128),
        "mixed3d-64-r3": Workload(
            "mixed3d-64-r3", 3, 3, [64, 64, 64], "outflow",
            "3D Euler 64^3, radius 3, learned gate + mixed precision: 8 seeded Voronoi regions (seed 5), each "
            "smooth sine or a constant, outflow, SSP-RK3 at CFL 0.4 (the 512^3 workload's scheme on a grid that "
            "profilers can capture)",
            lambda dev, crop=None: wl.mixed_voronoi(3, 64, 8, seed=5, R=3, device=dev, crop=crop),
            gate="gate_params_3d.npy", cpu_crop=16),
        "mixed3d-512-r3": Workload(
            "mixed3d-512-r3", 3, 3, [512, 512, 512], "outflow",
            "3D Euler 512^3, radius 3, learned gate + mixed precision: 512 seeded Voronoi regions (seed 5), each smooth "
            "sine or a constant, outflow, SSP-RK3 at CFL 0.4; plain FP64 timed on 16 z-planes of the same state",
            lambda dev, crop=None: wl.mixed_voronoi(3, 512, 512, seed=5, R=3, device=dev, crop=crop),
            gate="gate_params_3d.npy", fp64_planes=16, cpu_crop=24),
    }


DEFAULT_WORKLOAD = "mixed3d-512-r3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", choices=["auto", "fp64", "fp64char", "fp32", "fp32char", "gated", "kxrcf"],
                    default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline path only (no other paths, e2e or CPU baseline): for profiler runs")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["voronoi2d-1024", "halfsine3d-256", "mixed2d-2048", "mixed3d-64-r3", "mixed3d-512-r3"])
    ap.add_argument("--crop", type=int, default=None,
                    help="with --headline-only: run on the corner crop of this edge of the workload's state (the "
                         "same regions at the same scale, a grid small enough for a profiler capture)")
    args = ap.parse_args()
    if args.crop is not None and not args.headline_only:
        ap.error("--crop needs --headline-only")
    return args


def cropped(W, c):
    """The corner crop c^d of workload W as a workload of its own."""
    return Workload(f"{W.name}-crop{c}", W.dims, W.R, [c] * W.dims, W.bc, f"{W.desc}; corner crop {c}^{W.dims}",
                    lambda dev, crop=None: W.make(dev, crop=c), gate=W.gate, cpu_crop=W.cpu_crop)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np

    import oracle
    W = _workloads()[args.workload]
    crop = W.cpu_crop
    U = np.ascontiguousarray(W.make("cpu", crop=crop).numpy())
    cores = host_cores()
    o = oracle.Oracle([crop] * W.dims, dim=W.dims, R=W.R, bc=W.bc, threaded=True)
    for _ in range(args.warmup):
        o.step(U, CFL)
    t0 = time.perf_counter()
    Ur = U
    for _ in range(args.steps):
        Ur, _ = o.step(Ur, CFL)
    el = time.perf_counter() - t0
    value = crop ** W.dims * 3 * args.steps / el
    shape = "x".join([str(crop)] * W.dims)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.desc, "grid": W.n, "radius": W.R,
                   "sample": f"{shape} corner crop of the workload per step"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"SSP-RK3 steps of a {shape} corner crop, C oracle (OpenMP build) on {cores} "
                                   "host cores"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(W, t_budget=10.0):
    """The oracle on the host cores: one SSP-RK3 step of a corner crop of the workload, on every core
    (OpenMP build, the value) and on one thread; each repeated until about t_budget seconds."""
    import numpy as np

    import oracle
    c = W.cpu_crop
    U = np.ascontiguousarray(W.make("cpu", crop=c).numpy())
    shape = [c] * W.dims
    cells = c ** W.dims
    out = {}
    for threaded in (True, False):
        o = oracle.Oracle(list(shape), dim=W.dims, R=W.R, bc=W.bc, threaded=threaded)
        k, t0 = 0, time.perf_counter()
        while True:
            o.step(U, CFL)
            k += 1
            el = time.perf_counter() - t0
            if el >= t_budget or k >= 50:
                break
        out[threaded] = (cells * 3 * k / el, k)
    cores = host_cores()
    return {"value": out[True][0], "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "single_thread_value": out[False][0],
            "sample": f"{out[True][1]} (all cores) / {out[False][1]} (one thread) SSP-RK3 steps of a "
                      f"{'x'.join(map(str, shape))} corner crop of the workload; C oracle, OpenMP build over "
                      f"{cores} host cores (value) and the single-threaded build (single_thread_value)"}


def matched_l1(pkg, W):
    """The accuracy side of the metric: L1 density error against the exact solution of the smooth
    translation (sine advection, periodic) of the workload's dimension and radius, for the headline
    gated mixed-precision path and the plain FP64 WENO-AO path; ratio = E_gated / E_fp64."""
    import numpy as np

    import workloads as wl
    if W.dims == 2:
        n, t_end = 64, 0.1
        U0 = wl.sine_2d(n, R=W.R)
        ex = wl.sine_2d_exact_density(n, t_end)
    else:
        n, t_end = 32, 0.05
        U0 = wl.sine_3d(n, R=W.R)
        ex = wl.sine_3d_exact_density(n, t_end)
    errs = {}
    for path in ("fp64", "gated", "fp32"):
        g = make_solver(W, path, [n] * W.dims, bc="periodic")
        if path == "gated":
            frac = float(g.gate_mask(U0.cuda()).float().mean().item())
        U = U0.cuda()
        g.run(U, CFL, t_end)
        errs[path] = float(np.abs(U[0].cpu().numpy() - ex).mean())
        del g
    ratio = errs["gated"] / errs["fp64"]
    return {"ratio": ratio, "E_gated": errs["gated"], "E_fp64_weno": errs["fp64"], "bar": 1 + 1e-6,
            "met": bool(ratio <= 1 + 1e-6), "gate_linear_fraction_t0": round(frac, 4),
            # the same run in float32 with WENO-AO on every cell (no gate): the precision-only spread
            "ratio_fp32_weno_everywhere": errs["fp32"] / errs["fp64"],
            "case": f"{W.dims}D sine translation {n}^{W.dims}, periodic, radius {W.R}, to t = {t_end}, CFL {CFL}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the GPU is loaded."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algo_flops_per_cell(dims, R, mode):
    """Algorithmic flops of the Riemann-state kernel per cell (FMA = 2): every contraction
    r_q(s).g_q and d_q(alpha).g_q (Eqs. 18, 22), the beta sums and the WENO-AO blend
    (Eq. 19), for every reconstruction variable; linear mode: r_0(s).g_0 only."""
    from paper_2401_16543_gb300 import stencil_info
    sizes, _, F, M = stencil_info(dims, R)
    nv, nq = dims + 2, len(sizes)
    if mode == "linear":
        return 2 * nv * sizes[0] * F
    return 2 * nv * (sum(n * (F + M) for n in sizes) + nq * M + nq * F)


def gate_flops_per_cell(dims):
    """Algorithmic flops of the learned gate per cell (FMA = 2): in -> 32 -> 32 -> 1 with in = 26 (2D) or
    68 (3D) inputs; it runs on the tensor pipe (mma.sync BF16, FP32 accumulation), not the FP32 pipe."""
    n_in = 26 if dims == 2 else 68
    return 2 * (n_in * 32 + 32 * 32 + 32)


def flush_l2(buf):
    buf.zero_()


def time_steps(g, U, steps, stream, flush_buf):
    """Per-step CUDA events on the launching stream, each step behind an L2 flush that lies outside its
    events.  The steps are enqueued back to back and the stream is synchronised once at the end, so the
    device never waits inside a timed step for the host to issue its launches (a per-step wait would
    put the host's launch latency of every step's first kernel inside the events)."""
    import torch
    pairs = []
    for k in range(steps):
        flush_l2(flush_buf)
        if k == 0:
            flush_l2(flush_buf)  # a longer lead for the first step, while the host issues its launches
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(U, CFL, sync=False, stream=stream)
        e1.record(stream)
        pairs.append((e0, e1))
    stream.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in pairs)  # ms


def make_solver(W, path, n=None, bc=None):
    import numpy as np

    from paper_2401_16543_gb300 import KFVM
    g = KFVM(list(n or W.n), dims=W.dims, radius=W.R, bc=bc or W.bc)
    if path in ("fp32", "fp32char", "gated", "kxrcf"):
        g.set_option("precision", 32)
    if path == "kxrcf":  # the paper's troubled-cell indicator (Sec. 3.5) instead of the learned gate
        g.set_option("recon", 4)
    if path in ("fp64char", "fp32char"):  # WENO-AO in characteristic variables (Sec. 3.4.1)
        g.set_option("variables", 1)
    if path == "gated":
        g.gate_set_params(np.load(W.gate_path()))
        g.set_option("gate_threshold", GATE_THRESHOLD)
        g.set_option("recon", 2)
    return g


def job_time_ms(ms, dist, device):
    """The job's time: the maximum over ranks (every rank runs its own replica of the workload)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, ncell, steps, ms):
    """Whole-job cell-updates/s per RK stage: every rank's cells x 3 stages x steps over the job time."""
    return world * ncell * 3 * steps / (ms * 1e-3)


def e2e_time(g, U0, steps, stream, flush_buf, warm=2):
    """ms for `steps` steps, each: upload the (pinned host) input state, flush L2, step the state,
    download the result (the flush is inside the timed region: a state smaller than L2 would otherwise
    arrive cache-warm from the upload)."""
    import torch
    Uh = U0.cpu().pin_memory()
    Uo = [torch.empty_like(Uh).pin_memory() for _ in range(2)]
    Ub = [torch.empty_like(U0) for _ in range(2)]
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for k in range(warm + steps):
        if k == warm:
            torch.cuda.synchronize()
            e0.record(s_up)
        b = k % 2
        if k >= 2:
            s_up.wait_event(ev_out[b])  # the download of step k-2 has left this buffer
        with torch.cuda.stream(s_up):
            Ub[b].copy_(Uh, non_blocking=True)
            ev_in[b].record(s_up)
        stream.wait_event(ev_in[b])
        with torch.cuda.stream(stream):
            flush_l2(flush_buf)
        g.step(Ub[b], CFL, sync=False, stream=stream)
        ev_done[b].record(stream)
        s_down.wait_event(ev_done[b])
        with torch.cuda.stream(s_down):
            Uo[b].copy_(Ub[b], non_blocking=True)
            ev_out[b].record(s_down)
    e1.record(s_down)
    e1.synchronize()
    torch.cuda.synchronize()
    g.sync_status(stream)
    return e0.elapsed_time(e1)


def measure_path(W, path, U0, steps, warmup, stream, flush_buf, n=None, min_warm_s=0.0, barrier=None):
    """W warm-up steps (and, with min_warm_s, at least that many seconds of steps, so that the clock
    sampler is running and the GPU is at its loaded clocks when the timed steps start), then the
    timed steps from the initial state, bracketed by `barrier` (all ranks) and a device sync."""
    import torch
    g = make_solver(W, path, n)
    U = U0.clone()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        k = 0
        while k < warmup or time.perf_counter() - t0 < min_warm_s:
            g.step(U, CFL, sync=False, stream=stream)
            k += 1
            if k % 8 == 0:
                stream.synchronize()
                if k >= warmup and time.perf_counter() - t0 >= min_warm_s:
                    break
                if k % 64 == 0:
                    U.copy_(U0)  # keep the warm-up on the workload's own states
        g.sync_status(stream)
        U.copy_(U0)
        torch.cuda.synchronize()
        launches0 = g.launches
        if barrier is not None:
            barrier()
        torch.cuda.synchronize()
        ms = time_steps(g, U, steps, stream, flush_buf)
        torch.cuda.synchronize()
        if barrier is not None:
            barrier()
        launches = g.launches - launches0
        g.sync_status(stream)
        U_final = U.clone()
        # the first (at most TRACED_STEPS) of the same steps again from the same state with the library's
        # per-launch event tracing on (kernel durations and shares; the tracing events would otherwise sit
        # inside the timed steps)
        U.copy_(U0)
        g.set_option("profile", 1)
        g.profile_reset()
        time_steps(g, U, min(steps, TRACED_STEPS), stream, flush_buf)
        torch.cuda.synchronize()
        prof = g.profile()
        g.set_option("profile", 0)
        g.sync_status(stream)
    return g, ms, prof, launches, U_final


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2401_16543_gb300 as pkg
    pkg.load()
    W = _workloads()[args.workload]
    if args.crop is not None:
        W = cropped(W, args.crop)
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    U0 = W.make(dev).contiguous()
    torch.cuda.synchronize()
    print(f"[bench] {W.name}: state generated in {time.perf_counter() - t_gen:.1f} s", file=sys.stderr, flush=True)
    ncell = W.ncell
    stream = torch.cuda.Stream(device=dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    path = args.path
    if path == "auto":
        path = "gated" if W.has_gate() else "fp32"
    sampler = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    sampler.start()
    # ---- headline path, resident inputs ----
    barrier = dist.barrier if dist is not None else None
    g, ms, prof, launches, g_final_state = measure_path(W, path, U0, args.steps, args.warmup, stream, flush_buf,
                                                        min_warm_s=1.0, barrier=barrier)
    ms = job_time_ms(ms, dist, dev)
    clocks = sampler.stop()
    value = job_value(world, ncell, args.steps, ms)
    print(f"[bench] {path}: {ms / args.steps:.3f} ms per step", file=sys.stderr, flush=True)

    # ---- the other paths on the same workload (plain FP64 is the metric's reference) ----
    others = {}
    for other in ("fp64", "fp64char", "fp32", "fp32char", "gated", "kxrcf"):
        if args.headline_only or other == path or (other == "gated" and not W.has_gate()):
            continue
        if other == "fp32char" and W.dims == 3 and W.R == 3:
            continue  # the radius-3 3D kernels reconstruct in linearized primitive variables only
        if other == "fp64char" and W.fp64_planes:
            continue  # radius 3 in float64 on 512^2 x 16 cells: ~25 s per step with three sets of weights
        k = max(3, args.steps // 4)
        Uo0, n_o, note = U0, None, None
        if other in ("fp64", "fp64char") and W.fp64_planes:
            # the plain FP64 path on the first z-planes of the same state (seconds per stage at full size)
            Uo0 = U0[:, :W.fp64_planes].contiguous()
            n_o = W.n[:2] + [W.fp64_planes]
            note = f"first {W.fp64_planes} z-planes of the state ({W.n[0]}x{W.n[1]}x{W.fp64_planes} cells)"
            k = 1
        go, mso, _, _, _ = measure_path(W, other, Uo0, k, 1 if other.startswith("fp64") else 2, stream, flush_buf, n_o,
                                        barrier=barrier)
        mso = job_time_ms(mso, dist, dev)
        cells = ncell if n_o is None else n_o[0] * n_o[1] * n_o[2]
        others[other] = {"value": job_value(world, cells, k, mso), "ms_per_step": mso / k, "steps": k}
        if other in ("gated", "kxrcf"):  # share of cells the indicator sends to the linear reconstruction
            m = go.gate_mask(Uo0) if other == "gated" else go.kxrcf_mask(Uo0)
            others[other]["smooth_fraction_initial_state"] = round(float(m.float().mean().item()), 4)
        del go
        print(f"[bench] {other}: {mso / k:.3f} ms per step", file=sys.stderr, flush=True)
        if note:
            others[other]["sample"] = note
        del Uo0
    fp64 = others.get("fp64", {"value": value, "ms_per_step": ms / args.steps})

    if args.headline_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                              "config": {"name": W.name, "path": path}, "gpu_launches": launches,
                              "kernel_ms": {k: round(v[1], 4) for k, v in prof.items()}, "headline_only": True}))
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its input state host->device from pinned memory, steps it through the C ABI and
    # copies the result back.  Two device buffers and three streams (upload, compute, download) let the
    # copies of neighbouring steps overlap the compute; the timed region runs from the first upload to
    # the last download (events on the upload and download streams).
    ms_e2e = e2e_time(g, U0, args.steps, stream, flush_buf)
    ms_e2e = job_time_ms(ms_e2e, dist, dev)
    e2e = {"value": job_value(world, ncell, args.steps, ms_e2e), "unit": "cell-updates/s",
           "h2d_bytes_per_step": U0.numel() * 8, "d2h_bytes_per_step": U0.numel() * 8,
           "pipelining": "double-buffered: upload k+1 and download k-1 overlap step k",
           "input": "every step uploads the workload's initial state (value advances the state through its steps; "
                    "the gate's share of linear cells changes as the state evolves)",
           "l2": "flushed before every step, inside the timed region"}

    # ---- roofline of the dominant kernel ----
    kern = "recon64" if path.startswith("fp64") else "recon32"
    n_launch, kms = prof.get(kern, (0, 0.0))
    mode = "weno" if path in ("fp64", "fp64char", "fp32") else "gated"
    flops = algo_flops_per_cell(W.dims, W.R, "weno") * ncell
    smooth_frac = None
    if path in ("gated", "kxrcf"):
        # WENO cells at WENO cost, gated cells at the linear reconstruction's cost, averaged over
        # the masks of the initial and the final state of the timed run
        fr = []
        for Us in (U0, g_final_state):
            m = g.gate_mask(Us) if path == "gated" else g.kxrcf_mask(Us)
            fr.append(float(m.float().mean().item()))
        smooth_frac = sum(fr) / len(fr)
        flops = ncell * (smooth_frac * algo_flops_per_cell(W.dims, W.R, "linear")
                         + (1 - smooth_frac) * algo_flops_per_cell(W.dims, W.R, "weno"))
    peak_flops = pkg.measure_fma_peak(64 if path.startswith("fp64") else 32)
    # algorithmic flops of every traced stage over the kernel's summed device time (3D grids above the
    # Riemann-state buffer run as several launches per stage, one per z-slab)
    traced = min(args.steps, TRACED_STEPS)
    achieved = flops * 3 * traced / (kms * 1e-3) if kms > 0 else 0.0
    traffic = None
    launches_per_stage = n_launch / (3 * traced) if n_launch else 1
    tfile = os.path.join(ROOT, "profiles", f"{kern}_{W.name}_traffic.txt")
    if os.path.exists(tfile) and path != "fp64char":  # the capture is of the linearized-primitive kernel
        for line in open(tfile):
            if line.startswith("traffic_bytes_per_launch"):
                traffic = float(line.split("=")[1])
    tensor = None
    if kern == "recon32" and W.dims == 3 and W.R == 3 and kms > 0:
        # the tcgen05 contraction's issued work: per tile of 128 cells and variable, 23 k-steps of three
        # kind::f16 MMAs of 128 x 96 x 16 (every tile counted as running all 23 k-steps: an upper bound, since
        # all-linear tiles run 8), against the measured dense bf16 peak (fp16 has the same nominal rate)
        import math
        # 8 x 4 x 4 tiles of the whole grid (z-slab launches also reconstruct each slab's two boundary planes,
        # 2.3% more tiles at 512^3, not counted here)
        tiles_total = math.ceil(W.n[0] / 8) * math.ceil(W.n[1] / 4) * math.ceil(W.n[2] / 4)
        mma_flops = tiles_total * 5 * 23 * 3 * (2 * 128 * 96 * 16)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        tpeak = peaks.get("bf16_tflops_sustained") or 1700.0
        issued = mma_flops * 3 * traced / (kms * 1e-3) / 1e12
        tensor = {"issued_tflops": issued, "peak": tpeak, "frac": issued / tpeak,
                  "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (kind::f16 FP16 has the bf16 rate)",
                  "note": "MMA flops issued for the grid's own tiles (three FP16 hi/lo products per k-step, every tile "
                          "counted at 23 k-steps although all-linear tiles run 8; the z-slabs' extra boundary-plane "
                          "tiles not counted) over the kernel's device time"}
    total_prof = sum(v[1] for v in prof.values())
    kname = {"recon64": "recon64_kernel", "recon32": "recon32_kernel"}[kern]
    if kern == "recon32" and W.dims == 3 and W.R == 3:
        kname = "recon33_tc_kernel (tcgen05)"
    roofline = {"bound": "alu", "kernel": kern, "kernel_name": kname, "achieved": achieved / 1e12,
                "peak": peak_flops / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_flops if peak_flops else None, "traffic": traffic,
                "peak_source": f"measured live: FP{64 if path.startswith('fp64') else 32} FMA loop on every SM",
                "algo_flops_per_cell": flops / ncell, "mode": mode, "gated_smooth_fraction": smooth_frac,
                # the learned gate's own work, on the tensor pipe (not in "achieved", which is FP32-pipe work)
                "gate_tensor_flops_per_cell": gate_flops_per_cell(W.dims) if path == "gated" else None,
                "achieved_incl_gate_tflops": ((flops + gate_flops_per_cell(W.dims) * ncell) * 3 * traced
                                              / (kms * 1e-3) / 1e12) if (path == "gated" and kms > 0) else None,
                "launches_per_stage": launches_per_stage,
                "tensor_pipe": tensor,
                "kernel_share": {k: round(v[1] / total_prof, 4) for k, v in prof.items()} if total_prof else {}}

    # ---- the accuracy side of the metric ----
    l1 = matched_l1(pkg, W) if (rank == 0 and path == "gated") else None

    # ---- the oracle on the host cores ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(W)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp64char": "f64", "fp32": "f32", "fp32char": "f32", "gated": "f32+bf16",
                      "kxrcf": "f32"}[path],
            "data": "synthetic",
            "config": {"workload": W.desc, "name": W.name, "grid": W.n, "radius": W.R, "path": path,
                       "gate": ({"params": f"paper_2401_16543_gb300/{W.gate}",
                                 "threshold": GATE_THRESHOLD} if path == "gated" else None),
                       "l2": "flushed between timed steps (256 MB write outside the step events)",
                       "warmup_min_s": 1.0,
                       "replicas": world},
            "fp64_plain": fp64,
            "other_paths": others,
            "speedup_vs_fp64": value / fp64["value"],
            "matched_l1": l1,
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": launches,
            "kernel_ms": {k: round(v[1], 4) for k, v in prof.items()}, "clocks": clocks,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
