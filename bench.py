"""Benchmark of the cRK-FR hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload swe2d|swe1d|swe1d-limited|swe2d-limited|swe2d-friction|
                                swe2d-wb|ensemble|adjoint]

A step is one cRK-FR time step (element-local inner stages, time averages,
face Riemann problems with non-conservative fluctuations, FR corrections,
update, and the device-side time step of Eq. time.step.2d for the next step)
over the whole mesh.  Default workload: 2D shallow water with bathymetry on a
periodic 1024 x 1024 quad mesh, N = 3 (16 nodes, 3 variables per element),
32 seeded Gaussians of bathymetry, a seeded Gaussian bump on the free
surface, zero velocity, FP64, CFL 0.5 of the von Neumann limit.

Prints one JSON line.  `value` is DoF-updates/s with the state resident in
HBM (state + work buffers are about 3 GB, far larger than the 129 MB L2, so
no L2 flush is needed between steps); `e2e` repeats the measurement through
the C ABI's host-buffer entry point with the host<->device copies inside the
timed region.  `--impl reference` times the CPU oracle instead (the only
reference this method has), on a bounded periodic patch of the same
workload.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cRK-FR DoF-updates/s per step (FP64), % HBM roofline; adjoint/forward cost"
G = 9.81


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA lanes per
# SM per cycle x 2 flop x 2070 MHz.  The library's FMA-chain probe
# (crkfr_fp64_probe) measures 1.254 TFLOP/s at 2070 MHz, and every default
# bench line reports its own measurement beside this figure.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
HBM_FALLBACK_GBS = 6800.0


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
class Workload:
    def __init__(self, name, mesh=None):
        self.name = name
        self.source, self.source_coef, self.current = None, 0.0, (0.0, 0.0)
        self.limiter = None
        if name in ("swe2d", "swe2d-friction", "swe2d-wb", "swe2d-limited"):
            side = mesh or 1024
            self.system, self.N, self.E, self.L = "swe2d", 3, (side, side), 100.0
            self.M, self.dim = 3, 2
            if name == "swe2d-wb":
                self.system = "swe2d_wb"
            if name == "swe2d-limited":
                self.limiter = "blend"
            if name == "swe2d-friction":
                self.source, self.source_coef, self.current = "chezy", 0.0025, (0.3, 0.2)
        elif name in ("swe1d", "swe1d-limited"):
            self.system, self.N, self.E, self.L = "swe1d", 4, (mesh or 100000,), 100.0
            self.M, self.dim = 2, 1
            if name == "swe1d-limited":
                self.limiter = "blend"
        else:
            raise ValueError(name)
        n = self.N + 1
        self.n = n
        self.elements = int(np.prod(self.E))
        self.nodes_per_elem = n ** self.dim
        self.dof = self.elements * self.nodes_per_elem * self.M
        # minimal HBM traffic per step: read u and the bathymetry, write u
        self.min_bytes = self.elements * self.nodes_per_elem * (2 * self.M + 1) * 8

    def label(self):
        e = "x".join(str(v) for v in self.E)
        fr = f"-chezy{self.source_coef:g}" if self.source else ""
        lim = "-limited" if self.limiter else ""
        return f"{self.system}-{e}-N{self.N}{fr}{lim}"

    def cfl_key(self):
        return "cfl_imex" if self.source else "cfl"

    def oracle_system(self):
        from oracle.systems import ShallowWater1D, ShallowWater2D, ShallowWater2DWB
        return {"swe2d": ShallowWater2D, "swe2d_wb": ShallowWater2DWB,
                "swe1d": ShallowWater1D}[self.system](G)

    def oracle_source(self):
        from oracle.sources import ChezyFriction
        return ChezyFriction(self.source_coef) if self.source == "chezy" else None

    def inputs(self, positions, seed=0):
        from paper_2512_08611_gb300.workloads import SWE1DInput, SWE2DInput, accept_seed
        if self.dim == 2:
            inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=self.L, current=self.current),
                                 positions, seed)
        else:
            inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=self.L), positions, seed)
        return inp.state(*positions)

    def local_flops_per_element(self):
        """FP64 flops (FMA = 2) of the element-local kernel per element, from
        the operation count of its formulation (paper_2512_08611_gb300.flops);
        the 2D limited kernel adds its first-order part."""
        from paper_2512_08611_gb300.flops import (limiter_local_flops_per_element,
                                                  local_flops_per_element)
        f = local_flops_per_element(self.system, self.N, imex=self.source is not None)
        if self.limiter and self.dim == 2:
            f += limiter_local_flops_per_element(self.system, self.N)
        return f


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def host_link_gbs(host, dev):
    """Copy bandwidth of this process's pinned host buffer to and from the
    device (after the end-to-end timing; torch copies of the whole state,
    best of three, overwriting the device state, which nothing reads
    afterwards): the link bounds the end-to-end step, and the rate a process
    gets can vary between processes on the same machine."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best = {"h2d": 0.0, "d2h": 0.0}
    for _ in range(3):
        for key, (dst, src) in (("h2d", (dev, host)), ("d2h", (host, dev))):
            torch.cuda.synchronize()
            ev[0].record()
            dst.copy_(src, non_blocking=True)
            ev[1].record()
            torch.cuda.synchronize()
            best[key] = max(best[key], host.numel() * 8 / (ev[0].elapsed_time(ev[1]) * 1e6))
    return best


def l2_note(wl):
    """How the timed steps stand to the 129 MB L2 (no flush between steps):
    the state, its copy and, in 2D, the face traces and work buffers."""
    ws = wl.dof * 8 * (7.5 if wl.dim == 2 else 2.0)
    if ws > 129e6:
        size = "%.2f GB" % (ws / 1e9) if ws >= 1e9 else "%.0f MB" % (ws / 1e6)
        return "no flush: state + work buffers (%s) exceed the 129 MB L2" % size
    return ("no flush: state + work buffers (%.0f MB) stay in the 129 MB L2 between steps, as "
            "in any run on this mesh; the step is FP64-bound" % (ws / 1e6))


# ---------------------------------------------------------------------------
# profiles/ summary of the dominant kernel: dram traffic, valid only while the
# kernel source is unchanged
# ---------------------------------------------------------------------------
def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2512_08611_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary, files, scale):
    """dram bytes per launch from a profiles/ summary, scaled to the bench
    launch, or None if absent or taken on another version of the sources."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(files):
        return None
    return float(m_bytes.group(1)) * scale


# ---------------------------------------------------------------------------
# CPU oracle timing on a bounded periodic patch of the workload
# ---------------------------------------------------------------------------
def oracle_patch(wl, side):
    """(scheme, stepper, u, b, dof): the stepper is the scheme, or its
    blending limiter for a limited workload."""
    from oracle.basis import Basis
    from oracle.crkfr import Scheme1D, Scheme2D
    from oracle.limiter import Blending1D, Blending2D
    bs = Basis(wl.N)
    if wl.dim == 2:
        dx = wl.L / wl.E[0]
        x = (np.arange(side)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
        y = (np.arange(side)[:, None, None, None] + bs.xi[None, None, :, None]) * dx
        x, y = np.broadcast_arrays(x, y)
        u, b = wl.inputs((x, y))
        sch = Scheme2D(wl.oracle_system(), wl.N, dx, dx, source=wl.oracle_source())
        dof = side * side * wl.nodes_per_elem * wl.M
    else:
        dx = wl.L / wl.E[0]
        x = (np.arange(side)[:, None] + bs.xi[None, :]) * dx
        u, b = wl.inputs((x,))
        sch = Scheme1D(wl.oracle_system(), wl.N, dx)
        dof = side * wl.nodes_per_elem * wl.M
    stepper = sch
    if wl.limiter:
        stepper = (Blending2D if wl.dim == 2 else Blending1D)(sch)
    return sch, stepper, u, b, dof


def time_oracle(wl, budget_s, max_steps):
    """Oracle steps on a periodic patch cut from the workload (same per-element
    work), sized so that max_steps steps take about budget_s seconds."""
    import oracle.fourier  # noqa: F401  (imports numpy-only modules)
    probe = 32 if wl.dim == 2 else 4096
    sch, stepper, u, b, dof = oracle_patch(wl, probe)
    t0 = time.perf_counter()
    stepper.step(u, b, 1e-4)
    per_dof = (time.perf_counter() - t0) / dof
    target = budget_s / max(max_steps, 1) / per_dof
    if wl.dim == 2:
        side = int(np.clip(np.sqrt(target / (wl.nodes_per_elem * wl.M)) // 8 * 8, 16, wl.E[0]))
    else:
        side = int(np.clip(target / (wl.nodes_per_elem * wl.M) // 128 * 128, 512, wl.E[0]))
    sch, stepper, u, b, dof = oracle_patch(wl, side)
    return sch, u, b, dof, side


def cpu_threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    return 1


def _oracle_worker(job):
    """One host process: warm-up and timed oracle steps on its own copy of
    the patch (single-threaded numpy)."""
    name, mesh, side, steps, warmup, cfl = job
    wl = Workload(name, mesh)
    sch, stepper, u, b, dof = oracle_patch(wl, side)
    v = u
    for _ in range(warmup):
        v = stepper.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    t0 = time.perf_counter()
    for _ in range(steps):
        v = stepper.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    return dof, time.perf_counter() - t0


def oracle_on_all_cores(wl, budget_s, steps, warmup, procs=None):
    """The oracle, unchanged, stepping one patch per host core in separate
    processes (spawned: no process inherits a CUDA context); throughput =
    all processes' DoF-updates / the slowest process's time.  ``procs``: one
    process per core by default."""
    import multiprocessing
    cpu_threads()
    procs = procs or os.cpu_count() or 1
    sch, u, b, dof, side = time_oracle(wl, budget_s, steps + warmup)
    cfl = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")))[wl.cfl_key()][f"{wl.N}_gl"]
    job = (wl.name, wl.E[0], side, steps, warmup, cfl)
    with multiprocessing.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [job] * procs)
    tot = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    patch = f"{side}x{side}" if wl.dim == 2 else f"{side}"
    return tot * steps / el, el, procs, patch, res[0][0]


# ---------------------------------------------------------------------------
def run_reference(args, wl):
    budget = 90.0
    value, el, procs, patch, dof = oracle_on_all_cores(wl, budget, args.steps, args.warmup)
    sample = (f"{procs} processes, one per host core, each stepping its own periodic "
              f"{patch}-element patch cut from the {wl.label()} workload (same per-element "
              f"work) {args.steps} times after {args.warmup} warm-up steps")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DoF-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.label(), "sample": patch, "dof_per_step_per_process": dof,
                   "processes": procs},
        "cpu_baseline": {"value": value, "unit": "DoF-updates/s", "cores": procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DoF-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def build_once(world, dist):
    """Build the library (if it is not up to date) in one process only; the
    other ranks wait for it, so no two processes write the same files."""
    from paper_2512_08611_gb300.build import build_library
    if world > 1:
        if dist.get_rank() == 0:
            build_library()
        dist.barrier()
    build_library()


def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build_once(world, dist)
    from paper_2512_08611_gb300 import crkfr

    # the slab (1D: range) path of the multi-GPU runs; --split runs it on one
    # GPU, where the slab is its own periodic neighbour
    split = world > 1 or args.split
    s = crkfr.Solver(wl.system, wl.N, gravity=G, cfl_safety=0.5, source=wl.source,
                     source_coef=wl.source_coef)
    if split and wl.dim == 2:
        # weak scaling: this rank's slab is a full 1024 x 1024 workload, stacked
        # in y with the other ranks' slabs into one periodic mesh
        s.set_mesh(list(wl.E), [0.0, rank * wl.L], [wl.L, (rank + 1) * wl.L])
        s.set_subdomain(True)
    elif split:
        # 1D: this rank's range is a full workload mesh, the ranges side by side
        s.set_mesh(list(wl.E), [rank * wl.L], [(rank + 1) * wl.L])
        s.set_subdomain(True)
    else:
        s.set_mesh(list(wl.E), [0.0] * wl.dim, [wl.L] * wl.dim)
    pos = s.positions()
    if split and wl.dim == 2:
        pos = (pos[0], pos[1] - rank * wl.L)
    elif split:
        pos = pos - rank * wl.L
    u0, b = wl.inputs(pos if wl.dim == 2 else (pos,))
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    if split:
        # slabs (ranges) are identical (the inputs are periodic over one of
        # them), so the rows (elements) beyond this one's ends are its own
        # last and first ones
        K = wl.E[-1]
        b = np.ascontiguousarray(b[[K - 1] + list(range(K)) + [0]])
    s.set_coefficients(torch.tensor(b, dtype=torch.float64, device="cuda"))
    if wl.limiter:
        s.set_limiter(wl.limiter)
    if wl.dim == 1 and args.tile_1d:
        s.set_tile_1d(args.tile_1d)
    u_init = u.clone()
    stepper = None
    dt_fixed = 0.0
    if split:
        from paper_2512_08611_gb300.distributed import SlabStepper
        from paper_2512_08611_gb300.distributed import min_over_ranks
        stepper = SlabStepper(s)
        dt_fixed = min_over_ranks(s.compute_dt(u))

    def advance(k):
        if stepper is None:
            s.step(u, 0.0, k)
        else:
            stepper.step(u, dt_fixed, k)

    # warm-up
    advance(args.warmup)
    torch.cuda.synchronize()
    s.status()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.profile(True)
    n0 = s.launch_count()
    ev0.record(stream)
    advance(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = s.launch_count() - n0
    elapsed_ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    s.status()
    t_sim, dt_last = s.time()

    el = torch.tensor([elapsed_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(el, op=dist.ReduceOp.MAX)
    elapsed_ms = float(el.item())
    value = wl.dof * args.steps * world / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / args.steps

    # end to end through the host-buffer entry point (pinned host memory)
    state_bytes = wl.dof * 8
    e2e = None
    if split and not args.no_e2e:
        # end to end per rank: host copy in, one split step, host copy out
        host = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
        host.copy_(u_init.cpu())
        e2e_steps = max(3, min(args.steps, 20))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            u.copy_(host, non_blocking=True)
            stepper.step(u, dt_fixed, 1)
            host.copy_(u, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = {"value": wl.dof * e2e_steps * world / float(t.item()), "unit": "DoF-updates/s",
               "h2d_bytes_per_step": state_bytes * world, "d2h_bytes_per_step": state_bytes * world,
               "note": "torch pinned copies around the split step (no host entry point for slabs)"}
    elif not args.no_e2e:
        host = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
        host.copy_(u_init.cpu())
        h = host.numpy()
        e2e_steps = max(3, min(args.steps, 20))
        s.step_host(h, h, dt=0.0, nsteps=1)   # warm the host path (allocates its device copy)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            s.step_host(h, h, dt=0.0, nsteps=1)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": wl.dof * e2e_steps / e2e_s, "unit": "DoF-updates/s",
               "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
               "host_link_gbs": host_link_gbs(host, u)}

    # roofline of the dominant kernel
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    if wl.dim == 2:
        kname, files = "local_2d", ["local_2d.cuh", "device_common.cuh", "tableau.h"]
        if wl.limiter:
            files = files + ["limit_2d.cuh"]
        summary = ("k_local_2d__swe2d_friction_N3.md" if wl.source else
                   "k_local_2d__swe2d_wb_N3.md" if wl.system == "swe2d_wb" else
                   "k_local_2d__swe2d_N3_limited.md" if wl.limiter else
                   "k_local_2d__swe2d_N3.md")
    else:
        kname, files = "step_1d", ["step_1d.cuh", "device_common.cuh", "tableau.h"]
        summary = "k_step_1d__swe1d_N4_limited.md" if wl.limiter else "k_step_1d__swe1d_N4.md"
    nk, ms_k = prof.get(kname, (0, float("nan")))
    avg_ms = ms_k / max(nk, 1)
    flops = wl.local_flops_per_element() * wl.elements
    achieved = flops / (avg_ms / 1e3) / 1e12
    traffic = profiled_traffic(summary, files, 1.0)
    shares = {k: round(v[1] / max(sum(x[1] for x in prof.values()), 1e-30), 4) for k, v in prof.items()}
    # the FP64 rate this GPU reaches with independent FMA chains (the
    # library's probe; the roofline keeps the unit-count peak as denominator)
    fp64_measured = crkfr.fp64_probe("fma", blocks=1216, iters=4096, repeats=5)

    out = {
        "metric": METRIC, "value": value, "unit": "DoF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.label(), "elements": wl.elements,
                   "nodes_per_element": wl.nodes_per_elem, "vars": wl.M, "dof": wl.dof,
                   "cfl_safety": 0.5, "cfl": s.cfl(), "dt_last": dt_last, "t_sim": t_sim,
                   "l2": l2_note(wl),
                   "parallelism": "single GPU" if not split else
                   (f"one slab, its own periodic neighbour (the multi-GPU path on one GPU), "
                    f"fixed dt {dt_fixed:.6g}" if world == 1 else
                    f"{world} slabs of a 1024 x {1024 * world} mesh, one NCCL trace exchange per "
                    f"step, fixed dt {dt_fixed:.6g}" if wl.dim == 2 else
                    f"{world} ranges of a {wl.E[0] * world}-element periodic mesh, one NCCL "
                    f"exchange of the end elements per step, fixed dt {dt_fixed:.6g}")},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": traffic, "avg_launch_ms": avg_ms,
                     "flops_per_launch": flops,
                     "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz",
                     **({"flops_note": "the unlimited step's operation count: a lower bound "
                                       "of the limited kernel's work"}
                        if wl.limiter and wl.dim == 1 else
                        {"flops_note": "the unlimited step's count plus the first-order part "
                                       "of the limiter"} if wl.limiter else {})},
        "fp64_peak_measured": {"value": fp64_measured, "unit": "TFLOP/s",
                               "frac_of_derived": fp64_measured / FP64_PEAK_TFLOPS,
                               "kernel_frac_of_measured": achieved / fp64_measured,
                               "probe": "crkfr_fp64_probe: 8 independent FMA chains per thread, "
                                        "1216 blocks x 256 threads x 4096 iterations, best of 5 "
                                        "launches, after the timed region"},
        "hbm": {"min_bytes_per_step": wl.min_bytes,
                "achieved_gbs": wl.min_bytes / (ms_per_step / 1e3) / 1e9,
                "peak_gbs": hbm_peak,
                "frac": wl.min_bytes / (ms_per_step / 1e3) / 1e9 / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"},
        "kernel_shares": shares,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if wl.dim == 1:
        out["config"]["tile_threads_1d"] = args.tile_1d or "per mesh"
    if rank == 0 and world == 1 and wl.name == "swe2d" and not args.no_adjoint:
        # the metric's third part: the adjoint's cost against the forward run
        a = measure_adjoint(crkfr)
        out["adjoint"] = {k: v for k, v in a.items() if k != "dof"}
    if rank == 0 and world == 1 and not args.no_cpu:
        value_cpu, el_cpu, procs, patch, dof = oracle_on_all_cores(wl, 15.0, 2, 0)
        # and on one core (the oracle is single-threaded numpy)
        value_1, el_1, _, patch_1, _ = oracle_on_all_cores(wl, 8.0, 2, 0, procs=1)
        out["cpu_baseline"] = {
            "value": value_cpu, "unit": "DoF-updates/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes, one per host core, 2 oracle steps each on its own "
                      f"periodic {patch}-element patch cut from the {wl.label()} workload (same "
                      f"per-element work), numpy FP64 single-threaded per process",
            "single_core": {"value": value_1, "unit": "DoF-updates/s", "cores": 1,
                            "sample": f"one process, 2 oracle steps on a {patch_1}-element "
                                      f"patch of the same workload"}}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_ensemble(args):
    """Ragged ensemble: 256 independent 1D shallow-water meshes, element counts
    log-uniform in [2^10, 2^16], degrees from {2, 3, 4}, own seeded
    bathymetry and surface each; K CFL steps of all of them in one graph
    launch, against looping the single-mesh step over the instances.  Under
    torchrun every rank runs its own 256-instance ensemble (seeded by its
    rank) with no communication but the timing barrier and maximum (weak
    scaling)."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build_once(world, dist)
    from paper_2512_08611_gb300 import crkfr
    from paper_2512_08611_gb300.flops import local_flops_per_element
    from paper_2512_08611_gb300.workloads import SWE1DInput, accept_seed, ensemble_members
    L = 100.0
    mem = ensemble_members(256, seed=rank)
    nodes = {N: crkfr.Solver("swe1d", N).nodes()[0] for N in (2, 3, 4)}
    members, us, cs = [], [], []
    for m in mem:
        N, E = m["N"], m["E"]
        x = (np.arange(E)[:, None] + nodes[N][None, :]) * (L / E)
        inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), m["seed"])
        u, b = inp.state(x)
        members.append((N, E, 0.0, L))
        us.append(u)
        cs.append(b)
    dof = sum(u.size for u in us)
    flops_step = sum(local_flops_per_element("swe1d", N) * E for N, E, _, _ in members)
    batch = crkfr.Batch("swe1d", members, gravity=G, cfl_safety=0.5)
    u = torch.cat([torch.tensor(x.ravel()) for x in us]).cuda()
    c = torch.cat([torch.tensor(x.ravel()) for x in cs]).cuda()
    u0 = u.clone()
    batch.set_coefficients(c)
    # launch shape chosen by the library's autotuner (times the shapes as
    # captured graphs on a scratch copy of the state)
    t_tune = time.perf_counter()
    tpb, order, parallel, tune_ms = batch.autotune(u, steps=5)
    t_tune = time.perf_counter() - t_tune
    batch.step(u, 0.0, args.steps, graph=True)     # capture + warm-up
    u.copy_(u0)
    batch.step(u, 0.0, args.warmup, graph=False)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    n0 = batch.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record()
    batch.step(u, 0.0, args.steps, graph=True)
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    batch.status()
    ms = ev0.elapsed_time(ev1)
    tot_dof = dof
    if world > 1:
        t = torch.tensor([ms, float(dof)], dtype=torch.float64, device="cuda")
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t[1:].clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms, tot_dof = float(mx.item()), float(sm.item())
    launches = batch.launch_count() - n0
    # time between kernels: the same steps without a graph with every kernel
    # timed (their sum) against the graph's wall time, for the tuned shape
    # and for one serial chain of launches
    batch.set_tuning(tpb, order, 0)
    u.copy_(u0)
    batch.step(u, 0.0, args.warmup, graph=False)
    batch.profile(True)
    batch.step(u, 0.0, args.steps, graph=False)
    n_k, kernel_ms = batch.profile_read()
    batch.profile(False)
    u.copy_(u0)
    batch.step(u, 0.0, args.steps, graph=True)     # capture + warm-up
    u.copy_(u0)
    torch.cuda.synchronize()
    ev0.record()
    batch.step(u, 0.0, args.steps, graph=True)
    ev1.record()
    torch.cuda.synchronize()
    ms_serial = ev0.elapsed_time(ev1)
    batch.set_tuning(tpb, order, parallel)
    # looping the single-mesh step over the instances
    solvers, states = [], []
    for (N, E, lo, hi), x, b in zip(members, us, cs):
        s = crkfr.Solver("swe1d", N, gravity=G, cfl_safety=0.5)
        s.set_mesh([E], [lo], [hi])
        s.set_coefficients(torch.tensor(b).cuda())
        solvers.append(s)
        states.append(torch.tensor(x).cuda())
    for s, x in zip(solvers, states):
        s.step(x, 0.0, args.warmup)
    torch.cuda.synchronize()
    ev0.record()
    for s, x in zip(solvers, states):
        s.step(x, 0.0, args.steps)
    ev1.record()
    torch.cuda.synchronize()
    ms_loop = ev0.elapsed_time(ev1)
    value = tot_dof * args.steps / (ms / 1e3)
    looped = dof * args.steps / (ms_loop / 1e3)
    achieved = flops_step * args.steps / (ms / 1e3) / 1e12
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "DoF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "ensemble-256-swe1d-E2^10..2^16-N2..4", "instances": len(members),
                   "elements": int(sum(m[1] for m in members)), "dof": int(dof),
                   "l2": "state 250 MB > 129 MB L2, no flush",
                   "mode": "one CUDA graph of K steps, one launch per degree class per step",
                   "tuning": {"tiles_per_block": tpb, "order": ["instance", "largest first"][order],
                              "degree_classes": "concurrent branches" if parallel else "serial",
                              "autotune_s": t_tune, "tuned_ms_per_step": tune_ms}},
        "looped": {"value": looped, "ms_per_step": ms_loop / args.steps,
                   "mode": "crkfr_step of K steps per instance, instances in sequence (rank 0)"},
        "speedup_vs_looped": (dof * args.steps / (ms / 1e3)) / looped,
        "launch_gaps": {
            "graph_ms_per_step": ms / args.steps,
            "serial_graph_ms_per_step": ms_serial / args.steps,
            "kernel_ms_per_step": kernel_ms / args.steps, "kernels_timed": n_k,
            "gap_fraction_serial": 1.0 - kernel_ms / ms_serial,
            "note": "kernel_ms: sum of every step kernel's duration (CUDA events, no graph, "
                    "degree classes one after another); the serial graph runs the same "
                    "kernels back to back, so its excess over the sum is the time between "
                    "kernels that one persistent launch could remove"},
        "fp64_ceiling": {
            "flop_per_dof_update": flops_step / dof,
            "dof_updates_per_s": FP64_PEAK_TFLOPS * 1e12 * dof / flops_step,
            "max_ratio_over_looped": FP64_PEAK_TFLOPS * 1e12 * dof / flops_step / looped},
        "roofline": {"bound": "alu", "kernel": "k_step_1d_batch (all kernels of the step)",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": profiled_traffic("k_step_1d_batch__ensemble256.md",
                                                 ["step_1d.cuh", "device_common.cuh", "tableau.h"],
                                                 1.0),
                     "traffic_unit": "bytes per step (the degree classes' launches)"},
        "gpu_launches": launches, "clocks": clk}))


def measure_adjoint(crkfr, E=256, N=3, L=100.0, nsteps=200, every=20, split=False):
    """Gradient of the final surface misfit w.r.t. the bathymetry on the 2D
    E x E, N = 3 mesh: nsteps fixed steps, checkpoints every `every` steps,
    the backward pass recomputing each segment with recorded steps.  Returns
    the forward and backward times (CUDA events) and the per-step costs.
    split: the slab path of the multi-GPU runs (one slab, its own periodic
    neighbour: SlabBathymetryToState over a SlabStepper)."""
    import torch
    from paper_2512_08611_gb300.adjoint import (BathymetryToState, SlabBathymetryToState,
                                                quadrature_weights, surface_misfit)
    from paper_2512_08611_gb300.distributed import SlabStepper
    from paper_2512_08611_gb300.workloads import SWE2DInput, accept_seed
    s = crkfr.Solver("swe2d", N, gravity=G, cfl_safety=0.5)
    s.set_mesh([E, E], [0.0, 0.0], [L, L])
    if split:
        s.set_subdomain(True)
        stepper = SlabStepper(s)
        apply = lambda bb: SlabBathymetryToState.apply(bb, stepper, eta0, dt, nsteps, every)
    else:
        apply = lambda bb: BathymetryToState.apply(bb, s, eta0, dt, nsteps, every)
    x, y = s.positions()
    inp, _ = accept_seed(lambda k: SWE2DInput(seed=k, L=L), (x, y), 0)
    _, b = inp.state(x, y)
    inp2, _ = accept_seed(lambda k: SWE2DInput(seed=k, L=L), (x, y), 7)
    _, b2 = inp2.state(x, y)
    eta0 = torch.tensor(inp.eta(x, y), device="cuda")
    bt, b2t = torch.tensor(b, device="cuda"), torch.tensor(b2, device="cuda")
    s.set_coefficients(torch.cat([b2t[-1:], b2t, b2t[:1]]).contiguous() if split else b2t)
    dt = 0.5 * s.compute_dt(torch.stack([eta0 - b2t, 0 * b2t, 0 * b2t]).contiguous())
    W = quadrature_weights(s)
    with torch.no_grad():
        target = apply(b2t)[0] + b2t
    # warm-up of both directions
    bb = bt.clone().requires_grad_(True)
    surface_misfit(apply(bb), bb, target, W).backward()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    bb = bt.clone().requires_grad_(True)
    s.profile(True)
    ev[0].record()
    J = surface_misfit(apply(bb), bb, target, W)
    ev[1].record()
    J.backward()
    ev[2].record()
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    n_adj, ms_adj = prof.get("adjoint_2d", (0, 0.0))
    return {"workload": f"adjoint-swe2d-{E}x{E}-N{N}-{nsteps}steps-ckpt{every}"
                        + ("-slab" if split else ""),
            "loss": "1/2 sum w (h + b - target)^2 at T", "dt": dt,
            "forward_ms": fwd, "backward_ms": bwd,
            "backward_over_forward": bwd / fwd,
            "forward_step_ms": fwd / nsteps,
            "adjoint_step_ms": ms_adj / max(n_adj, 1),
            "adjoint_step_over_forward_step": (ms_adj / max(n_adj, 1)) / (fwd / nsteps),
            "backward": "segments recomputed from checkpoints with recorded steps "
                        "(face traces and stage values kept), adjoint steps read the records",
            "gradient_norm": float(bb.grad.norm()),
            "dof": 3 * E * E * (N + 1) ** 2}


def run_adjoint(args):
    """The adjoint workload alone: cost of the adjoint relative to the forward
    run (Sec. 3, Eq. crkfr.non.cons.final reversed)."""
    import torch
    from paper_2512_08611_gb300.build import build_library
    build_library()
    from paper_2512_08611_gb300 import crkfr
    torch.cuda.set_device(0)
    nsteps = 200
    a = measure_adjoint(crkfr, nsteps=nsteps, split=args.split)
    print(json.dumps({
        "metric": METRIC, "value": a["dof"] * nsteps / (a["backward_ms"] / 1e3),
        "unit": "DoF-updates/s (adjoint)",
        "n_gpus": 1, "steps": nsteps, "warmup": 1, "ms_per_step": a["backward_ms"] / nsteps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": a["workload"], "loss": a["loss"], "dt": a["dt"]},
        **{k: v for k, v in a.items() if k not in ("workload", "loss", "dt", "dof")}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="swe2d",
                    choices=["swe2d", "swe1d", "swe1d-limited", "swe2d-limited", "swe2d-friction",
                             "swe2d-wb",
                             "ensemble", "adjoint"])
    ap.add_argument("--mesh", type=int, default=None,
                    help="elements per side (2D) or elements (1D); profiling of small cases")
    ap.add_argument("--split", action="store_true",
                    help="run the multi-GPU (slab / range) path on one GPU")
    ap.add_argument("--tile-1d", type=int, default=0, choices=[0, 64, 96, 128],
                    help="threads per block of the 1D step (0: chosen per mesh)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint measurement of the default workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "adjoint":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the adjoint workload reports its own adjoint/forward ratio"}))
            return
        run_adjoint(args)
        return
    if args.workload == "ensemble":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the ensemble workload is timed against looping the GPU step"}))
            return
        run_ensemble(args)
        return
    wl = Workload(args.workload, args.mesh)
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
