"""Benchmark: one RK stage (ibm_substep) of the immersed-boundary solver.

A step is one pass of the whole hot path over one state: E1 explicit terms,
L2 marker motion, L1 interpolation / force / spreading, three Helmholtz
solves, divergence, the refined Poisson solve and the projection with the
pressure update.  Workload: 128^3 grid on [0,2pi) x [0,2] x [0,2pi]
(periodic x, z; walls in y), FP32 fields with one refinement step, a
20,000-marker Fibonacci sphere (radius 0.25, centre (pi, 1, pi)) translating
at 0.1 in x, a seeded discretely divergence-free velocity with energy
spectrum ~ k^-5/3 (k <= 16).  Four independent states rotate across steps
(4 x 56 MB > 129 MB L2) so every step reads its fields from HBM.

Output: one JSON line (rank 0).  `value` is grid points advanced per second
(all ranks) over the untraced timed region, `e2e` the same through host
buffers, `roofline` the dominant kernel's achieved HBM bandwidth from CUDA
events around each of its launches in an identical second pass of the same
steps, `cpu_baseline` the FP64 CPU oracle on a bounded sample.
`--impl reference` times that oracle alone.
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Poisson solves/s and grid-pts/s at 1 GB300 (% HBM roofline); FP32-refined vs FP64 at 1e-6; "
          "p50/p99")
NX = NY = NZ = 128
N_MARKERS = 20000
DT, NU = 1e-3, 1e-2
N_STATES = 4
KERNEL_SOURCES = {"forward": ("transforms.cu", "axis.cu", "fft2.cuh"),
                  "inverse": ("transforms.cu", "axis.cu", "fft2.cuh"), "pencil": ("pencil.cu",),
                  "residual": ("stencil.cu",), "explicit": ("substep.cu",), "divergence": ("substep.cu",),
                  "project": ("substep.cu",), "interp": ("ibm_kernels.cu",), "spread": ("ibm_kernels.cu",),
                  "motion": ("ibm_kernels.cu",)}
# kernel-name prefix -> kind (the names ncu prints)
KERNEL_KIND = (("k_plane_fwd", "forward"), ("k_rows_fwd", "forward"), ("k_cplane_fwd", "forward"),
               ("k_plane_inv", "inverse"), ("k_rows_inv", "inverse"), ("k_cplane_inv", "inverse"),
               ("k_pencil", "pencil"), ("k_residual", "residual"), ("k_explicit", "explicit"),
               ("k_divergence", "divergence"), ("k_project", "project"), ("k_interp", "interp"),
               ("k_spread", "spread"), ("k_motion", "motion"))
WORKLOAD = "ibm_substep 128^3 FP32+1 refinement, 20k-marker sphere"


def workload_grid():
    from paper_2406_19920_gb300 import synth
    return synth.grid(NX, NY, NZ)


def make_inputs(g):
    """Seeded host inputs (FP64) shared by the GPU arm and the CPU baseline."""
    from paper_2406_19920_gb300 import synth
    u, v, w = synth.div_free_velocity(g, workload=1, kmax=16.0)
    X0, dV = synth.fibonacci_sphere(N_MARKERS, 0.25, (math.pi, 1.0, math.pi), g[3])
    return (u, v, w), X0, dV


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def source_digest(kind):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2406_19920_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind, workload):
    """DRAM bytes per step of a kernel kind from the committed ncu summary,
    if its sources are unchanged since the capture; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kind)
    if not e or e.get("workload") != workload or e.get("source_sha256_16") != source_digest(kind):
        return None
    return e.get("dram_bytes_per_step")


def algorithmic_bytes(kind, esz=4):
    """Compulsory HBM bytes per step (one RK stage) of each kernel kind.

    pts = nx ny nz real points; spec = ny nz (nx/2+1) complex entries.  A
    stage transforms five fields each way: the three Helmholtz increments
    (one shared launch set) and the Poisson solve plus its refinement.
    forward: read field + write spectrum, x5; inverse: read spectrum + write
    field, x5, plus the added field of the three Helmholtz increments and of
    the refinement update; pencil: read + write spectrum, x5; residual: read
    b, x, write r; explicit: read u,v,w,p, N x3, write du,dv,dw, N x3;
    divergence: read u,v,w, write b; project: read u,v,w,p,phi, write
    u,v,w,p; markers: positions, weights, 27-point stencils of 3 components.
    The spectrum round trip between the split x and z passes is not counted
    (it is not compulsory: the one-CTA plane kernels avoid it).
    """
    pts = NX * NY * NZ
    spec = NY * NZ * (NX // 2 + 1)
    cs = 2 * esz
    table = {
        "forward": 5 * (pts * esz + spec * cs),
        "inverse": 5 * (spec * cs + pts * esz) + 4 * pts * esz,
        "pencil": 5 * 2 * spec * cs,
        "residual": 3 * pts * esz,
        "explicit": 13 * pts * esz,
        "divergence": 4 * pts * esz,
        "project": 9 * pts * esz,
        "interp": N_MARKERS * 3 * (3 * esz + 27 * 2 * esz),
        "spread": N_MARKERS * 3 * (5 * esz + 27 * esz * 2),
        "motion": N_MARKERS * (3 + 6) * esz,
    }
    return table.get(kind)


def kernel_kind(name):
    name = name.replace("void ", "", 1).replace("ibm::", "")
    if name.startswith("k_cols<"):  # k_cols<T, N, INV>
        return "inverse" if name.split(">")[0].split(",")[-1].strip() in ("true", "1") else "forward"
    for prefix, kind in KERNEL_KIND:
        if name.startswith(prefix):
            return kind
    return None


def ncu_summary(csv_path, steps):
    """Per-kind launches, device time and DRAM bytes per step from an ncu
    --csv launch list of `bench.py --quick` (profiler region = the timed
    steps); writes profiles/dram_traffic.json and prints a markdown table."""
    import csv
    rows = []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        rows.append(r)
    agg = {}
    for r in rows:
        kind = kernel_kind(r["Kernel Name"])
        if kind is None:
            continue
        short = r["Kernel Name"].replace("void ", "", 1).replace("ibm::", "").split("(")[0]
        a = agg.setdefault((kind, short), {"ids": set(), "ns": 0.0, "rd": 0.0, "wr": 0.0})
        a["ids"].add(r["ID"])
        val = float(r["Metric Value"].replace(",", ""))
        unit = r["Metric Unit"]
        scale = {"ns": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6, "nsecond": 1.0,
                 "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1.0)
        if r["Metric Name"] == "gpu__time_duration.sum":
            a["ns"] += val * scale
        elif r["Metric Name"] == "dram__bytes_read.sum":
            a["rd"] += val * scale
        elif r["Metric Name"] == "dram__bytes_write.sum":
            a["wr"] += val * scale
    total_ns = sum(a["ns"] for a in agg.values())
    print("| kernel | kind | launches/step | us/step | share | DRAM MB/step (read+write) |")
    print("|---|---|---|---|---|---|")
    kinds = {}
    for (kind, name), a in sorted(agg.items(), key=lambda kv: -kv[1]["ns"]):
        print("| %s | %s | %.1f | %.2f | %.1f%% | %.2f |" % (name, kind, len(a["ids"]) / steps, a["ns"] / 1e3 / steps,
                                                         100 * a["ns"] / total_ns, (a["rd"] + a["wr"]) / 1e6 / steps))
        k = kinds.setdefault(kind, {"ns": 0.0, "bytes": 0.0})
        k["ns"] += a["ns"]
        k["bytes"] += a["rd"] + a["wr"]
    out = {kind: {"workload": WORKLOAD, "dram_bytes_per_step": v["bytes"] / steps,
                  "device_us_per_step": v["ns"] / 1e3 / steps, "share": v["ns"] / total_ns,
                  "source_sha256_16": source_digest(kind),
                  "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum summed over the kind's launches of "
                          "one step, each launch replayed with caches flushed"}
           for kind, v in kinds.items()}
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def job_ms(ms, dist=None, device="cpu"):
    """The job's time: the maximum of the ranks' times (every rank runs the
    same steps between the same barriers)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world_size, ms):
    """Whole-job rate: the units all ranks processed over the job's time
    (weak scaling: each rank advances its own replica)."""
    return units_per_rank * world_size / (ms * 1e-3)


def run_gpu(args):
    import torch
    import paper_2406_19920_gb300 as ibm
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    g = workload_grid()
    (u, v, w), X0, dV = make_inputs(g)
    f32 = torch.float32
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", f32)
    plan = ibm.ibm_plan_create(NX, NY, NZ, g[3:], ibm.IBM_FP32_REFINED, 1)
    # N_STATES independent states; each step advances the next one
    states, keep = [], []
    for s in range(N_STATES):
        fields = [dev(u), dev(v), dev(w), torch.zeros((NY, NZ, NX), dtype=f32, device="cuda")]
        Ns = [torch.zeros((NY, NZ, NX), dtype=f32, device="cuda") for _ in range(3)]
        st = ibm.ibm_state(*[t.data_ptr() for t in fields + Ns], 0.0)
        states.append(st)
        keep.append((fields, Ns))
    X0d, dVd = dev(X0), dev(dV)
    X = torch.empty((N_MARKERS, 3), dtype=f32, device="cuda")
    Ud = torch.empty_like(X)
    F = torch.empty_like(X)
    params = (ctypes.c_double * 4)(0.1, 0.0, 0.0, 0.0)
    mk = ibm.ibm_markers(N_MARKERS, X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                         ibm.IBM_MOTION_TRANSLATE, params)
    stream = torch.cuda.current_stream()

    def step(i):
        st = states[i % N_STATES]
        ibm.ibm_substep(plan, st, (i // N_STATES) % 3 + 1, DT, NU, mk, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    info = ibm.ibm_substep(plan, states[0], 1, DT, NU, mk, info=True)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    if args.quick:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.cudart().cudaProfilerStart()  # `ncu --profile-from-start off` captures these steps only
        e0.record()
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record()
        barrier()
        torch.cuda.cudart().cudaProfilerStop()
        ms = e0.elapsed_time(e1)
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": ms / args.steps,
                              "value": NX * NY * NZ * args.steps * ws / (ms * 1e-3)}), flush=True)
        ibm.ibm_plan_destroy(plan)
        return

    # ---- timed region: K steps, no tracing; clocks sampled throughout ----
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        time.sleep(0.3)  # let the sampler start before the timed region
        barrier()
        t_host0 = time.time()
        ev[0].record()
        for i in range(args.steps):
            step(args.warmup + i)
            ev[i + 1].record()
        barrier()
        t_host1 = time.time()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = job_ms(ev[0].elapsed_time(ev[-1]), dist, "cuda")
    pts = NX * NY * NZ
    value = job_throughput(pts * args.steps, ws, total_ms)

    # ---- identical pass with CUDA events around every kernel (roofline) ----
    ibm.ibm_plan_profile(plan, True)
    ibm.ibm_plan_profile_read(plan)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        step(args.warmup + args.steps + i)
    e1.record()
    barrier()
    traced_ms = e0.elapsed_time(e1)
    prof = ibm.ibm_plan_profile_read(plan)
    ibm.ibm_plan_profile(plan, False)

    # ---- end to end: host buffers, copies inside the timed region ----
    # Every step uploads its inputs (7 fields) from pinned host memory and
    # reads its 4 result fields back.  Two device state sets alternate: step
    # i's upload runs on an upload stream while step i-1 computes, and its
    # download on a download stream while step i+1 computes (the plan's
    # stages stay in order on the compute stream).
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).to(f32).pin_memory()
               for a in (u, v, w, np.zeros_like(u), np.zeros_like(u), np.zeros_like(u), np.zeros_like(u))]
    host_out = [torch.empty((NY, NZ, NX), dtype=f32).pin_memory() for _ in range(4)]
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    e2e_steps = max(3, min(args.steps, 20))
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]
    barrier()
    e0.record()
    s_up.wait_stream(stream)
    s_down.wait_stream(stream)
    for i in range(e2e_steps):
        b = i % 2
        fields_b, Ns_b = keep[b]
        with torch.cuda.stream(s_up):
            if i >= 2:
                s_up.wait_event(ev_down[b])  # buffer b's previous results are out
            for dsrc, hsrc in zip(fields_b + Ns_b, host_in):
                dsrc.copy_(hsrc, non_blocking=True)
            ev_up[b].record(s_up)
        stream.wait_event(ev_up[b])
        states[b].t = 0.0
        ibm.ibm_substep(plan, states[b], 1, DT, NU, mk, stream=stream)
        ev_done[b].record(stream)
        with torch.cuda.stream(s_down):
            s_down.wait_event(ev_done[b])
            for hdst, dsrc in zip(host_out, fields_b):
                hdst.copy_(dsrc, non_blocking=True)
            ev_down[b].record(s_down)
    stream.wait_stream(s_up)
    stream.wait_stream(s_down)
    e1.record()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = pts * e2e_steps * ws / (e2e_ms * 1e-3)

    # ---- standalone Poisson: FP32-refined vs FP64 at 128^3, and 256^3 ----
    solves = poisson_compare(ibm, torch, NX, (("fp32_refined", ibm.IBM_FP32_REFINED, 1), ("fp64", ibm.IBM_FP64, 0)))
    solves_256 = None
    if not args.no_extras:
        solves_256 = poisson_compare(ibm, torch, 256, (("fp32", ibm.IBM_FP32_REFINED, 0),
                                                       ("fp32_refined", ibm.IBM_FP32_REFINED, 1),
                                                       ("fp64", ibm.IBM_FP64, 0)), nb=4, K=20)
        # triply periodic branch (y-FFT pencil step instead of the Thomas sweep)
        solves_256["triply_periodic"] = poisson_compare(
            ibm, torch, 256, (("fp32", ibm.IBM_FP32_REFINED, 0), ("fp64", ibm.IBM_FP64, 0)), nb=4, K=20,
            bc=ibm.IBM_BC_TRIPLY_PERIODIC)

    # ---- spreading: atomic L1 kernel vs deterministic Eulerian gather ----
    spreading = spread_compare(ibm, torch) if not args.no_extras else None

    # ---- batched (64 instances, one graph launch) and served workloads ----
    batched = batched_compare(ibm, torch) if not args.no_extras else None
    dft = dft_compare(ibm, torch) if not args.no_extras else None
    serving = serve_sample(ibm) if not args.no_extras else None
    plate = large_plate(ibm, torch) if not args.no_extras else None
    plate_inflow = large_plate(ibm, torch, v_in=1.0) if not args.no_extras else None

    # ---- roofline of the dominant kernel kind (all its launches of a step) ----
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    avg_ms = dom_ms / max(dom_launches, 1)
    dom_step_ms = dom_ms / args.steps
    alg = algorithmic_bytes(dom)
    peak, peak_src = measured_peak()
    achieved = alg / (dom_step_ms * 1e-3) / 1e9
    workload_name = WORKLOAD
    traffic = ncu_traffic(dom, workload_name)
    launches = sum(c for _, c in prof.values())

    clocks = clk.summary()
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "grid-pts/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name, "grid": [NX, NY, NZ], "domain": "[0,2pi)x[0,2]x[0,2pi]",
                   "markers": N_MARKERS, "precision": "FP32 fields, FP64 zero mode, 1 float-float refinement",
                   "l2": "4 rotating states (224 MB) > 129 MB L2", "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "e2e": {"value": e2e_value, "unit": "grid-pts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps,
                "overlap": "two device state sets: step i's upload and download overlap the neighbouring "
                           "steps' compute (separate upload, compute and download streams)"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                     "per": "step (all launches of the kind in one RK stage)",
                     "algorithmic_bytes": alg, "ms_per_step": dom_step_ms,
                     "launches_per_step": dom_launches / args.steps, "avg_launch_ms": avg_ms},
        "kernels_ms_per_step": {k: prof[k][0] / args.steps for k in prof},
        "launches_per_step": {k: prof[k][1] / args.steps for k in prof},
        "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "value_traced": pts * args.steps * ws / (traced_ms * 1e-3),
        "poisson": solves,
        "poisson_256": solves_256,
        "spreading": spreading,
        "batched": batched,
        "dft_tensor_core": dft,
        "serving": serving,
        "large_plate": plate,
        "large_plate_inflow": plate_inflow,
        "stage_info": {k: info[k] for k in ("div_max", "div_before", "removed_mean")},
        "clocks": clocks,
        "timed_region_s": t_host1 - t_host0,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    ibm.ibm_plan_destroy(plan)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def method_bytes(n, precision_bytes, refine):
    """Compulsory HBM bytes of one Poisson solve on an n^3 grid: forward
    (read field, write spectrum), pencil (read + write spectrum), inverse
    (read spectrum, write field); a refinement step adds the residual (read
    b and x, write r), a second solve and the read of the updated field."""
    pts = n ** 3
    spec = n * n * (n // 2 + 1)
    s = precision_bytes
    solve = pts * s + 2 * spec * s + 2 * 2 * spec * s + 2 * spec * s + pts * s
    return solve + refine * (3 * pts * s + solve + pts * s)


def poisson_compare(ibm, torch, n, variants, nb=16, K=40, bc=None):
    """Standalone Poisson solves on an n^3 grid ([0,2pi)x[0,2]x[0,2pi],
    low-passed noise right-hand side): solves/s, p50/p99 latency, and the
    achieved fraction of the measured HBM bandwidth for the solve's method
    bytes; relative L2 of each FP32 result against the FP64 GPU result."""
    from paper_2406_19920_gb300 import synth
    g = synth.grid(n, n, n)
    b = synth.rhs_lowpass_noise(n, n, n, kmax=min(32.0, n / 4), workload=1)
    res = {}
    outs = {}
    for name, prec, ref in variants:
        dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
        plan = ibm.ibm_plan_create(n, n, n, g[3:], prec, ref, bc=bc if bc is not None else ibm.IBM_BC_PXZ_WALL_Y)
        rhs = [torch.from_numpy(b).to("cuda", dt) for _ in range(nb)]  # nb rhs + nb solutions > L2
        phi = [torch.empty_like(r) for r in rhs]
        for i in range(3):
            ibm.ibm_poisson_solve(plan, rhs[i], phi[i])
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        torch.cuda.synchronize()
        evs[0].record()
        for i in range(K):
            ibm.ibm_poisson_solve(plan, rhs[i % nb], phi[i % nb])
            evs[i + 1].record()
        torch.cuda.synchronize()
        lat = [evs[i].elapsed_time(evs[i + 1]) for i in range(K)]
        ms = evs[0].elapsed_time(evs[-1]) / K
        outs[name] = phi[0].double().cpu().numpy()
        mb = method_bytes(n, 4 if dt == torch.float32 else 8, ref if dt == torch.float32 else 0)
        res[name] = {"solves_per_s": 1e3 / ms, "grid_pts_per_s": n ** 3 * 1e3 / ms, "ms": ms,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "method_bytes": mb,
                     "hbm_frac_method_bytes": mb / (ms * 1e-3) / 1e9 / measured_peak()[0]}
        ibm.ibm_plan_destroy(plan)
        del rhs, phi
        torch.cuda.empty_cache()
    for name in outs:
        if name != "fp64" and "fp64" in outs:
            d = outs[name] - outs["fp64"]
            res[name]["rel_l2_vs_fp64"] = float(np.linalg.norm(d) / np.linalg.norm(outs["fp64"]))
    if "fp32_refined" in res and "fp64" in res:
        res["speedup_fp32_refined_over_fp64"] = res["fp32_refined"]["solves_per_s"] / res["fp64"]["solves_per_s"]
    return res


def spread_compare(ibm, torch):
    """Spreading (Eq. 2d) of a Fibonacci sphere at 128^3, FP32: the default
    atomic kernel (shared-memory pre-aggregation per CTA), the paper's L1
    kernel (direct global atomics) and the deterministic Eulerian gather; us
    per call, markers per second, and whether four repeated calls give the
    same bytes."""
    from paper_2406_19920_gb300 import synth
    res = {}
    g = workload_grid()
    for n in (N_MARKERS, 100000):
        X, dV = synth.fibonacci_sphere(n, 0.25, (math.pi, 1.0, math.pi), g[3])
        F = synth.marker_forces(n, workload=3)
        plan = ibm.ibm_plan_create(NX, NY, NZ, g[3:], ibm.IBM_FP32_REFINED, 1)
        Xd, Fd, dVd = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32) for a in (X, F, dV))
        row = {}
        for name, mode in (("atomic", ibm.IBM_SPREAD_ATOMIC), ("atomic_direct", ibm.IBM_SPREAD_ATOMIC_DIRECT),
                           ("gather", ibm.IBM_SPREAD_GATHER)):
            ibm.ibm_plan_set_spread(plan, mode)
            outs = []
            for _ in range(4):
                f = [torch.zeros((NY, NZ, NX), dtype=torch.float32, device="cuda") for _ in range(3)]
                ibm.ibm_spread(plan, n, Xd, Fd, dVd, *f)
                outs.append(f)
            torch.cuda.synchronize()
            same = all(torch.equal(a, b) for o in outs[1:] for a, b in zip(outs[0], o))
            f = outs[0]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            K = 20
            e0.record()
            for _ in range(K):
                ibm.ibm_spread(plan, n, Xd, Fd, dVd, *f)
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / K * 1e3
            row[name] = {"us": us, "markers_per_s": n / (us * 1e-6), "bitwise_repeatable": bool(same)}
        res["sphere_%dk" % (n // 1000)] = row
        ibm.ibm_plan_destroy(plan)
    return res


def solve_twice(n, plane_mode=None):
    """Two refined FP32 Poisson solves on an n^3 grid of the workload domain
    (N(0,1) right-hand side): the launch sequence the profiles of the 256^3
    solve are taken from.  plane_mode: forces that plane mode of the
    transforms (-1 the tensor-core DFT products)."""
    import torch
    import paper_2406_19920_gb300 as ibm
    from paper_2406_19920_gb300 import synth
    g = synth.grid(n, n, n)
    if plane_mode is not None:
        os.environ["IBM_PLANE_MODE"] = str(plane_mode)
    try:
        plan = ibm.ibm_plan_create(n, n, n, g[3:], ibm.IBM_FP32_REFINED, 1)
    finally:
        os.environ.pop("IBM_PLANE_MODE", None)
    b = torch.randn((n, n, n), device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(1))
    x = torch.empty_like(b)
    for _ in range(2):
        ibm.ibm_poisson_solve(plan, b, x)
    torch.cuda.synchronize()
    ibm.ibm_plan_check(plan)
    ibm.ibm_plan_destroy(plan)


def spread_twice(n, mode):
    """Profiling aid: two spreads of an n-marker Fibonacci sphere (radius
    0.25) on the 128^3 workload grid, FP32, in spreading mode `mode`
    (atomic, direct or gather)."""
    import torch
    import paper_2406_19920_gb300 as ibm
    from paper_2406_19920_gb300 import synth
    g = workload_grid()
    X, dV = synth.fibonacci_sphere(n, 0.25, (math.pi, 1.0, math.pi), g[3])
    F = synth.marker_forces(n, workload=3)
    plan = ibm.ibm_plan_create(NX, NY, NZ, g[3:], ibm.IBM_FP32_REFINED, 1)
    ibm.ibm_plan_set_spread(plan, {"atomic": ibm.IBM_SPREAD_ATOMIC, "direct": ibm.IBM_SPREAD_ATOMIC_DIRECT,
                                   "gather": ibm.IBM_SPREAD_GATHER}[mode])
    Xd, Fd, dVd = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32) for a in (X, F, dV))
    f = [torch.zeros((NY, NZ, NX), dtype=torch.float32, device="cuda") for _ in range(3)]
    for _ in range(2):
        ibm.ibm_spread(plan, n, Xd, Fd, dVd, *f)
    torch.cuda.synchronize()
    ibm.ibm_plan_check(plan)
    ibm.ibm_plan_destroy(plan)


def _batch_ms(ibm, torch, dims, hs, rhs, phi, reps=5):
    """Creates (and tunes) a batch, runs the four right-hand-side sets once,
    then times `reps` rounds of them; returns (batch, ms per round, create s)."""
    t0 = time.perf_counter()
    b = ibm.ibm_batch_create(dims, hs, ibm.IBM_FP32_REFINED, 1)
    create_s = time.perf_counter() - t0
    for k in range(4):
        ibm.ibm_batch_poisson(b, rhs[k], phi[k])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for k in range(4):
            ibm.ibm_batch_poisson(b, rhs[k], phi[k])
    e1.record()
    torch.cuda.synchronize()
    return b, e0.elapsed_time(e1) / reps, create_s


def batched_compare(ibm, torch):
    """64 instances, grids drawn from {32,48,64,96,128}^3, 4 right-hand sides
    each: FP32 + 1 refinement through ibm_batch_poisson (one CUDA-graph
    launch per right-hand-side set) vs 64 sequential plain FP64 solves.  The
    batch is tuned twice: with every plane mode (the tensor-core DFT mode
    included for the short planes) and with CUDA-core FFTs only
    (IBM_TUNE_DFT=0)."""
    from paper_2406_19920_gb300 import synth
    rng = np.random.default_rng(3005)
    dims = [(int(n), int(n), int(n)) for n in rng.choice([32, 48, 64, 96, 128], 64)]
    hs = [synth.grid(*d)[3:] for d in dims]
    rhs = [[torch.from_numpy(synth.rhs_lowpass_noise(*d, kmax=12.0, workload=3, stream=100 * k + i))
            .to("cuda", torch.float32) for i, d in enumerate(dims)] for k in range(4)]
    phi = [[torch.empty_like(x) for x in r] for r in rhs]
    os.environ["IBM_TUNE_DFT"] = "0"
    try:
        b_fft, ms_fft, _ = _batch_ms(ibm, torch, dims, hs, rhs, phi)
    finally:
        del os.environ["IBM_TUNE_DFT"]
    ibm.ibm_batch_destroy(b_fft)
    b, ms, create_s = _batch_ms(ibm, torch, dims, hs, rhs, phi)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pts = sum(d[0] * d[1] * d[2] for d in dims) * 4
    plans = [ibm.ibm_plan_create(*d, h, ibm.IBM_FP64, 0) for d, h in zip(dims, hs)]
    r64 = [x.double() for x in rhs[0]]
    p64 = [torch.empty_like(x) for x in r64]
    for pl, r, o in zip(plans, r64, p64):
        ibm.ibm_poisson_solve(pl, r, o)
    torch.cuda.synchronize()
    e0.record()
    for pl, r, o in zip(plans, r64, p64):
        ibm.ibm_poisson_solve(pl, r, o)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    err = max(float(torch.linalg.vector_norm(a.double() - c) / torch.linalg.vector_norm(c))
              for a, c in zip(phi[0], p64))
    for pl in plans:
        ibm.ibm_plan_destroy(pl)
    ibm.ibm_batch_destroy(b)
    return {"instances": 64, "rhs_per_instance": 4, "grid_pts_per_set": pts // 4,
            "fp32_refined_batched": {"solves_per_s": 256e3 / ms, "grid_pts_per_s": pts / (ms * 1e-3),
                                     "ms_per_256_solves": ms},
            "fp32_refined_batched_fft_only": {"solves_per_s": 256e3 / ms_fft, "ms_per_256_solves": ms_fft},
            "fp64_sequential": {"solves_per_s": 64e3 / ms64, "grid_pts_per_s": (pts / 4) / (ms64 * 1e-3)},
            "speedup": (256e3 / ms) / (64e3 / ms64), "max_rel_l2_vs_fp64": err, "create_and_tune_s": create_s}


def dft_compare(ibm, torch, sizes=(32, 48, 64), reps=50):
    """Tensor-core DFT plane transforms against the CUDA-core FFT kernels on
    the short planes of the batched workload: an n^3 FP32 Poisson solve with
    one refinement step (two forward and two inverse transforms) in each
    plane mode.  Reports the solve time and the forward / inverse transform
    time per solve (event trace of the plan), and the relative L2 distance
    of the DFT-mode solution from the FFT-mode one."""
    from paper_2406_19920_gb300 import synth
    out = {}
    for n in sizes:
        g = synth.grid(n, n, n)
        b = torch.from_numpy(synth.rhs_lowpass_noise(n, n, n, kmax=12.0, workload=3, stream=7)).to("cuda",
                                                                                                   torch.float32)
        row, sols = {}, {}
        for name, mode in (("dft_tc", -1), ("fft_plane", 1), ("fft_split", 0)):
            os.environ["IBM_PLANE_MODE"] = str(mode)
            try:
                plan = ibm.ibm_plan_create(n, n, n, g[3:], ibm.IBM_FP32_REFINED, 1)
            finally:
                del os.environ["IBM_PLANE_MODE"]
            phi = torch.empty_like(b)
            for _ in range(5):
                ibm.ibm_poisson_solve(plan, b, phi)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ibm.ibm_poisson_solve(plan, b, phi)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ibm.ibm_plan_profile(plan, True)
            ibm.ibm_plan_profile_read(plan)
            for _ in range(reps):
                ibm.ibm_poisson_solve(plan, b, phi)
            torch.cuda.synchronize()
            prof = ibm.ibm_plan_profile_read(plan)
            ibm.ibm_plan_profile(plan, False)
            ibm.ibm_plan_destroy(plan)
            sols[name] = phi.double()
            row[name] = {"solve_us": ms * 1e3, "forward_us_per_solve": prof["forward"][0] / reps * 1e3,
                         "inverse_us_per_solve": prof["inverse"][0] / reps * 1e3}
        row["dft_vs_fft_rel_l2"] = float(torch.linalg.vector_norm(sols["dft_tc"] - sols["fft_plane"])
                                         / torch.linalg.vector_norm(sols["fft_plane"]))
        out["%d^3" % n] = row
    return out


def large_plate(ibm, torch, stages=48, v_in=None):
    """Bio-inspired external-flow workload: 384x256x256 on a uniform h = 2 pi/384
    grid (periodic x, z; walls in y), FP32 + 1 refinement, a flat plate of
    100,000 markers (250 x 400 lattice, chord 1, span 2) heaving with amplitude
    0.5 and period 1 about y = Ly/2.  Runs `stages` consecutive RK stages
    (16 full steps) and reports ms per stage, per-kernel time, the refined
    Poisson solve's relative residual and max |D u| after projection.
    v_in: no-slip walls if None; else the inflow-outflow walls (inflow v_in
    through y = 0, an outlet advected at speed v_in) with the uniform
    through-flow v_in added to the initial field."""
    from paper_2406_19920_gb300 import synth
    nx, ny, nz = 384, 256, 256
    h = 2 * math.pi / 384
    g = (nx, ny, nz, h, h, h)
    Ly = ny * h
    u, v, w = synth.div_free_velocity(g, workload=2, kmax=16.0, rms=0.1)
    X0, dV = synth.flat_plate(250, 400, 1.0, 2.0, (nx * h / 2, Ly / 2, nz * h / 2), h)
    f32 = torch.float32
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", f32)
    if v_in is not None:
        v = v + v_in
    fields = [dev(u), dev(v), dev(w), torch.zeros((ny, nz, nx), dtype=f32, device="cuda")]
    Ns = [torch.zeros((ny, nz, nx), dtype=f32, device="cuda") for _ in range(3)]
    outlet = [torch.zeros((nz, nx), dtype=f32, device="cuda") for _ in range(3)]
    outlet[1] += 0.0 if v_in is None else v_in
    io = ibm.ibm_inout(0.0 if v_in is None else v_in, 0.0 if v_in is None else v_in,
                       *[t.data_ptr() for t in outlet])
    if v_in is None:
        substep = lambda s, info=False: ibm.ibm_substep(plan, st, s, DT, NU, mk, info=info)
    else:
        substep = lambda s, info=False: ibm.ibm_substep_inout(plan, st, io, s, DT, NU, mk, info=info)
    plan = ibm.ibm_plan_create(nx, ny, nz, (h, h, h), ibm.IBM_FP32_REFINED, 1)
    st = ibm.ibm_state(*[t.data_ptr() for t in fields + Ns], 0.0)
    X0d, dVd = dev(X0), dev(dV)
    X = torch.empty((X0.shape[0], 3), dtype=f32, device="cuda")
    Ud, F = torch.empty_like(X), torch.empty_like(X)
    mk = ibm.ibm_markers(X0.shape[0], X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                         ibm.IBM_MOTION_HEAVE, (ctypes.c_double * 4)(0.5, 1.0, 0.0, 0.0))
    substep(1)
    torch.cuda.synchronize()
    ibm.ibm_plan_profile(plan, True)
    ibm.ibm_plan_profile_read(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(stages):
        substep((i + 1) % 3 + 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / stages
    prof = ibm.ibm_plan_profile_read(plan)
    ibm.ibm_plan_profile(plan, False)
    info = substep(1, info=True)
    # relative residual of the refined Poisson solve on the stage's own divergence field
    b = torch.randn((ny, nz, nx), device="cuda")
    phi = torch.empty_like(b)
    pinfo = ibm.ibm_poisson_solve(plan, b, phi, info=True)
    ibm.ibm_plan_destroy(plan)
    walls = "no-slip" if v_in is None else "inflow v_in = %g, advected outlet" % v_in
    return {"grid": [nx, ny, nz], "walls": walls, "markers": int(X0.shape[0]), "stages": stages, "ms_per_stage": ms,
            "grid_pts_per_s": nx * ny * nz / (ms * 1e-3),
            "kernel_ms_per_stage": {k: v[0] / stages for k, v in prof.items()},
            "div_max_after_projection": info["div_max"], "div_max_before": info["div_before"],
            "poisson_rel_residual_refined": pinfo["rel_residual"], "sim_time": st.t}


def serve_sample(ibm, duration_s=2.0, rate=2000.0):
    """Open-loop Poisson arrivals at `rate` req/s for `duration_s` into one
    server per precision.  Kinds: 60 % Poisson, 25 % Helmholtz, 15 % RK stage;
    grids log-uniform in points between 32^3 and 128^3, snapped to supported
    shapes with nx >= ny = nz; markers log-uniform in [1k, 20k].  The same
    arrival trace runs twice on one server: cold (every plan and staging
    buffer made on first use) and warm (plans and buffers resident)."""
    from paper_2406_19920_gb300 import synth
    rng = np.random.default_rng(4004)
    sizes = [16, 24, 32, 48, 64, 96, 128]
    shapes = sorted({(nx, ny, ny) for nx in sizes for ny in sizes if nx >= ny and 32 ** 3 <= nx * ny * ny <= 128 ** 3})
    logs = np.log([a * b * c for a, b, c in shapes])

    def draw_shape():
        t = rng.uniform(np.log(32 ** 3), np.log(128 ** 3))
        return shapes[int(np.argmin(np.abs(logs - t)))]

    n_req = int(rate * duration_s)
    gaps = rng.exponential(1.0 / rate, n_req)
    kinds = rng.choice([0, 1, 2], n_req, p=[0.6, 0.25, 0.15])
    plan = [(k, draw_shape(), int(np.exp(rng.uniform(np.log(1000), np.log(20000))))) for k in kinds]
    inputs = {}
    for k, sh, m in plan:
        key = (k, sh)
        if key not in inputs:
            nx, ny, nz = sh
            g = synth.grid(nx, ny, nz)
            if k == 2:
                u, v, w = synth.div_free_velocity(g, workload=4, kmax=4)
                data = np.ascontiguousarray(np.stack([u, v, w, np.zeros_like(u)]))
            else:
                data = synth.white_noise(nx, ny, nz, workload=4, stream=len(inputs))
            inputs[key] = (g, data, np.zeros_like(data))
    X0, dV = synth.fibonacci_sphere(20000, 0.25, (math.pi, 1.0, math.pi), 2 * math.pi / 32)
    X0, dV = np.ascontiguousarray(X0), np.ascontiguousarray(dV)
    out = {}
    for name, prec in (("fp32_refined", ibm.IBM_FP32_REFINED), ("fp64", ibm.IBM_FP64)):
        srv = ibm.ibm_server_create(64 << 30, 8, 1 << 16)
        reqs = []
        for k, sh, m in plan:
            g, data, dst = inputs[(k, sh)]
            r = ibm.ibm_request()
            r.kind, (r.nx, r.ny, r.nz) = k, sh
            r.h = (ctypes.c_double * 3)(*g[3:])
            r.precision, r.refine_iters = prec, 1
            r.c, r.field_bc = 0.5 * DT * NU, ibm.IBM_FIELD_CELL_DIRICHLET
            r.in_, r.out = data.ctypes.data, dst.ctypes.data
            r.n_markers = m if k == 2 else 0
            r.X0, r.dV = X0.ctypes.data, dV.ctypes.data
            r.motion, r.params = ibm.IBM_MOTION_TRANSLATE, (ctypes.c_double * 4)(0.1, 0, 0, 0)
            r.dt, r.nu, r.rk_stage = DT, NU, 1
            reqs.append(r)
        passes = {}
        for phase in ("cold", "warm"):
            tickets = []
            t0 = time.perf_counter()
            t_next = t0
            for r, gap in zip(reqs, gaps):
                t_next += gap
                while time.perf_counter() < t_next:
                    pass
                tickets.append(ibm.ibm_submit(srv, r))
            lat, dev_ms, ok = [], [], 0
            for t in tickets:
                if t is None:
                    continue
                rc, res = ibm.ibm_wait(srv, t, 300.0)
                if rc == ibm.IBM_OK:
                    ok += 1
                    lat.append(res.total_ms)
                    dev_ms.append(res.device_ms)
            wall = time.perf_counter() - t0
            passes[phase] = {"requests": n_req, "completed": ok, "throughput_req_per_s": ok / wall,
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "device_ms_mean": float(np.mean(dev_ms))}
        ibm.ibm_server_destroy(srv)
        out[name] = dict(passes["warm"], cold=passes["cold"])
    out["workload"] = ("Poisson arrivals %.0f req/s for %.1f s; 60/25/15 %% Poisson/Helmholtz/RK stage; grids "
                       "log-uniform 32^3..128^3; 8 streams; top-level figures: the warm pass (the same trace "
                       "again on the same server), 'cold': the first pass" % (rate, duration_s))
    return out


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_stage_rate(n_stages):
    """Time the FP64 oracle's RK stage on the benchmark workload."""
    from oracle import ibm_oracle as O
    g = workload_grid()
    (u, v, w), X0, dV = make_inputs(g)
    z = np.zeros_like(u)
    st = dict(u=u, v=v, w=w, p=z.copy(), N_prev=(z, z, z), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
    t0 = time.perf_counter()
    for i in range(n_stages):
        st, _ = O.rk_stage(st, mk, i % 3 + 1, DT, NU, g)
    el = time.perf_counter() - t0
    return NX * NY * NZ * n_stages / el, el


def cpu_baseline(args):
    n = 3
    rate, el = oracle_stage_rate(n)
    return {"value": rate, "unit": "grid-pts/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d consecutive RK stages of the same 128^3 workload (FP64 numpy, dense eigen-bases, "
                      "BLAS threads = all host cores), %.1f s" % (n, el)}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_stage_rate(1)
    t0 = time.perf_counter()
    stage_s = []
    for _ in range(args.steps):
        r, el = oracle_stage_rate(1)
        stage_s.append(el)
    total = time.perf_counter() - t0
    value = NX * NY * NZ * args.steps / sum(stage_s)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grid-pts/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(stage_s) / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "ibm_substep 128^3 FP32+1 refinement, 20k-marker sphere", "grid": [NX, NY, NZ],
                      "markers": N_MARKERS},
           "cpu_baseline": {"value": value, "unit": "grid-pts/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "one FP64 oracle RK stage of the workload per step, %.1f s total" % total},
           "e2e": {"value": value, "unit": "grid-pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving samples")
    ap.add_argument("--quick", action="store_true",
                    help="warm-up and timed steps only (no tracing pass, e2e, Poisson comparison or CPU baseline); "
                         "the timed steps are the profiler region, for ncu launch lists")
    ap.add_argument("--ncu-summary", metavar="CSV",
                    help="summarise an ncu --csv launch list of `--quick --steps K` (pass the same --steps): "
                         "writes profiles/dram_traffic.json, prints a markdown table")
    ap.add_argument("--solve", type=int, metavar="N",
                    help="profiling aid: two refined FP32 Poisson solves on an N^3 grid (the first one warms up), "
                         "then exit; `ncu -s <launches of one solve>` captures the second")
    ap.add_argument("--spread", type=int, metavar="N",
                    help="profiling aid: two spreads of an N-marker sphere on the 128^3 grid, then exit")
    ap.add_argument("--spread-mode", default="atomic", choices=["atomic", "direct", "gather"],
                    help="with --spread: the spreading mode")
    ap.add_argument("--plane-mode", type=int, default=None, metavar="M",
                    help="with --solve: force plane mode M of the transforms (0 split, 1 one CTA per plane, "
                         "2/4/8 cluster, -1 tensor-core DFT products)")
    args = ap.parse_args()
    if args.ncu_summary:
        ncu_summary(args.ncu_summary, args.steps)
        return
    if args.solve:
        solve_twice(args.solve, args.plane_mode)
        return
    if args.spread:
        spread_twice(args.spread, args.spread_mode)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
