"""Benchmark: the FP32-refined Poisson solve at 256^3 (the metric's headline).

A step is one call of ibm_poisson_solve on a 256^3 grid of the domain
[0,2pi) x [0,2] x [0,2pi] (periodic x, z; homogeneous Neumann walls in y):
forward x/z transforms, the y tridiagonal solves with the FP64 zero mode,
inverse transforms, one FP32 residual (computed inside the correction's
forward x-rows pass) and the correction solve, and the FP64 mean removal.  The right-hand side is seeded zero-mean N(0,1) noise
low-pass filtered to |k| <= 32.  Four right-hand sides and four solutions
rotate across steps (512 MB > 129 MB L2), so every step reads from HBM.

Output: one JSON line (rank 0).  `value` is grid points solved per second
(all ranks) over the untraced timed region (`solves_per_s` beside it),
`e2e` the same through ibm_poisson_solve with host buffers (upload of the
right-hand side and download of the solution inside the timed region),
`roofline` the dominant kernel kind's achieved HBM bandwidth from CUDA
events around each of its launches in an identical second pass,
`roofline_solve` the whole solve against its method bytes, `oracle_error`
the result's relative L2 and max-abs error against the FP64 oracle, and
`cpu_baseline` the oracle's 256^3 solve on the host cores (one thread and
all cores, best of 3).  Extra keys: the FP32 solve without refinement and
the FP64 solve at 256^3, the triply periodic branch, one RK stage at 128^3
(with its oracle error), the heaving-plate stage at 384x256x256 (with its
oracle error), spreading, batched, tensor-core DFT and serving samples.
`--impl reference` times the oracle's solve alone, on the same config.
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
# the headline workload: one refined FP32 Poisson solve at 256^3
HEAD_N = 256
HEAD_REFINE = 1
HEAD_BUFS = 4
HEAD_KMAX = 32.0
WORKLOAD = "ibm_poisson_solve 256^3 FP32 + 1 float-float refinement step"
CONFIG = {"workload": WORKLOAD, "grid": [HEAD_N, HEAD_N, HEAD_N], "domain": "[0,2pi)x[0,2]x[0,2pi]",
          "bc": "periodic x, z; homogeneous Neumann walls in y",
          "rhs": "seeded zero-mean N(0,1) noise low-pass filtered to |k| <= 32",
          "precision": "FP32 fields, FP64 zero mode, nullspace and norms, 1 float-float refinement step",
          "l2": "4 rotating right-hand sides and solutions (512 MB) > 129 MB L2"}
# the RK-stage extra: 128^3, 20k-marker translating sphere
NX = NY = NZ = 128
N_MARKERS = 20000
DT, NU = 1e-3, 1e-2
N_STATES = 4
# sources of each kernel kind per workload (a DRAM-traffic figure taken by ncu
# is reported only while these are unchanged)
KERNEL_SOURCES = {
    "headline": {"forward": ("slab.cu", "fft2.cuh"), "pencil": ("slab.cu", "seg.cuh", "fft2.cuh"),
                 "inverse": ("slab.cu", "fft2.cuh"), "residual": ("slab.cu", "stencil.cuh", "fft2.cuh")},
    "stage": {"forward": ("transforms.cu", "axis.cu", "fft2.cuh"),
              "inverse": ("transforms.cu", "axis.cu", "fft2.cuh"), "pencil": ("pencil.cu", "seg.cuh"),
              "residual": ("stencil.cu",), "explicit": ("substep.cu",), "divergence": ("substep.cu",),
              "project": ("substep.cu",), "interp": ("ibm_kernels.cu",), "spread": ("ibm_kernels.cu",),
              "motion": ("ibm_kernels.cu",)}}
# kernel-name prefix -> kind (the names ncu prints)
KERNEL_KIND = (("k_plane_fwd", "forward"), ("k_rows_fwd_res", "residual"), ("k_rows_fwd", "forward"), ("k_cplane_fwd", "forward"),
               ("k_plane_inv", "inverse"), ("k_rows_inv", "inverse"), ("k_cplane_inv", "inverse"),
               ("k_pencil", "pencil"), ("k_slab", "pencil"), ("k_residual", "residual"), ("k_explicit", "explicit"),
               ("k_divergence", "divergence"), ("k_project", "project"), ("k_interp", "interp"),
               ("k_spread", "spread"), ("k_motion", "motion"))
STAGE_WORKLOAD = "ibm_substep 128^3 FP32+1 refinement, 20k-marker sphere"


def head_grid():
    from paper_2406_19920_gb300 import synth
    return synth.grid(HEAD_N, HEAD_N, HEAD_N)


def head_rhs():
    """The headline right-hand side, FP32 (both arms and the oracle check
    use these same FP32 values)."""
    from paper_2406_19920_gb300 import synth
    return synth.rhs_lowpass_noise(HEAD_N, HEAD_N, HEAD_N, kmax=HEAD_KMAX, workload=1).astype(np.float32)


def workload_grid():
    from paper_2406_19920_gb300 import synth
    return synth.grid(NX, NY, NZ)


def make_inputs(g):
    """Seeded host inputs (FP64) of the 128^3 RK-stage extra."""
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


def source_digest(kind, which="headline"):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[which][kind]:
        with open(os.path.join(ROOT, "paper_2406_19920_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind, which="headline"):
    """DRAM bytes per step of a kernel kind (its launches in one step) from
    the committed single-kernel ncu captures, if the kind's sources are
    unchanged since the capture; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(which, {}).get(kind)
    if not e or e.get("source_sha256_16") != source_digest(kind, which):
        return None
    return e.get("dram_bytes_per_step")


def ncu_counters(csv_path, which, launches_per_step):
    """Records, from a raw-page CSV of a single-kernel ncu capture
    (`ncu -i rep --page raw --csv`), the captured kernel's DRAM bytes per
    launch times its launches per step in profiles/dram_traffic.json under
    `which` ("headline" or "stage") and the kernel's kind."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr, units, data = rows[0], rows[1], rows[2:]
    idx = {h: k for k, h in enumerate(hdr)}
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    per = {}
    for d in data:
        kind = kernel_kind(d[idx["Kernel Name"]])
        b = sum(float(d[idx[m]].replace(",", "")) * scale.get(units[idx[m]], 1.0)
                for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"))
        per.setdefault(kind, []).append(b)
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            out = json.load(f)
    except (OSError, ValueError):
        out = {}
    for kind, vals in per.items():
        out.setdefault(which, {})[kind] = {
            "dram_bytes_per_launch": sum(vals) / len(vals), "launches_per_step": launches_per_step,
            "dram_bytes_per_step": sum(vals) / len(vals) * launches_per_step,
            "source_sha256_16": source_digest(kind, which),
            "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a single-kernel capture (-k, -c <= 3) of "
                    "`bench.py --solve 256`, averaged over the captured launches; the replay flushes caches before a "
                    "launch, not after, so writes still in L2 at the kernel's end are not counted"}
        print(kind, out[which][kind]["dram_bytes_per_launch"])
    with open(p, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def solve_kind_bytes(n, esz=4, refine=HEAD_REFINE, fused=True):
    """Compulsory HBM bytes per Poisson solve on an n^3 grid, per kernel kind.

    pts = n^3 real points; spec = n n (n/2+1) complex entries; a solve with
    `refine` refinement steps transforms 1 + refine right-hand sides.
    forward: read field + write spectrum per transform; pencil: read + write
    spectrum; inverse: read spectrum + write field, plus the read of the
    field the correction is added to; residual: read b and x, write r, or,
    `fused` (the slab path), read b and x and write the correction's
    spectrum (its forward x rows run in the same pass).  The spectrum round
    trip between split x and z passes is not counted (it is not compulsory:
    a plane kernel avoids it)."""
    pts = n ** 3
    spec = n * n * (n // 2 + 1)
    cs = 2 * esz
    sets = 1 + refine
    fwd_sets = 1 if fused else sets
    res = refine * (2 * pts * esz + spec * cs) if fused else refine * 3 * pts * esz
    return {"forward": fwd_sets * (pts * esz + spec * cs), "pencil": sets * 2 * spec * cs,
            "inverse": sets * (spec * cs + pts * esz) + refine * pts * esz, "residual": res}


def slab_path(n, precision_fp32, bc=None, env=None):
    """Whether an n^3 plan takes the fused slab path (the library's default:
    FP32 wall-bounded 256 x 256 (y, z) slabs; IBM_SLAB forces it on or off)."""
    flag = (env or {}).get("IBM_SLAB", os.environ.get("IBM_SLAB"))
    walls = bc is None or bc == 1  # IBM_BC_PXZ_WALL_Y
    if not precision_fp32 or not walls or n not in (64, 128, 256):
        return False
    if flag is not None:
        return flag == "1"
    return n == 256


def algorithmic_bytes(kind, esz=4):
    """Compulsory HBM bytes per step of the 128^3 RK-stage extra, per kernel kind.

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
    """Per-kernel launches, device time per step and share from an ncu --csv
    launch list (gpu__time_duration.sum) of `bench.py --quick --steps K`
    (profiler region = the timed steps); prints a markdown table."""
    import csv
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    agg = {}
    for r in csv.DictReader(lines):
        if r["Metric Name"] != "gpu__time_duration.sum":
            continue
        kind = kernel_kind(r["Kernel Name"])
        if kind is None:
            continue
        short = r["Kernel Name"].replace("void ", "", 1).replace("ibm::", "").split("(")[0]
        a = agg.setdefault((kind, short), {"ids": set(), "ns": 0.0})
        a["ids"].add(r["ID"])
        val = float(r["Metric Value"].replace(",", ""))
        a["ns"] += val * {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6}.get(
            r["Metric Unit"], 1.0)
    total_ns = sum(a["ns"] for a in agg.values())
    print("| kernel | kind | launches/step | us/step | share |")
    print("|---|---|---|---|---|")
    for (kind, name), a in sorted(agg.items(), key=lambda kv: -kv[1]["ns"]):
        print("| %s | %s | %.1f | %.2f | %.1f%% |" % (name, kind, len(a["ids"]) / steps, a["ns"] / 1e3 / steps,
                                                      100 * a["ns"] / total_ns))


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


def clock_verdict(clk, low=0.9):
    """Whether a timed region's clock record passes the timing rules: no
    hardware or thermal slowdown active, and the median SM clock under load
    not stuck well below the maximum with no reason given (a clock lock left
    by another user); a power cap is kept and noted."""
    reasons = clk.get("reasons") or []
    bad = [r for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown") if r in reasons]
    if bad:
        return {"accepted": False, "why": ",".join(bad)}
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm is None or not mx:
        return {"accepted": None, "why": "no clock samples"}
    if sm < low * mx and "sw_power_cap" not in reasons:
        return {"accepted": False, "why": "pinned_low"}
    return {"accepted": True, "why": "sw_power_cap" if "sw_power_cap" in reasons else ""}


def run_gpu(args):
    import torch
    import paper_2406_19920_gb300 as ibm
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    n = HEAD_N
    g = head_grid()
    b32 = head_rhs()
    f32 = torch.float32
    plan = ibm.ibm_plan_create(n, n, n, g[3:], ibm.IBM_FP32_REFINED, HEAD_REFINE)
    rhs = [torch.from_numpy(b32).to("cuda") for _ in range(HEAD_BUFS)]
    phi = [torch.empty_like(r) for r in rhs]
    stream = torch.cuda.current_stream()

    def step(i):
        ibm.ibm_poisson_solve(plan, rhs[i % HEAD_BUFS], phi[i % HEAD_BUFS], stream=stream)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ibm.ibm_plan_check(plan)

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
                              "value": n ** 3 * args.steps * ws / (ms * 1e-3)}), flush=True)
        ibm.ibm_plan_destroy(plan)
        return

    # ---- timed region: K solves, no tracing; clocks sampled throughout ----
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
    pts = n ** 3
    value = job_throughput(pts * args.steps, ws, total_ms)
    ms_step = total_ms / args.steps

    # ---- identical pass with CUDA events around every kernel kind (roofline) ----
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
    info = ibm.ibm_poisson_solve(plan, rhs[0], phi[0], info=True)
    ibm.ibm_plan_check(plan)

    # ---- accuracy of the timed result against the FP64 oracle ----
    got = phi[0].double().cpu().numpy()
    oracle_error = None
    if rank == 0 and not args.no_oracle:
        from oracle import ibm_oracle as O
        t0 = time.perf_counter()
        ref, _ = O.poisson_solve(b32.astype(np.float64), g)
        d = got - ref
        oracle_error = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
                        "rel_max_abs": float(np.abs(d).max() / np.abs(ref).max()),
                        "target": 1e-6, "oracle_s": time.perf_counter() - t0,
                        "what": "FP32-refined GPU solution against the FP64 oracle's solution of the same FP32 "
                                "right-hand side (dense eigen-bases, mean-zero nullspace)"}
        del ref, d

    # ---- end to end: host buffers, copies inside the timed region ----
    # Every step uploads its right-hand side from pinned host memory, solves
    # through ibm_poisson_solve and reads the solution back.  NB device
    # buffer sets rotate: step i's upload runs on an upload stream while
    # earlier steps solve, its download on a download stream while later
    # steps solve (the solves stay in order on the compute stream).  With two
    # sets the period is (upload + solve + download) / 2, as step i's upload
    # waits for step i-2's download; with NB >= 3 it is bounded by the slower
    # copy direction alone.
    NB = len(rhs)
    host_in = torch.from_numpy(b32).pin_memory()
    host_out = [torch.empty((n, n, n), dtype=f32).pin_memory() for _ in range(NB)]
    h2d = host_in.numel() * host_in.element_size()
    d2h = host_out[0].numel() * host_out[0].element_size()
    e2e_steps = max(3, min(args.steps, 40))
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(NB)]
    ev_done = [torch.cuda.Event() for _ in range(NB)]
    ev_down = [torch.cuda.Event() for _ in range(NB)]
    barrier()
    e0.record()
    s_up.wait_stream(stream)
    s_down.wait_stream(stream)
    for i in range(e2e_steps):
        bi = i % NB
        with torch.cuda.stream(s_up):
            if i >= NB:
                s_up.wait_event(ev_down[bi])  # buffer bi's previous solution is out
            rhs[bi].copy_(host_in, non_blocking=True)
            ev_up[bi].record(s_up)
        stream.wait_event(ev_up[bi])
        ibm.ibm_poisson_solve(plan, rhs[bi], phi[bi], stream=stream)
        ev_done[bi].record(stream)
        with torch.cuda.stream(s_down):
            s_down.wait_event(ev_done[bi])
            host_out[bi].copy_(phi[bi], non_blocking=True)
            ev_down[bi].record(s_down)
    stream.wait_stream(s_up)
    stream.wait_stream(s_down)
    e1.record()
    barrier()
    e2e_ms = job_ms(e0.elapsed_time(e1), dist, "cuda")
    e2e_value = job_throughput(pts * e2e_steps, ws, e2e_ms)
    e2e_same = bool(np.array_equal(host_out[(e2e_steps - 1) % NB].numpy(), got.astype(np.float32)))
    ibm.ibm_plan_destroy(plan)
    del rhs, phi, host_in, host_out
    torch.cuda.empty_cache()

    # ---- roofline: the dominant kernel kind, and the whole solve ----
    fused = slab_path(n, True)
    kb = solve_kind_bytes(n, fused=fused)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_launches = kinds[dom]
    dom_step_ms = dom_ms / args.steps
    peak, peak_src = measured_peak()
    alg = kb[dom]
    achieved = alg / (dom_step_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom, "headline")
    launches = sum(c for _, c in kinds.values())
    mb = method_bytes(n, 4, HEAD_REFINE, fused)
    clocks = clk.summary()
    clocks.update(clock_verdict(clocks))
    cfg = dict(CONFIG, parallelism="replicas" if ws > 1 else "1 GPU")
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "grid-pts/s",
        "solves_per_s": value / pts,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": cfg,
        "e2e": {"value": e2e_value, "unit": "grid-pts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "solves_per_s": e2e_value / pts, "result_matches_device_run": e2e_same,
                "overlap": "%d device buffer sets: step i's upload and download overlap other steps' solves "
                           "and each other (separate upload, compute and download streams)" % NB},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                     "per": "step (all launches of the kind in one refined solve)",
                     "algorithmic_bytes": alg, "ms_per_step": dom_step_ms,
                     "launches_per_step": dom_launches / args.steps, "avg_launch_ms": dom_ms / dom_launches},
        "roofline_solve": {"bound": "hbm", "method_bytes": mb, "achieved": mb / (ms_step * 1e-3) / 1e9,
                           "peak": peak, "unit": "GB/s", "frac": mb / (ms_step * 1e-3) / 1e9 / peak,
                           "peak_source": peak_src, "target_frac": 0.6,
                           "method": "forward, pencil and inverse passes each read and write the field once "
                                     "(24 B/pt FP32) per transform set; the refinement step adds "
                                     + ("the residual fused with the correction's forward x rows (reads b and x, "
                                        "writes the spectrum: 12 B/pt), its pencil and inverse passes and the read "
                                        "of the corrected field (4 B/pt)" if fused else
                                        "the residual pass (12 B/pt), a second set and the read of the corrected "
                                        "field (4 B/pt)")},
        "oracle_error": oracle_error,
        "info": {k: info[k] for k in ("rel_residual", "removed_mean", "refine_iters")},
        "phase_ms_per_solve": {k: v for k, v in info["phase_ms"].items() if v > 0},
        "kernels_ms_per_step": {k: kinds[k][0] / args.steps for k in kinds},
        "launches_per_step": {k: kinds[k][1] / args.steps for k in kinds},
        "p50_ms": float(np.percentile(step_ms, 50)),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "value_traced": pts * args.steps * ws / (traced_ms * 1e-3),
        "clocks": clocks,
        "timed_region_s": t_host1 - t_host0,
    }

    # ---- extras (outside the timed region) ----
    if not args.no_extras:
        # the split x / z passes (IBM_SLAB=0) beside the fused slab path, same solves
        out["poisson_256"] = poisson_compare(ibm, torch, 256, (("fp32", ibm.IBM_FP32_REFINED, 0),
                                                               ("fp32_refined", ibm.IBM_FP32_REFINED, 1),
                                                               ("fp32_split", ibm.IBM_FP32_REFINED, 0,
                                                                {"IBM_SLAB": "0"}),
                                                               ("fp32_refined_split", ibm.IBM_FP32_REFINED, 1,
                                                                {"IBM_SLAB": "0"}),
                                                               ("fp64", ibm.IBM_FP64, 0)), nb=4, K=20,
                                             oracle=rank == 0 and not args.no_oracle)
        # triply periodic branch (y-FFT pencil step instead of the Thomas sweep)
        out["poisson_256"]["triply_periodic"] = poisson_compare(
            ibm, torch, 256, (("fp32", ibm.IBM_FP32_REFINED, 0), ("fp64", ibm.IBM_FP64, 0)), nb=4, K=20,
            bc=ibm.IBM_BC_TRIPLY_PERIODIC)
        out["poisson_128"] = poisson_compare(ibm, torch, NX, (("fp32_refined", ibm.IBM_FP32_REFINED, 1),
                                                              ("fp32_refined_split", ibm.IBM_FP32_REFINED, 1,
                                                               {"IBM_SLAB": "0"}),
                                                              ("fp64", ibm.IBM_FP64, 0)))
        out["stage_128"] = stage_128(ibm, torch, args, oracle=rank == 0 and not args.no_oracle)
        out["spreading"] = spread_compare(ibm, torch)
        out["batched"] = batched_compare(ibm, torch)
        out["dft_tensor_core"] = dft_compare(ibm, torch)
        out["serving"] = serve_sample(ibm, torch, duration_s=args.serve_seconds, oracle=rank == 0 and not args.no_oracle)
        out["large_plate"] = large_plate(ibm, torch, oracle=rank == 0 and not args.no_oracle)
        out["large_plate_inflow"] = large_plate(ibm, torch, v_in=1.0)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def quick_stage(args):
    """Profiling aid: `args.warmup` then `args.steps` RK stages of the 128^3
    workload (20k-marker sphere, four rotating states), the timed stages
    inside cudaProfilerStart/Stop (`ncu --profile-from-start off`)."""
    import torch
    import paper_2406_19920_gb300 as ibm
    g = workload_grid()
    (u, v, w), X0, dV = make_inputs(g)
    f32 = torch.float32
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", f32)
    plan = ibm.ibm_plan_create(NX, NY, NZ, g[3:], ibm.IBM_FP32_REFINED, 1)
    states, keep = [], []
    for _ in range(N_STATES):
        f = [dev(u), dev(v), dev(w)] + [torch.zeros((NY, NZ, NX), dtype=f32, device="cuda") for _ in range(4)]
        states.append(ibm.ibm_state(*[t.data_ptr() for t in f], 0.0))
        keep.append(f)
    X0d, dVd = dev(X0), dev(dV)
    X = torch.empty((N_MARKERS, 3), dtype=f32, device="cuda")
    Ud, F = torch.empty_like(X), torch.empty_like(X)
    mk = ibm.ibm_markers(N_MARKERS, X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                         ibm.IBM_MOTION_TRANSLATE, (ctypes.c_double * 4)(0.1, 0.0, 0.0, 0.0))
    for i in range(args.warmup):
        ibm.ibm_substep(plan, states[i % N_STATES], (i // N_STATES) % 3 + 1, DT, NU, mk)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    for i in range(args.steps):
        j = args.warmup + i
        ibm.ibm_substep(plan, states[j % N_STATES], (j // N_STATES) % 3 + 1, DT, NU, mk)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ibm.ibm_plan_check(plan)
    ibm.ibm_plan_destroy(plan)
    print(json.dumps({"quick_stage": True, "steps": args.steps}))


def stage_128(ibm, torch, args, oracle=True):
    """One RK stage (ibm_substep, every row of the path) at 128^3 with FP32
    fields and one refinement step, a 20,000-marker Fibonacci sphere (radius
    0.25, centre (pi, 1, pi)) translating at 0.1 in x, from a seeded
    discretely divergence-free velocity with energy ~ k^-5/3 (k <= 16).
    Four independent states rotate (4 x 56 MB > 129 MB L2).  Reports grid
    points per second, the dominant kernel kind's HBM roofline from an
    event-traced pass, and the stage's per-field error against the oracle's
    rk_stage from the same FP32 inputs."""
    g = workload_grid()
    (u, v, w), X0, dV = make_inputs(g)
    f32 = torch.float32
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", f32)
    plan = ibm.ibm_plan_create(NX, NY, NZ, g[3:], ibm.IBM_FP32_REFINED, 1)
    states, keep = [], []
    for s in range(N_STATES):
        fields = [dev(u), dev(v), dev(w), torch.zeros((NY, NZ, NX), dtype=f32, device="cuda")]
        Ns = [torch.zeros((NY, NZ, NX), dtype=f32, device="cuda") for _ in range(3)]
        states.append(ibm.ibm_state(*[t.data_ptr() for t in fields + Ns], 0.0))
        keep.append((fields, Ns))
    X0d, dVd = dev(X0), dev(dV)
    X = torch.empty((N_MARKERS, 3), dtype=f32, device="cuda")
    Ud, F = torch.empty_like(X), torch.empty_like(X)
    params = (ctypes.c_double * 4)(0.1, 0.0, 0.0, 0.0)
    mk = ibm.ibm_markers(N_MARKERS, X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                         ibm.IBM_MOTION_TRANSLATE, params)
    stream = torch.cuda.current_stream()
    steps = 200

    def step(i):
        ibm.ibm_substep(plan, states[i % N_STATES], (i // N_STATES) % 3 + 1, DT, NU, mk, stream=stream)

    # the oracle comparison: stage 1 of state 1 from the initial fields (run first)
    err = None
    if oracle:
        from oracle import ibm_oracle as O
        ibm.ibm_substep(plan, states[1], 1, DT, NU, mk, stream=stream)
        torch.cuda.synchronize()
        fields, Ns = keep[1]
        got = {k: t.double().cpu().numpy() for k, t in zip("uvwp", fields)}
        got["F"] = F.double().cpu().numpy()
        c32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
        z = np.zeros_like(u)
        st = dict(u=c32(u), v=c32(v), w=c32(w), p=z.copy(), N_prev=(z, z, z), t=0.0)
        mko = dict(X0=c32(X0), dV=c32(dV), kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
        t0 = time.perf_counter()
        ref, rinfo = O.rk_stage(st, mko, 1, DT, NU, g)
        ref["F"] = rinfo["F"]
        err = {"oracle_s": time.perf_counter() - t0}
        for k in ("u", "v", "w", "p", "F"):
            d = got[k] - ref[k]
            err[k] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref[k])),
                      "rel_max_abs": float(np.abs(d).max() / np.abs(ref[k]).max())}
        # back to the initial state for the timed steps
        for t, a in zip(fields, (u, v, w, z)):
            t.copy_(dev(a))
        for t in Ns:
            t.zero_()
        states[1].t = 0.0
    for i in range(5):
        step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        step(5 + i)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ibm.ibm_plan_profile(plan, True)
    ibm.ibm_plan_profile_read(plan)
    for i in range(steps):
        step(5 + steps + i)
    prof = ibm.ibm_plan_profile_read(plan)
    ibm.ibm_plan_profile(plan, False)
    info = ibm.ibm_substep(plan, states[0], 1, DT, NU, mk, info=True)
    ibm.ibm_plan_destroy(plan)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_step_ms = kinds[dom][0] / steps
    peak, peak_src = measured_peak()
    alg = algorithmic_bytes(dom)
    achieved = alg / (dom_step_ms * 1e-3) / 1e9
    return {"workload": STAGE_WORKLOAD, "ms_per_stage": ms, "grid_pts_per_s": NX * NY * NZ / (ms * 1e-3),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src, "algorithmic_bytes": alg,
                         "ms_per_step": dom_step_ms, "traffic": ncu_traffic(dom, "stage")},
            "kernels_ms_per_stage": {k: kinds[k][0] / steps for k in kinds},
            "launches_per_stage": {k: kinds[k][1] / steps for k in kinds},
            "phase_ms_one_stage": {k: v for k, v in info["phase_ms"].items() if v > 0},
            "oracle_error": err, "tolerance_per_field": 3e-6,
            "stage_info": {k: info[k] for k in ("div_max", "div_before", "removed_mean")}}


def method_bytes(n, precision_bytes, refine, fused=False):
    """Compulsory HBM bytes of one Poisson solve on an n^3 grid: forward
    (read field, write spectrum), pencil (read + write spectrum), inverse
    (read spectrum, write field); a refinement step adds the residual (read
    b and x, write r), a second solve and the read of the updated field.
    `fused` (the slab path): the residual and the correction's forward x
    rows are one pass (read b and x, write the spectrum)."""
    pts = n ** 3
    spec = n * n * (n // 2 + 1)
    s = precision_bytes
    solve = pts * s + 2 * spec * s + 2 * 2 * spec * s + 2 * spec * s + pts * s
    if fused:
        return solve + refine * (2 * pts * s + 2 * spec * s + 2 * 2 * spec * s + 2 * spec * s + 2 * pts * s)
    return solve + refine * (3 * pts * s + solve + pts * s)


def poisson_compare(ibm, torch, n, variants, nb=16, K=40, bc=None, oracle=False):
    """Standalone Poisson solves on an n^3 grid ([0,2pi)x[0,2]x[0,2pi],
    low-passed noise right-hand side): solves/s, p50/p99 latency, and the
    achieved fraction of the measured HBM bandwidth for the solve's method
    bytes; relative L2 of each FP32 result against the FP64 GPU result and,
    with `oracle`, every result's relative L2 and max-abs error against the
    FP64 oracle (the FP32 right-hand side's values on both sides)."""
    from paper_2406_19920_gb300 import synth
    g = synth.grid(n, n, n)
    b = synth.rhs_lowpass_noise(n, n, n, kmax=min(32.0, n / 4), workload=1).astype(np.float32).astype(np.float64)
    res = {}
    outs = {}
    for variant in variants:
        name, prec, ref = variant[:3]
        env = variant[3] if len(variant) > 3 else {}
        dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
        old = {k: os.environ.get(k) for k in env}
        os.environ.update(env)
        try:
            plan = ibm.ibm_plan_create(n, n, n, g[3:], prec, ref, bc=bc if bc is not None else ibm.IBM_BC_PXZ_WALL_Y)
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
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
        fused = dt == torch.float32 and ref > 0 and slab_path(n, True, bc, env)
        mb = method_bytes(n, 4 if dt == torch.float32 else 8, ref if dt == torch.float32 else 0, fused)
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
    if oracle:
        from oracle import ibm_oracle as O
        ref, _ = O.poisson_solve(b, g)
        for name in outs:
            d = outs[name] - ref
            res[name]["oracle_rel_l2"] = float(np.linalg.norm(d) / np.linalg.norm(ref))
            res[name]["oracle_rel_max_abs"] = float(np.abs(d).max() / np.abs(ref).max())
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
    stage = batched_stage(ibm, torch, b, dims, hs)
    ibm.ibm_batch_destroy(b)
    return {"instances": 64, "rhs_per_instance": 4, "grid_pts_per_set": pts // 4, "rk_stage_with_markers": stage,
            "fp32_refined_batched": {"solves_per_s": 256e3 / ms, "grid_pts_per_s": pts / (ms * 1e-3),
                                     "ms_per_256_solves": ms},
            "fp32_refined_batched_fft_only": {"solves_per_s": 256e3 / ms_fft, "ms_per_256_solves": ms_fft},
            "fp64_sequential": {"solves_per_s": 64e3 / ms64, "grid_pts_per_s": (pts / 4) / (ms64 * 1e-3)},
            "speedup": (256e3 / ms) / (64e3 / ms64), "max_rel_l2_vs_fp64": err, "create_and_tune_s": create_s}


def batched_stage(ibm, torch, b, dims, hs, reps=6):
    """The batched workload's instances with their marker spheres: each of the
    64 instances gets a still Fibonacci sphere of radius 0.25 with a marker
    count drawn uniformly from [500, 8000] and one RK stage (ibm_substep:
    explicit terms, interpolation, force and spreading on its sphere, three
    Helmholtz and one refined Poisson solve, projection) -- all 64 stages as
    one graph launch (ibm_batch_substep, replayed) against the same stages
    run one instance after another (FP32 + refinement, and plain FP64).
    Reports stages/s, grid points/s and the first instance's stage against
    the FP64 oracle."""
    from paper_2406_19920_gb300 import synth
    rng = np.random.default_rng(3006)
    counts = [int(c) for c in rng.integers(500, 8001, len(dims))]
    pts = sum(d[0] * d[1] * d[2] for d in dims)
    out = {"markers_per_instance": [min(counts), max(counts)], "markers_total": sum(counts)}
    keep = []

    def make(prec, i, d, m):
        g = synth.grid(*d)
        dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
        u, v, w = synth.div_free_velocity(g, workload=90 + i % 8, kmax=min(d) / 4)
        X0, dV = synth.fibonacci_sphere(m, 0.25, (math.pi, 1.0, math.pi), g[3])
        f = [torch.from_numpy(a).to("cuda", dt) for a in (u, v, w, np.zeros_like(u))]
        f += [torch.zeros(u.shape, dtype=dt, device="cuda") for _ in range(3)]
        Xd, dVd = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt) for a in (X0, dV))
        X, Ud, F = (torch.empty((m, 3), dtype=dt, device="cuda") for _ in range(3))
        keep.append((f, Xd, dVd, X, Ud, F))
        st = ibm.ibm_state(*[t.data_ptr() for t in f], 0.0)
        mk = ibm.ibm_markers(m, Xd.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                             ibm.IBM_MOTION_STATIC, (ctypes.c_double * 4)(0, 0, 0, 0))
        return st, mk, (u, v, w, X0, dV, g)

    inst = [make(ibm.IBM_FP32_REFINED, i, d, m) for i, (d, m) in enumerate(zip(dims, counts))]
    states, mks = [x[0] for x in inst], [x[1] for x in inst]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ibm.ibm_batch_substep(b, states, mks, 1, DT, NU)  # capture
    ibm.ibm_batch_substep(b, states, mks, 1, DT, NU)  # replay
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        ibm.ibm_batch_substep(b, states, mks, 1, DT, NU)
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / reps
    out["fp32_refined_batched"] = {"ms_per_64_stages": ms_batch, "stages_per_s": 64e3 / ms_batch,
                                   "grid_pts_per_s": pts / (ms_batch * 1e-3)}
    for name, prec in (("fp32_refined_sequential", ibm.IBM_FP32_REFINED), ("fp64_sequential", ibm.IBM_FP64)):
        plans = [ibm.ibm_plan_create(*d, h, prec, 1 if prec == ibm.IBM_FP32_REFINED else 0) for d, h in zip(dims, hs)]
        seq = inst if prec == ibm.IBM_FP32_REFINED else [make(prec, i, d, m) for i, (d, m) in
                                                         enumerate(zip(dims, counts))]
        for pl, x in zip(plans, seq):
            ibm.ibm_substep(pl, x[0], 1, DT, NU, x[1])
        torch.cuda.synchronize()
        e0.record()
        for _ in range(2):
            for pl, x in zip(plans, seq):
                ibm.ibm_substep(pl, x[0], 1, DT, NU, x[1])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        out[name] = {"ms_per_64_stages": ms, "stages_per_s": 64e3 / ms, "grid_pts_per_s": pts / (ms * 1e-3)}
        for pl in plans:
            ibm.ibm_plan_destroy(pl)
    out["speedup_batched_fp32_over_sequential_fp64"] = out["fp64_sequential"]["ms_per_64_stages"] / ms_batch
    # the first instance, one fresh batched stage, against the oracle
    from oracle import ibm_oracle as O
    solo = ibm.ibm_batch_create([dims[0]], [hs[0]], ibm.IBM_FP32_REFINED, 1)
    try:
        st, mk, (u, v, w, X0, dV, g) = make(ibm.IBM_FP32_REFINED, 0, dims[0], counts[0])
        ibm.ibm_batch_substep(solo, [st], [mk], 1, DT, NU)
        torch.cuda.synchronize()
        f = keep[-1][0]
        c32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
        z = np.zeros_like(u)
        ref, _ = O.rk_stage(dict(u=c32(u), v=c32(v), w=c32(w), p=z.copy(), N_prev=(z, z, z), t=0.0),
                            dict(X0=c32(X0), dV=c32(dV), kind=O.MOTION_STATIC, params=()), 1, DT, NU, g)
        out["oracle_error_instance0"] = {
            k: {"rel_l2": float(np.linalg.norm(f[c].double().cpu().numpy() - ref[k]) / np.linalg.norm(ref[k])),
                "rel_max_abs": float(np.abs(f[c].double().cpu().numpy() - ref[k]).max() / np.abs(ref[k]).max())}
            for c, k in enumerate("uvwp")}
        out["oracle_grid"] = list(dims[0])
    finally:
        ibm.ibm_batch_destroy(solo)
    del keep
    return out


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


def large_plate(ibm, torch, stages=48, v_in=None, oracle=False):
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
    err = None
    if oracle:
        # one stage from the initial fields on both sides, field by field
        from oracle import ibm_oracle as O
        st.t = 0.0
        substep(1)
        torch.cuda.synchronize()
        got = {k: t.double().cpu().numpy() for k, t in zip("uvwp", fields)}
        got["F"] = F.double().cpu().numpy()
        c32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
        z = np.zeros((ny, nz, nx))
        ost = dict(u=c32(u), v=c32(v), w=c32(w), p=z.copy(), N_prev=(z, z, z), t=0.0)
        mko = dict(X0=c32(X0), dV=c32(dV), kind=O.MOTION_HEAVE, params=(0.5, 1.0))
        t0 = time.perf_counter()
        ref, rinfo = O.rk_stage(ost, mko, 1, DT, NU, g)
        ref["F"] = rinfo["F"]
        err = {"oracle_s": time.perf_counter() - t0, "stage": 1}
        for k in ("u", "v", "w", "p", "F"):
            d = got[k] - ref[k]
            err[k] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref[k])),
                      "rel_max_abs": float(np.abs(d).max() / np.abs(ref[k]).max())}
        del ref, rinfo, got
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
            "phase_ms_one_stage": {k: v for k, v in info["phase_ms"].items() if v > 0},
            "poisson_rel_residual_refined": pinfo["rel_residual"], "sim_time": st.t, "oracle_error": err}


SERVE_SIZES = (32, 48, 64, 96, 128, 192, 256, 384)
SERVE_MARKERS = (1000, 2000, 5000, 10000, 20000, 50000, 100000)


def serve_trace(seed, duration_s, rate):
    """The request trace of the serving workload: Poisson arrivals at `rate`
    per second for `duration_s`; kinds 60 % Poisson, 25 % Helmholtz, 15 % RK
    stage; grid points log-uniform between 32^3 and 384 x 256 x 256, snapped
    to the nearest supported shape (nx >= ny = nz, lengths 2^a 3^b); marker
    counts log-uniform in [1k, 100k], snapped to a precomputed sphere size.
    Returns [(arrival offset s, kind, shape, markers)]."""
    rng = np.random.default_rng(seed)
    lo, hi = 32 ** 3, 384 * 256 * 256
    shapes = sorted({(nx, ny, ny) for nx in SERVE_SIZES for ny in SERVE_SIZES if nx >= ny and lo <= nx * ny * ny <= hi})
    logs = np.log([a * b * c for a, b, c in shapes])
    mlog = np.log(SERVE_MARKERS)
    n = int(rng.poisson(rate * duration_s))
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    kinds = rng.choice([0, 1, 2], n, p=[0.6, 0.25, 0.15])
    pts = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    mk = np.exp(rng.uniform(np.log(1000), np.log(100000), n))
    out = []
    for k in range(n):
        sh = shapes[int(np.argmin(np.abs(logs - np.log(pts[k]))))]
        m = SERVE_MARKERS[int(np.argmin(np.abs(mlog - np.log(mk[k]))))] if kinds[k] == 2 else 0
        out.append((float(t[k]), int(kinds[k]), sh, m))
    return out


class ServeInputs:
    """Device-resident inputs of the serving workload in one precision: per
    (kind, shape) one input and a ring of outputs (requests of one shape
    cycle through the ring), and Fibonacci spheres of every marker count
    (radius 0.25, centre (pi, 1, pi))."""

    RING = 4

    @staticmethod
    def host_data(keys):
        """Seeded host inputs (FP64) per (kind, shape) and the spheres."""
        from paper_2406_19920_gb300 import synth
        data = {}
        for kind, sh in sorted(keys):
            nx, ny, nz = sh
            g = synth.grid(nx, ny, nz)
            if kind == 2:
                u, v, w = synth.div_free_velocity(g, workload=4, kmax=4)
                x = np.stack([u, v, w, np.zeros_like(u)])
            else:
                x = synth.white_noise(nx, ny, nz, workload=4, stream=kind)
            data[(kind, sh)] = (g, np.ascontiguousarray(x))
        spheres = {m: synth.fibonacci_sphere(m, 0.25, (math.pi, 1.0, math.pi), 2 * math.pi / 32)
                   for m in SERVE_MARKERS}
        return data, spheres

    def __init__(self, ibm, torch, prec, host):
        self.ibm, self.torch, self.prec = ibm, torch, prec
        self.dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
        self.fields, self.next = {}, {}
        data, spheres = host
        for key, (g, x) in data.items():
            din = torch.from_numpy(x).to("cuda", self.dt)
            self.fields[key] = (g, din, [torch.empty_like(din) for _ in range(self.RING)])
            self.next[key] = 0
        self.spheres = {m: (torch.from_numpy(np.ascontiguousarray(X0)).to("cuda", self.dt),
                            torch.from_numpy(np.ascontiguousarray(dV)).to("cuda", self.dt))
                        for m, (X0, dV) in spheres.items()}

    def request(self, kind, sh, m, out=None):
        ibm = self.ibm
        g, din, ring = self.fields[(kind, sh)]
        if out is None:
            out = ring[self.next[(kind, sh)] % self.RING]
            self.next[(kind, sh)] += 1
        r = ibm.ibm_request()
        r.kind, (r.nx, r.ny, r.nz) = kind, sh
        r.h = (ctypes.c_double * 3)(*g[3:])
        r.precision, r.refine_iters = self.prec, 1
        r.c, r.field_bc = 0.5 * DT * NU, ibm.IBM_FIELD_CELL_DIRICHLET
        r.in_, r.out, r.data = din.data_ptr(), out.data_ptr(), ibm.IBM_DATA_DEVICE
        r.n_markers = m
        if m:
            X0, dV = self.spheres[m]
            r.X0, r.dV = X0.data_ptr(), dV.data_ptr()
        r.motion, r.params = ibm.IBM_MOTION_TRANSLATE, (ctypes.c_double * 4)(0.1, 0, 0, 0)
        r.dt, r.nu, r.rk_stage = DT, NU, 1
        return r


def serve_run(ibm, srv, inputs, trace, checks=()):
    """Submits `trace` open loop (busy-waiting for each arrival time) and
    waits for every request; `checks` = [(index, out tensor)] gives some
    requests private outputs.  Returns latency and throughput figures."""
    chk = dict(checks)
    reqs = [inputs.request(k, sh, m, chk.get(i)) for i, (_, k, sh, m) in enumerate(trace)]
    tickets = []
    t0 = time.perf_counter()
    for (t_arr, _, _, _), r in zip(trace, reqs):
        while time.perf_counter() - t0 < t_arr:
            pass
        tickets.append(ibm.ibm_submit(srv, r))
    submit_s = time.perf_counter() - t0
    lat, dev_ms, ok, failed = [], [], 0, 0
    for t in tickets:
        if t is None:
            failed += 1
            continue
        rc, res = ibm.ibm_wait(srv, t, 600.0)
        if rc == ibm.IBM_OK:
            ok += 1
            lat.append(res.total_ms)
            dev_ms.append(res.device_ms)
        else:
            failed += 1
    wall = time.perf_counter() - t0
    return {"requests": len(trace), "completed": ok, "failed_or_rejected": failed, "offered_req_per_s":
            len(trace) / max(trace[-1][0], 1e-9) if trace else 0.0, "throughput_req_per_s": ok / wall,
            "wall_s": wall, "submit_s": submit_s,
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "device_ms_mean": float(np.mean(dev_ms)) if dev_ms else None}


def serve_oracle_checks(ibm, torch, inputs, outs):
    """Relative L2 and max-abs errors of sampled results against the FP64
    oracle (the request's own input values in the plan precision)."""
    from oracle import ibm_oracle as O
    res = []
    for (kind, sh, m), out in outs:
        g, din, _ = inputs.fields[(kind, sh)]
        x = din.double().cpu().numpy()
        if kind == 0:
            ref, _ = O.poisson_solve(x, g)
            refs = [ref]
            got = [out.double().cpu().numpy()]
        elif kind == 1:
            refs = [O.helmholtz_solve(x, g, 0.5 * DT * NU, O.CELL_DIRICHLET)]
            got = [out.double().cpu().numpy()]
        else:
            X0, dV = (a.double().cpu().numpy() for a in inputs.spheres[m])
            z = np.zeros_like(x[0])
            st = dict(u=x[0], v=x[1], w=x[2], p=x[3], N_prev=(z, z, z), t=0.0)
            mko = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
            ref, _ = O.rk_stage(st, mko, 1, DT, NU, g)
            refs = [ref[k] for k in ("u", "v", "w", "p")]
            o = out.double().cpu().numpy()
            got = [o[c] for c in range(4)]
        l2 = max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(got, refs))
        mx = max(float(np.abs(a - b).max() / np.abs(b).max()) for a, b in zip(got, refs))
        res.append({"kind": ("poisson", "helmholtz", "rk_stage")[kind], "grid": list(sh), "markers": m,
                    "rel_l2": l2, "rel_max_abs": mx})
    return res


def serve_sample(ibm, torch, duration_s=60.0, duration_fp64_s=10.0, rate=2000.0, oracle=True):
    """The serving workload: Poisson arrivals at 2000 req/s; 60 % Poisson,
    25 % Helmholtz, 15 % RK stage; grids log-uniform in points from 32^3 to
    384 x 256 x 256; spheres of 1k-100k markers; requests carry device data
    in the plan precision (IBM_DATA_DEVICE) into one server per precision (8
    streams, resident plans).  Every (kind, shape) of the trace is served
    once first (plans and slot buffers made); then the timed trace runs,
    `duration_s` for FP32 with one refinement step and `duration_fp64_s`
    for plain FP64 (whose capacity is below the offered rate), followed by
    4-second runs at rising rates: the sustainable rate is the highest one
    whose requests all complete at >= 95 % of the offered rate with p99 <=
    20 ms.  A sample of results (one of each kind, the largest grid among
    them) is checked against the FP64 oracle."""
    trace = serve_trace(4004, duration_s, rate)
    keys = {(k, sh) for _, k, sh, _ in trace}
    samples = [(0, (384, 256, 256), 0), (1, (128, 64, 64), 0), (2, (64, 32, 32), 1000), (0, (48, 48, 48), 0)]
    keys |= {(k, sh) for k, sh, _ in samples}
    out = {"workload": "Poisson arrivals %.0f req/s; 60/25/15 %% Poisson/Helmholtz/RK stage; grids log-uniform in "
                       "points 32^3 .. 384x256x256 (%d shapes); markers 1k..100k; device data in the plan precision; "
                       "8 streams; %.0f s FP32-refined, %.0f s FP64" % (rate, len({sh for _, sh in keys}), duration_s,
                                                                     duration_fp64_s)}
    host = ServeInputs.host_data(keys)
    for name, prec, dur, rates in (("fp32_refined", ibm.IBM_FP32_REFINED, duration_s, (4000.0, 8000.0, 16000.0)),
                                   ("fp64", ibm.IBM_FP64, duration_fp64_s, (250.0, 500.0, 1000.0))):
        inputs = ServeInputs(ibm, torch, prec, host)
        srv = ibm.ibm_server_create(96 << 30, 8, 1 << 18)
        try:
            warm = [(0.0, k, sh, (1000 if k == 2 else 0)) for k, sh in sorted(keys)]
            serve_run(ibm, srv, inputs, warm)
            tr = [x for x in trace if x[0] < dur]
            priv = {}
            for j, (k, sh, m) in enumerate(samples):  # private outputs for the checked requests
                idx = (j + 1) * len(tr) // (len(samples) + 1)
                tr[idx] = (tr[idx][0], k, sh, m)
                priv[idx] = ((k, sh, m), torch.empty_like(inputs.fields[(k, sh)][1]))
            row = serve_run(ibm, srv, inputs, tr, [(i, o) for i, (_, o) in priv.items()])
            if oracle:
                row["oracle_check"] = serve_oracle_checks(ibm, torch, inputs, list(priv.values()))
            sweep, sustainable = [], None
            for lam in (rate,) + rates:
                tr2 = [x for x in serve_trace(5000 + int(lam), 4.0, lam) if (x[1], x[2]) in inputs.fields]
                rr = serve_run(ibm, srv, inputs, tr2)
                good = rr["failed_or_rejected"] == 0 and rr["throughput_req_per_s"] >= 0.95 * rr["offered_req_per_s"] \
                    and rr["p99_ms"] is not None and rr["p99_ms"] <= 20.0
                sweep.append({"rate": lam, "throughput_req_per_s": rr["throughput_req_per_s"], "p50_ms": rr["p50_ms"],
                              "p99_ms": rr["p99_ms"], "sustained": good})
                if good:
                    sustainable = lam
            row["rate_sweep_4s"] = sweep
            row["sustainable_req_per_s"] = sustainable
            out[name] = row
        finally:
            ibm.ibm_server_destroy(srv)
            del inputs
            torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_solve_times(rhs_path, reps):
    """Wall times of `reps` oracle 256^3 Poisson solves of the right-hand
    side stored at rhs_path (this process's BLAS threads)."""
    from oracle import ibm_oracle as O
    g = head_grid()
    b = np.load(rhs_path).astype(np.float64)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.poisson_solve(b, g)
        times.append(time.perf_counter() - t0)
    return times


def _oracle_child(rhs_path, reps, threads=None):
    """oracle_solve_times in a fresh child process, with `threads` BLAS /
    OpenMP threads (None: the library default, every host core)."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-time", rhs_path, "--reps", str(reps)],
                       env=env, capture_output=True, text=True, timeout=1800)
    if p.returncode != 0:
        raise RuntimeError("oracle child failed: " + p.stderr[-2000:])
    return json.loads([ln for ln in p.stdout.splitlines() if ln.startswith("{")][-1])["times_s"]


def _head_rhs_file():
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".npy", prefix="ibm_rhs_")
    os.close(fd)
    np.save(path, head_rhs())
    return path


def cpu_baseline(args):
    """The oracle's solve of the headline workload on the host cores: one
    BLAS thread and all cores, best of 3 each, in child processes."""
    path = _head_rhs_file()
    try:
        one = _oracle_child(path, 3, threads=1)
        allc = _oracle_child(path, 3)
    finally:
        os.unlink(path)
    pts = HEAD_N ** 3
    cores = os.cpu_count()
    return {"value": pts / min(allc), "unit": "grid-pts/s", "cores": cores, "kind": "oracle",
            "solves_per_s": 1.0 / min(allc),
            "single_thread": {"value": pts / min(one), "threads": 1, "best_s": min(one), "times_s": one},
            "all_cores": {"value": pts / min(allc), "threads": cores, "best_s": min(allc), "times_s": allc},
            "sample": "the FP64 oracle's 256^3 Poisson solve (numpy, dense eigen-bases, no FFT or Thomas) of "
                      "the headline right-hand side, best of 3, in child processes with 1 BLAS thread and with "
                      "the default BLAS threads (all %d host cores); %.1f s of CPU work" % (cores, sum(one) + sum(allc))}


def run_reference(args):
    """The reference arm: the FP64 oracle's solve of the headline workload,
    as it stands, on the host cores.  One step is one 256^3 solve."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    path = _head_rhs_file()
    try:
        times = _oracle_child(path, args.warmup + args.steps)
    finally:
        os.unlink(path)
    solve_s = times[args.warmup:]
    pts = HEAD_N ** 3
    value = pts * args.steps / sum(solve_s)
    cfg = dict(CONFIG, parallelism="replicas" if ws > 1 else "1 GPU")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grid-pts/s",
           "solves_per_s": value / pts, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(solve_s) / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": "grid-pts/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "one FP64 oracle 256^3 Poisson solve per step (numpy, dense eigen-bases, "
                                      "default BLAS threads on all host cores), %.1f s timed" % sum(solve_s)},
           "e2e": {"value": value, "unit": "grid-pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="the headline solve only (no 128^3 stage, plate, batched, serving or other samples)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error checks")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the FP32-refined serving trace (the workload's 60 s by default)")
    ap.add_argument("--oracle-time", metavar="NPY", help=argparse.SUPPRESS)
    ap.add_argument("--reps", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--quick-stage", action="store_true",
                    help="profiling aid: --warmup then --steps RK stages of the 128^3 workload, the timed stages the "
                         "profiler region")
    ap.add_argument("--quick", action="store_true",
                    help="warm-up and timed steps only (no tracing pass, e2e, Poisson comparison or CPU baseline); "
                         "the timed steps are the profiler region, for ncu launch lists")
    ap.add_argument("--ncu-summary", metavar="CSV",
                    help="summarise an ncu --csv launch list (gpu__time_duration.sum) of `--quick --steps K` (pass "
                         "the same --steps): prints a markdown table")
    ap.add_argument("--ncu-counters", metavar="CSV",
                    help="record the DRAM bytes of a single-kernel ncu capture (raw-page CSV) of `--solve 256` in "
                         "profiles/dram_traffic.json (with --launches-per-step)")
    ap.add_argument("--launches-per-step", type=int, default=2, help=argparse.SUPPRESS)
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
    if args.oracle_time:
        print(json.dumps({"times_s": oracle_solve_times(args.oracle_time, args.reps)}), flush=True)
        return
    if args.ncu_summary:
        ncu_summary(args.ncu_summary, args.steps)
        return
    if args.ncu_counters:
        ncu_counters(args.ncu_counters, "headline", args.launches_per_step)
        return
    if args.solve:
        solve_twice(args.solve, args.plane_mode)
        return
    if args.quick_stage:
        quick_stage(args)
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
