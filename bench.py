"""Benchmark: Dormand-Prince time steps of the 1024 x 1024 x 1 film (4 x 4 x 2 nm
cells, Ms 8e5 A/m, A 1.3e-11 J/m, Ku 5e3 J/m^3 along x, alpha 0.01, open
boundaries -> 2048 x 2048 padded FFT, vortex-plus-noise start, applied field
0-50 mT in a random direction).  One bench step = one adaptive RKDP step =
6 effective-field evaluations (FFT demag + exchange + anisotropy + Zeeman + LL
torque + stage combination) and the device-side step controller.

Metric: effective-field cell-evaluations per second (all evaluations counted,
rejected steps included), with the dominant pass compared with the HBM
roofline.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on this host instead (bounded sample
of the same workload).  Under torchrun (N > 1) each rank runs an independent
replica of the workload (the path has no data exchange between GPUs).
"""

import argparse
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

WORKLOAD = "film_1024x1024"
METRIC = "Heff cell-evals/s"
UNIT = "cell-evals/s"
EVALS_PER_STEP = 6
# workload -> time stepping used for it
METHODS = {
    "film_1024x1024": {"method": "RKDP", "tol": 1e-6, "evals": 6,
                       "desc": "RKDP adaptive, tol 1e-6"},
    "cube_256x256x64": {"method": "HEUN", "dt": 50e-15, "evals": 2,
                        "desc": "Heun, dt 50 fs, thermal field at 300 K (one Philox draw per step)"},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def aggregate_ranks(ms, cell_evals, device):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' cell-evaluations.  Returns (max ms, whole-job cell-evals/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, cell_evals], device=device, dtype=torch.float64)
    mx = t[:1].clone()
    tot = t[1:].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(mx[0])
    return ms_max, float(tot[0]) / (ms_max * 1e-3)


HOT_SOURCES = ("fft32.cuh", "hotpath.cu", "hotpath_kernels.cuh", "mm_internal.cuh")   # the kernels of the timed step


def _source_hash():
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_1102_3069_gb300", "csrc")
    for fn in HOT_SOURCES:
        with open(os.path.join(cdir, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on these sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != _source_hash():
            return None
        return d["kernels"][kernel]["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


def algorithmic_bytes(nx, ny):
    """Bytes each pass must move per launch (2-D open film, FP32, Sec. 3.2 pass layout).

    One RKDP step = x forward of the stage-2 input, then six evaluations: y
    column pass each, inverse x + local terms fused with the next stage's
    forward x transform for stages 2-6, and the plain inverse x + local terms
    + error/torque reductions for stage 7.
    """
    N = nx * ny
    px, py = 2 * nx, 2 * ny
    hx = px // 2 + 1
    spec = 3 * hx * ny * 8                 # half spectrum of the valid rows, complex64
    kern = 4 * hx * (py // 2 + 1) * 4      # real kernel octant, 4 components
    m = 12 * N
    # stage s = 2..6 reads m_s (halo), m_n and k_1..k_{s-1} (k2 unused from stage 6 on),
    # writes k_s and m_{s+1}; stage 7 reads m_7, k1, k3..k6 and writes k7
    reads = {2: 2, 3: 3, 4: 4, 5: 5, 6: 5}
    fused = [spec + m + m * (reads[s] + 2) + spec for s in range(2, 7)]
    final = spec + m + m * 5 + m
    xf = spec + 3 * m                      # stage 2 input m_n + h a21 k1, written out as m_2
    # split passes (padded x length >= 64): the inverse x pass writes H_demag
    # (m bytes) and the cell pass reads it back; that round trip is not part
    # of the method's bytes, so "step" leaves it out
    cell = [m + m + m * (reads[s] + 2) for s in range(2, 7)] + [m + m + 5 * m + m]
    return {
        "k_xfwd": float(xf),
        "k_colconv_y": float(2 * spec + kern),
        "k_xinv_local_fused": sum(fused) / 5.0,
        "k_xinv_local": float(final),
        "k_xinv_h": float(spec + m),
        "k_local_h": sum(cell) / 6.0,
        "k_xfwd_next": float(m + spec),
        "step": float(xf + 6 * (2 * spec + kern) + sum(fused) + final),
    }


def algorithmic_bytes_3d(shape, pz, images_axes=(True, True, False), axes=True):
    """Bytes per pass for the 3-D sequence (x fused, y forward, z column, y inverse), Heun stages;
    axes: the cell pass also reads a per-cell easy axis (12 B per cell)."""
    nx, ny, nz = shape
    N = nx * ny * nz
    px = nx if images_axes[0] else 2 * nx
    py = ny if images_axes[1] else 2 * ny
    hx = px // 2 + 1
    s1 = 3 * hx * nz * ny * 8
    s2 = 3 * hx * py * nz * 8
    kern = 6 * hx * (py // 2 + 1) * (pz // 2 + 1) * 4
    m = 12 * N
    ax = m if axes else 0
    heun1 = s1 + m + 2 * m + s1 + ax       # k1 and the predictor written, next spectrum written
    heun2 = s1 + m + 2 * m + m + s1 + ax   # m_n and k1 read, m_{n+1} written, next spectrum written
    return {
        "k_yfwd": float(s1 + s2),
        "k_colconv_z": float(2 * s2 + kern),
        "k_yinv": float(s2 + s1),
        "k_xinv_local_fused": (heun1 + heun2) / 2.0,
        "k_xinv_h": float(s1 + m),
        "k_local_h": (4 * m + 5 * m) / 2.0 + ax,   # H_demag read back + the Heun stage's reads and writes
        "k_xfwd_next": float(m + s1),
        "step": float(2 * (2 * (s1 + s2) + 2 * s2 + kern) + heun1 + heun2),
    }


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    wname = args.workload
    spec = METHODS[wname]
    w = inputs.workload(wname, seed=rank)
    nx, ny, nz = w["shape"]
    N = nx * ny * nz
    if spec["method"] == "RKDP":
        method, first_dt, dt_step, tol = B.MM_RKDP, 1e-13, 0.0, spec["tol"]
    else:
        method, first_dt, dt_step, tol = B.MM_HEUN, spec["dt"], spec["dt"], 0.0
    stream = torch.cuda.Stream()
    dft = B.MM_DFT_SPLIT_BF16 if args.dft == "split-bf16" else None
    with torch.cuda.stream(stream):
        s = B.Solver(w["shape"], w["cell"], pbc=w["pbc"], stream=stream.cuda_stream, dft_precision=dft,
                     **w["material"])
        axes = None
        if w.get("axes") is not None:             # per-cell easy axes (the cube's polycrystal)
            axes = torch.from_numpy(w["axes"]).cuda()
            B.mm_set_anisotropy_axes(s.ctx, axes)
        m = torch.from_numpy(w["m"]).cuda()
        ctx = s.ctx
        B.mm_load(ctx, m)
        # warm-up (also settles the step size)
        B.mm_advance(ctx, method, args.warmup, dt_s=first_dt, tol=tol)
        st0 = B.mm_get_stats(ctx)
        flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")    # > 129 MB L2
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        # the timed window of `steps` steps is repeated until the clock sampler
        # has seen at least min_timed_s of load; the median window is reported
        windows = []                                  # (ms of the window, evals, simulated time)
        with ClockSampler(dev) as clk:
            t_wall0 = time.perf_counter()
            while True:
                sa = B.mm_get_stats(ctx)
                for k in range(args.steps):
                    flush.fill_(k & 0xFF)                 # evict the previous step from L2
                    ev[k][0].record(stream)
                    B.mm_advance(ctx, method, 1, dt_s=dt_step, tol=tol)
                    ev[k][1].record(stream)
                torch.cuda.synchronize()
                sb = B.mm_get_stats(ctx)
                windows.append((sum(a.elapsed_time(b) for a, b in ev), sb["evals"] - sa["evals"], sb["t"] - sa["t"]))
                if time.perf_counter() - t_wall0 >= args.min_timed_s or len(windows) >= 1000:
                    break
            t_wall = time.perf_counter() - t_wall0
        st1 = B.mm_get_stats(ctx)
        assert st1["status"] == 0, st1
        gpu_ms, evals, sim_t = sorted(windows)[len(windows) // 2]

        # per-pass durations over a second timed region of the same steps
        passes = B.pass_times(ctx, lambda: B.mm_advance(ctx, method, min(args.steps, 200), dt_s=dt_step, tol=tol))

        # end to end through the host-buffer entry point: H2D + step + D2H per step
        mh = torch.from_numpy(w["m"]).pin_memory()
        mh_np = mh.numpy()
        B.mm_run_host(ctx, mh_np, method, 1, dt_s=first_dt, tol=tol)
        torch.cuda.synchronize()
        e0 = B.mm_get_stats(ctx)["evals"]
        ke = max(3, min(args.steps // 2, 200))
        te = time.perf_counter()
        ev_total = 0
        for _ in range(ke):
            B.mm_run_host(ctx, mh_np, method, 1, dt_s=dt_step, tol=tol)
            ev_total += B.mm_get_stats(ctx)["evals"]
        te = time.perf_counter() - te
        del e0

    if ws > 1:
        gpu_ms_max, value = aggregate_ranks(gpu_ms, float(evals * N), "cuda")
    else:
        gpu_ms_max, value = gpu_ms, evals * N / (gpu_ms * 1e-3)
    if rank != 0:
        return None

    hbm, peak_kind = _peaks()
    ab = algorithmic_bytes(nx, ny) if nz == 1 else algorithmic_bytes_3d(w["shape"], 2 * nz, tuple(bool(v) for v in w["pbc"]))
    # dominant pass = largest share of the step time
    dom = max((k for k in passes if k in ab), key=lambda k: passes[k]["ms_total"])
    dms = passes[dom]["ms_per_launch"]
    achieved = ab[dom] / (dms * 1e-3) / 1e9
    step_bytes = ab["step"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": gpu_ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded vortex-plus-noise state, random applied field)",
        "config": {"workload": wname, "grid": [nx, ny, nz], "cell_nm": [round(c * 1e9, 3) for c in w["cell"]],
                   "pbc": list(w["pbc"]), "method": spec["desc"], "evals_per_step": spec["evals"],
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "timing": "median of repeated windows of `steps` steps (CUDA events on the launching stream)",
                   "dft": args.dft},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": _traffic_for(dom), "kernel": dom, "peak_source": peak_kind,
                     "bytes_per_launch": ab[dom], "ms_per_launch": dms},
        "step_roofline": {"bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (gpu_ms / args.steps * 1e-3) / 1e9,
                          "frac": step_bytes / (gpu_ms / args.steps * 1e-3) / 1e9 / hbm},
        "passes": passes,
        "ns_simulated_per_hour": sim_t * 1e9 / (gpu_ms * 1e-3 / 3600.0) if gpu_ms > 0 else None,
        "clocks": dict(clk.summary(), timed_windows=len(windows), timed_wall_s=t_wall,
                       window_ms_min=min(x[0] for x in windows), window_ms_max=max(x[0] for x in windows)),
        "gpu_launches": int(sum(v["launches"] for v in passes.values()) / max(1, min(args.steps, 200)) * args.steps),
        "e2e": {"value": ev_total * N / te if te > 0 else None, "unit": UNIT,
                "h2d_bytes_per_step": 12 * N, "d2h_bytes_per_step": 12 * N,
                "note": "mm_run_host: pinned host m in, one step (RKDP: 7 evaluations, fresh k1 + 6), m out"},
    }
    return line


def run_reference(args):
    """Time the FP64 oracle (as it stands) on this host on a bounded sample."""
    import numpy as np

    from oracle import llg
    from paper_1102_3069_gb300 import inputs

    ws, rank = _dist()
    if rank != 0:
        return None
    w = inputs.workload(WORKLOAD, seed=0)
    mat = w["material"]
    t0 = time.perf_counter()
    p = llg.Problem(w["shape"], w["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"], u=mat["easy_axis"],
                    B=mat["B"])
    setup_s = time.perf_counter() - t0
    m = w["m"].astype(np.float64)
    N = int(np.prod(w["shape"]))
    # one sample = one Heff evaluation of the full grid with its LL right-hand side
    for _ in range(args.warmup):
        p.rhs(m)
    t = time.perf_counter()
    for _ in range(args.steps):
        p.rhs(m)
    dt = time.perf_counter() - t
    value = args.steps * N / dt
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "grid": list(w["shape"]), "sample": "one full-grid H_eff + LL rhs per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full-grid H_eff evaluations of {WORKLOAD} (kernel setup "
                                       f"{setup_s:.0f} s untimed)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline_sample(seconds=20.0):
    """Oracle on a bounded sample of the same workload (rank 0, N = 1 only)."""
    import numpy as np

    from oracle import llg
    from paper_1102_3069_gb300 import inputs

    w = inputs.workload(WORKLOAD, seed=0)
    mat = w["material"]
    p = llg.Problem(w["shape"], w["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"], u=mat["easy_axis"],
                    B=mat["B"])
    m = w["m"].astype(np.float64)
    N = int(np.prod(w["shape"]))
    n = 0
    t = time.perf_counter()
    while time.perf_counter() - t < seconds or n < 2:
        p.rhs(m)
        n += 1
    dt = time.perf_counter() - t
    return {"value": n * N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full-grid H_eff evaluations (FP64 numpy, one thread) of {WORKLOAD}"}


def run_table1(args):
    """Euler steps (one field evaluation + LL + update each) on the Table-1 grids."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    rows = []
    sizes = ([("N2", n) for n in (32, 64, 128, 256, 512, 600, 700, 992, 1024, 2048)] +
             [("N3", n) for n in (8, 16, 32, 64, 128)])
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    for kind, n in sizes:
        w = inputs.workload(f"table1_{kind}_{n}")
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s = B.Solver(w["shape"], w["cell"], stream=stream.cuda_stream, **w["material"])
            m = torch.from_numpy(w["m"]).cuda()
            B.mm_load(s.ctx, m)
            B.mm_advance(s.ctx, B.MM_EULER, 5, dt_s=1e-14)
            k = 50
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            for i in range(k):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                B.mm_advance(s.ctx, B.MM_EULER, 1, dt_s=1e-14)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)[k // 2]
        cells = int(np.prod(w["shape"]))
        rows.append({"grid": f"{n}^{2 if kind == 'N2' else 3}", "cells": cells, "ms_per_euler_step": ms,
                     "cell_evals_per_s": cells / (ms * 1e-3)})
        s.close()
        del s, m
        torch.cuda.empty_cache()
    return {"metric": "Euler step time (Table 1 grids)", "unit": "ms", "rows": rows,
            "config": {"material": "Ms 8e5 A/m, A 1.3e-11 J/m, Ku 5e3 J/m^3 along x, Bz 10 mT, alpha 0.01",
                       "cell_nm": 4, "timing": "median of 50 steps, CUDA events, L2 flushed between steps"}}


def _host_cpu():
    """Core count and CPU model of this host (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.split(":")[0].strip() == "Model name":
                    break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _oracle_euler_worker(args):
    """One process: oracle Euler steps of a table-1 grid for `seconds` (kernel build untimed)."""
    name, seconds = args
    import numpy as np

    from oracle import llg
    from paper_1102_3069_gb300 import inputs
    w = inputs.workload(name)
    mat = w["material"]
    p = llg.Problem(w["shape"], w["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"], u=mat["easy_axis"],
                    B=mat["B"])
    m = w["m"].astype(np.float64)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds or k < 2:
        m = llg.euler_step(p, m, 1e-14)
        k += 1
    return k, time.perf_counter() - t0, int(np.prod(w["shape"]))


def run_cpu_sweep(args):
    """The FP64 oracle timed on this host: Euler steps of the Table-1 grids on one
    thread (the paper's CPU column is one core), and the throughput of all host
    cores running independent oracle processes on the 256^2 grid."""
    import multiprocessing as mp
    rows = []
    grids = [("N2", n) for n in (32, 64, 128, 256, 512)] + [("N3", n) for n in (8, 16, 32)]
    for kind, n in grids:
        k, t, cells = _oracle_euler_worker((f"table1_{kind}_{n}", 2.0))
        rows.append({"grid": f"{n}^{2 if kind == 'N2' else 3}", "cells": cells, "ms_per_euler_step": t / k * 1e3,
                     "steps": k})
    host = _host_cpu()
    ncore = host["nproc"] or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(ncore) as pool:
        res = pool.map(_oracle_euler_worker, [("table1_N2_256", 10.0)] * ncore)
    wall = time.perf_counter() - t0
    evals = sum(k * c for k, _, c in res)
    per = [k * c / t for k, t, c in res]
    return {"metric": "oracle Euler step time (Table 1 grids), one thread", "unit": "ms", "rows": rows,
            "all_cores": {"grid": "256^2", "processes": ncore, "cell_evals_per_s": sum(per),
                          "cell_evals_per_s_one_process": per[0], "wall_s_including_kernel_builds": wall,
                          "evals": evals},
            "host": host,
            "config": {"oracle": "numpy float64 (FFT convolution, one thread per process)",
                       "timing": "wall clock per Euler step after the kernel build; all cores: one spawn process "
                                 "per core, each 10 s of steps"}}


def run_ensemble(args):
    """Batched Dormand-Prince steps of the 512-sample ensemble (grids 32..256 x
    32..256 x 1..4 of 4 nm cells, per-sample material and field, alpha 0.02),
    next to the same samples stepped one context at a time."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    ws, rank = _dist()
    samples = inputs.ensemble(args.ensemble, seed=rank)
    stream = torch.cuda.Stream()
    cells = [int(np.prod(s["shape"])) for s in samples]
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        sol = [B.Solver(s["shape"], s["cell"], pbc=s["pbc"], stream=stream.cuda_stream, tensor=False,
                        fft_lengths=B.MM_FFT_POW2,
                        **s["material"]) for s in samples]
        ms = [torch.from_numpy(inputs.random_unit(s["shape"], s["m_seed"])).cuda() for s in samples]
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        bt = B.Batch(sol, stream.cuda_stream)
        B.mm_batch_load(bt.b, ms)
        B.mm_batch_advance(bt.b, B.MM_RKDP, args.warmup, dt_s=1e-13, tol=1e-6)
        st0 = B.mm_batch_get_stats(bt.b, len(sol))
        flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                B.mm_batch_advance(bt.b, B.MM_RKDP, 1, dt_s=0.0, tol=1e-6)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        st1 = B.mm_batch_get_stats(bt.b, len(sol))
        gpu_ms = sum(a.elapsed_time(b) for a, b in ev)
        evals = [b_["evals"] - a_["evals"] for a_, b_ in zip(st0, st1)]
        assert all(x["status"] == 0 for x in st1)
        value = sum(e * n for e, n in zip(evals, cells)) / (gpu_ms * 1e-3)
        # the same samples, one context at a time (each replaying its own step graph)
        k_seq = max(2, min(args.steps, 10))
        for s_, m in zip(sol, ms):
            B.mm_load(s_.ctx, m)
            B.mm_advance(s_.ctx, B.MM_RKDP, 2, dt_s=1e-13, tol=1e-6)
        e_seq0 = [B.mm_get_stats(s_.ctx)["evals"] for s_ in sol]
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(k_seq):
            for s_ in sol:
                B.mm_advance(s_.ctx, B.MM_RKDP, 1, dt_s=0.0, tol=1e-6)
        b_.record(stream)
        torch.cuda.synchronize()
        e_seq1 = [B.mm_get_stats(s_.ctx)["evals"] for s_ in sol]
        seq_value = sum((e1 - e0) * n for e0, e1, n in zip(e_seq0, e_seq1, cells)) / (a_.elapsed_time(b_) * 1e-3)
    # method bytes per accepted-or-rejected step, summed over the samples
    step_bytes = 0.0
    for s_, e0, e1 in zip(samples, st0, st1):
        nx, ny, nz = s_["shape"]
        ab = algorithmic_bytes(nx, ny) if nz == 1 else algorithmic_bytes_rk_3d(s_["shape"])
        step_bytes += ab["step"]
    hbm, peak_kind = _peaks()
    ms_step = gpu_ms / args.steps
    achieved = step_bytes / (ms_step * 1e-3) / 1e9
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded per-sample geometry, material, field and random unit m)",
        "config": {"workload": f"ensemble_{len(samples)}", "samples": len(samples), "cells_total": sum(cells),
                   "grids": "nx, ny U{32..256}, nz U{1..4}, 4 nm cells, open boundaries",
                   "method": "RKDP adaptive per sample, tol 1e-6", "launches": "one per pass and FFT length",
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "parallelism": "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "whole batched step", "peak_source": peak_kind,
                     "bytes_per_launch": step_bytes, "ms_per_launch": ms_step},
        "one_context_at_a_time": {"value": seq_value, "unit": UNIT, "steps": k_seq},
        "setup_s": setup_s,
        "clocks": clk.summary(),
    }


def run_relax(args):
    """Time to relax: films of 128 x 128 x 1 cells (random material, in-plane
    field and easy axis, alpha 1) from random unit vectors to max |m x H|/Ms
    < 1e-4 with adaptive Dormand-Prince steps, batched (mm_batch_relax) and one
    film at a time (mm_relax)."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    ws, rank = _dist()
    films = inputs.relax_films(args.relax, seed=rank)
    stream = torch.cuda.Stream()
    # per-step error 1e-6: at 1e-5 the state jitters by ~1e-5 per ~1 ps step
    # near equilibrium, a torque floor close to the 1e-4 target (measured)
    tq_tol, err_tol, max_steps = 1e-4, 1e-6, args.relax_max_steps
    with torch.cuda.stream(stream):
        sol = [B.Solver(f["shape"], f["cell"], pbc=f["pbc"], stream=stream.cuda_stream, tensor=False,
                        fft_lengths=B.MM_FFT_POW2,
                        **f["material"]) for f in films]
        m0 = [torch.from_numpy(inputs.random_unit(f["shape"], f["m_seed"])).cuda() for f in films]
        bt = B.Batch(sol, stream.cuda_stream)
        mb = [m.clone() for m in m0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, steps, tq, conv = B.mm_batch_relax(bt.b, mb, tq_tol, err_tol, max_steps)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        st = B.mm_batch_get_stats(bt.b, len(sol))
        evals = sum(x["evals"] for x in st)
        k_one = min(len(films), 8)
        t1 = time.perf_counter()
        steps_one = []
        conv_one = 0
        for s_, m in zip(sol[:k_one], m0[:k_one]):
            mm = m.clone()
            try:
                n, _ = B.mm_relax(s_.ctx, mm, tq_tol, err_tol, max_steps)
                conv_one += 1
            except B.MMError as e:
                if e.code != B.MM_ENOTCONVERGED:
                    raise
                n = B.mm_get_stats(s_.ctx)["accepted"] + B.mm_get_stats(s_.ctx)["rejected"]
            steps_one.append(n)
        torch.cuda.synchronize()
        t_one = (time.perf_counter() - t1) / k_one
    cells = films[0]["shape"][0] * films[0]["shape"][1]
    return {
        "metric": "time to relax (torque < 1e-4)", "value": t_batch, "unit": "s", "higher_is_better": False,
        "n_gpus": ws, "films": len(films), "converged": conv, "status": rc,
        "per_film_s_batched": t_batch / len(films), "per_film_s_one_at_a_time": t_one,
        "steps_median": float(np.median(steps)), "steps_max": int(max(steps)),
        "torque_max": float(max(tq)), "converged_one_at_a_time": conv_one, "films_one_at_a_time": k_one,
        "steps_one_at_a_time": [int(x) for x in steps_one],
        "steps": [int(x) for x in steps], "torques": [float(x) for x in tq],
        "cell_evals_per_s_batched": evals * cells / t_batch,
        "data": "synthetic (seeded material, field, easy axis and random unit m per film)",
        "config": {"workload": f"relax_films_{len(films)}", "grid": [128, 128, 1], "cell_nm": [4, 4, 3],
                   "alpha": 1.0, "method": "RKDP adaptive, tol 1e-6 per step", "torque_tol": tq_tol,
                   "timing": "wall clock around mm_batch_relax (host polls every 64 steps) and around mm_relax "
                             f"for the first {k_one} films"},
    }


def _relax_films(films, m_start, stream, tq_tol, err_tol, max_steps):
    """Relax the films from the given start states together (mm_batch_relax);
    returns (relaxed states, wall seconds of the relaxation, steps, torques, converged)."""
    import torch

    from paper_1102_3069_gb300 import binding as B
    with torch.cuda.stream(stream):
        sol = [B.Solver(f["shape"], f["cell"], pbc=f["pbc"], stream=stream.cuda_stream, tensor=False,
                        fft_lengths=B.MM_FFT_POW2,
                        **f["material"]) for f in films]
        bt = B.Batch(sol, stream.cuda_stream)
        ms = [m.clone() for m in m_start]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, steps, tq, conv = B.mm_batch_relax(bt.b, ms, tq_tol, err_tol, max_steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    del bt, sol
    return ms, t, steps, tq, conv


def run_warmstart(args):
    """Learned warm start of the relaxation (128 x 128 x 1 films, 4 x 4 x 3 nm,
    random material, in-plane easy axis and field, alpha 1): the solver relaxes
    n_train films from random unit vectors to max |m x H|/Ms < 1e-4 (the
    training set), the Fourier neural operator learns relaxed m from the film's
    parameters (Adam, bf16 tensor-core kernels), and on held-out films the
    time to relax from its prediction (inference included) is compared with
    the time from random unit vectors."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    n_train, n_eval, bs = args.warmstart, args.warmstart_eval, 32
    epochs, lr0 = args.warmstart_epochs, 1e-3
    tq_tol, err_tol, max_steps = 1e-4, 1e-6, args.relax_max_steps
    stream = torch.cuda.Stream()
    # training set: relaxed states from the solver itself
    t0 = time.perf_counter()
    train = inputs.relax_films(n_train, seed=100)
    Y = torch.empty((n_train, 3, 128, 128), dtype=torch.float32, device="cuda")
    chunk = 256
    gen_steps = []
    for i in range(0, n_train, chunk):
        films = train[i:i + chunk]
        m0 = [torch.from_numpy(inputs.random_unit(f["shape"], f["m_seed"])).cuda() for f in films]
        ms, _, steps, _, _ = _relax_films(films, m0, stream, tq_tol, err_tol, max_steps)
        for j, m in enumerate(ms):
            Y[i + j] = m.view(3, 128, 128)
        gen_steps += steps
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    X = torch.from_numpy(inputs.fno_features(train)).cuda()
    # training
    net = B.Fno(bs, stream.cuda_stream)
    net.set_params(inputs.fno_init(0))
    g = np.random.default_rng(0)
    nb = n_train // bs
    total = epochs * nb
    losses = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    with torch.cuda.stream(stream):
        it = 0
        for ep in range(epochs):
            perm = torch.from_numpy(g.permutation(n_train)).cuda()
            ep_loss = []
            for k in range(nb):
                idx = perm[k * bs:(k + 1) * bs]
                xb, yb = X[idx].contiguous(), Y[idx].contiguous()
                lr = lr0 * 0.5 * (1.0 + np.cos(np.pi * it / total))
                want = k == nb - 1 or k % 16 == 0
                l = B.mm_fno_train_step(net.f, xb, yb, bs, lr, want_loss=want)
                if want:
                    ep_loss.append(l)
                it += 1
            losses.append(float(np.mean(ep_loss)))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    # held-out films: plain relaxation against the warm start
    evalf = inputs.relax_films(n_eval, seed=7)
    m_rand = [torch.from_numpy(inputs.random_unit(f["shape"], f["m_seed"])).cuda() for f in evalf]
    _, t_plain, steps_plain, tq_plain, conv_plain = _relax_films(evalf, m_rand, stream, tq_tol, err_tol, max_steps)
    nev8 = (n_eval + 7) // 8 * 8
    xe = np.zeros((nev8, 16, 128, 128), dtype=np.float32)
    xe[:n_eval] = inputs.fno_features(evalf)
    pred = torch.empty((nev8, 3, 128, 128), dtype=torch.float32, device="cuda")
    evnet = B.Fno(nev8, stream.cuda_stream)
    evnet.set_params(net.get_params())
    xed = torch.from_numpy(xe).cuda()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    with torch.cuda.stream(stream):
        B.mm_fno_predict(evnet.f, xed, nev8, pred)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t2
    m_warm = [pred[i].reshape(-1).contiguous() for i in range(n_eval)]
    ms_w, t_warm, steps_warm, tq_warm, conv_warm = _relax_films(evalf, m_warm, stream, tq_tol, err_tol, max_steps)
    # the prediction's own error: distance to the state the solver then reached
    err = [float(torch.sqrt(((m_warm[i].view(3, -1) - ms_w[i].view(3, -1)) ** 2).sum(0)).mean()) for i in range(n_eval)]
    t_warm_total = t_inf + t_warm
    return {
        "metric": "time to relax (torque < 1e-4), learned warm start vs plain", "value": t_warm_total, "unit": "s",
        "higher_is_better": False, "n_gpus": 1,
        "plain_s": t_plain, "warm_inference_s": t_inf, "warm_relax_s": t_warm,
        "speedup": t_plain / t_warm_total,
        "films": n_eval, "converged_plain": conv_plain, "converged_warm": conv_warm,
        "steps_median_plain": float(np.median(steps_plain)), "steps_median_warm": float(np.median(steps_warm)),
        "torque_max_plain": float(max(tq_plain)), "torque_max_warm": float(max(tq_warm)),
        "prediction_mean_dm": float(np.mean(err)),
        "training": {"films": n_train, "generation_s": t_gen, "generation_steps_median": float(np.median(gen_steps)),
                     "epochs": epochs, "batch": bs, "train_s": t_train, "loss_first_epoch": losses[0],
                     "loss_last_epoch": losses[-1], "optimizer": "Adam lr 1e-3 cosine to 0, betas (0.9, 0.999)"},
        "dtype": "bf16 operands, fp32 accumulation (operator); f32 solver",
        "data": "synthetic (seeded material, field, easy axis; training targets relaxed by the solver from random m)",
        "config": {"workload": f"warmstart_films_128x128_train{n_train}_eval{n_eval}", "grid": [128, 128, 1],
                   "cell_nm": [4, 4, 3], "alpha": 1.0, "method": "RKDP adaptive, tol 1e-6 per step",
                   "torque_tol": tq_tol,
                   "timing": "wall clock around mm_batch_relax of the held-out films (all at once) from random m "
                             "and from the prediction; the prediction's inference time is added to the latter"},
    }


def run_relax_ensemble(args):
    """Time to relax an ensemble of independent samples of uneven sizes (grids
    32..256 x 32..256 x 1..4 of 4 nm cells, random material, easy axis and
    field) from random unit vectors to max |m x H|/Ms < 1e-4, all samples in
    one batch (mm_batch_relax: per-sample step control, finished samples leave
    the batched launches)."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    samples = inputs.ensemble(args.relax_ensemble, alpha=args.relax_alpha)
    tq_tol, err_tol, max_steps = 1e-4, 1e-6, args.relax_max_steps
    stream = torch.cuda.Stream()
    m0 = [torch.from_numpy(inputs.random_unit(x["shape"], x["m_seed"])).cuda() for x in samples]
    t0 = time.perf_counter()
    ms, t, steps, tq, conv = _relax_films(samples, m0, stream, tq_tol, err_tol, max_steps)
    setup_and_relax = time.perf_counter() - t0
    cells = [int(np.prod(x["shape"])) for x in samples]
    left = [i for i in range(len(samples)) if not tq[i] < tq_tol]
    unconverged = [{"sample": i, "shape": list(samples[i]["shape"]), "Ms": samples[i]["material"]["Ms"],
                    "Ku": samples[i]["material"]["Ku"], "B_T": float(np.linalg.norm(samples[i]["material"]["B"])),
                    "steps": int(steps[i]), "torque": float(tq[i])} for i in left]
    return {"metric": "time to relax the ensemble (torque < 1e-4)", "value": t, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "samples": len(samples), "converged": conv,
            "cells_total": sum(cells), "steps_median": float(np.median(steps)), "steps_max": int(max(steps)),
            "torque_max": float(max(tq)), "setup_plus_relax_s": setup_and_relax,
            "steps_quantiles": {q: float(np.quantile(steps, float(q))) for q in ("0.5", "0.9", "0.95")},
            "unconverged": unconverged,
            "data": "synthetic (seeded per-sample geometry, material, field and random unit m)",
            "config": {"workload": f"ensemble_{len(samples)}_relax", "alpha": args.relax_alpha,
                       "grids": "nx, ny U{32..256}, nz U{1..4}, 4 nm cells, open boundaries",
                       "method": "RKDP adaptive per sample, tol 1e-6 per step", "torque_tol": tq_tol,
                       "max_steps": max_steps,
                       "timing": "wall clock around mm_batch_relax (host polls every 64 steps)"}}


def run_gemm(args):
    """The library's tensor-core product (tcgen05) alone: C = A B^T, bf16
    operands, fp32 accumulation, timed with CUDA events against the measured
    bf16 tensor peak."""
    import torch

    from paper_1102_3069_gb300 import binding as B
    m, n, k = args.gemm
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.randn((m, k), device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn((n, k), device="cuda", generator=g).to(torch.bfloat16)
    c = torch.empty((m, n), device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        B.mm_gemm_bf16(a, k, 0, b, k, 0, c, n, 0, m, n, k, stream=stream)
    torch.cuda.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        B.mm_gemm_bf16(a, k, 0, b, k, 0, c, n, 0, m, n, k, stream=stream)
    e1.record()
    torch.cuda.synchronize()
    assert B.mm_gemm_status(stream) == B.MM_OK
    ms = e0.elapsed_time(e1) / reps
    tflops = 2.0 * m * n * k / (ms * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    err = float((c - a.float() @ b.float().T).abs().max() / (a.float() @ b.float().T).abs().max())
    return {"metric": "tcgen05 bf16 product throughput", "value": tflops, "unit": "TFLOP/s",
            "shape": [m, n, k], "ms": ms, "max_rel_err_vs_fp32_product": err,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "peak_source": kind + " (bf16 cuBLAS burst)"}}


def run_cufft_comparison(args):
    """The demag convolution of the 1024 x 1024 film through cuFFT (torch.fft:
    zero-padded 2048 x 2048 R2C of the three components, the 3x3 real kernel
    product, C2R) next to this library's three passes (forward x, column pass
    with the product, inverse x) for the same evaluation."""
    import numpy as np
    import torch

    from paper_1102_3069_gb300 import binding as B
    from paper_1102_3069_gb300 import inputs

    w = inputs.workload("film_1024x1024")
    nx, ny, _ = w["shape"]
    px, py = 2 * nx, 2 * ny
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = B.Solver(w["shape"], w["cell"], stream=stream.cuda_stream, **w["material"])
        m = torch.from_numpy(w["m"]).cuda()
        B.mm_load(s.ctx, m)
        B.mm_advance(s.ctx, B.MM_RKDP, 20, dt_s=1e-13, tol=1e-6)
        passes = B.pass_times(s.ctx, lambda: B.mm_advance(s.ctx, B.MM_RKDP, 100, tol=1e-6))
        ours = (passes["k_xfwd_next"]["ms_per_launch"] + passes["k_colconv_y"]["ms_per_launch"]
                + passes["k_xinv_h"]["ms_per_launch"])
        # cuFFT: the kernel spectrum (real, 4 components for a film) on the full padded grid
        K = torch.randn(4, py, px // 2 + 1, device="cuda", dtype=torch.float32)
        mp = torch.zeros(3, py, px, device="cuda", dtype=torch.float32)
        mp[:, :ny, :nx] = m[:, 0]
        def conv():
            Mk = torch.fft.rfft2(mp)
            Hk = torch.stack([K[0] * Mk[0] + K[3] * Mk[1], K[3] * Mk[0] + K[1] * Mk[1], K[2] * Mk[2]])
            return torch.fft.irfft2(Hk, s=(py, px))[:, :ny, :nx]
        for _ in range(5):
            conv()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 50
        a.record(stream)
        for _ in range(n):
            conv()
        b.record(stream)
        torch.cuda.synchronize()
        cufft = a.elapsed_time(b) / n
    return {"metric": "demag convolution time per evaluation", "unit": "ms", "higher_is_better": False,
            "value": ours, "cufft_torch_fft": cufft, "ratio_cufft_over_ours": cufft / ours,
            "config": {"workload": "film_1024x1024", "fft": [py, px],
                       "ours": "k_xfwd_r + k_colconv + k_xinv_h (CUDA events per pass, RKDP steps)",
                       "cufft": "torch.fft.rfft2 of the zero-padded 3 x 2048 x 2048 magnetisation, "
                                "3x3 real kernel product, irfft2, crop (CUDA events over 50 evaluations)"}}


def algorithmic_bytes_rk_3d(shape):
    """Method bytes of one Dormand-Prince step of an open 3-D grid (Sec. 3.2
    passes: x, y forward, z column pass, y, x inverse per evaluation).  With
    nz <= 8 the y and z stages are one pass over the x spectrum (read and
    written once, plus the kernel); beyond, the y forward pass writes the
    z-padded spectrum s2, the z column pass reads and writes it and the y
    inverse pass reads it back."""
    nx, ny, nz = shape
    N = nx * ny * nz
    px, py = 2 * nx, 2 * ny
    pz = 1
    while pz < 2 * nz - 1:
        pz *= 2
    hx = px // 2 + 1
    s1 = 3 * hx * nz * ny * 8
    s2 = 3 * hx * py * nz * 8
    kern = 6 * hx * (py // 2 + 1) * (pz // 2 + 1) * 4
    m = 12 * N
    reads = {2: 2, 3: 3, 4: 4, 5: 5, 6: 5}
    fused = [s1 + m + m * (reads[s] + 2) + s1 for s in range(2, 7)]
    final = s1 + m + m * 5 + m
    xf = s1 + 3 * m
    col = 2 * s1 + kern if nz <= 8 else 2 * (s1 + s2) + 2 * s2 + kern
    return {"step": float(xf + 6 * col + sum(fused) + final)}


def cpu_baseline_cube(seconds=20.0):
    """Oracle on a 32^3 crop of the cube workload (its full periodic kernel is out of reach in numpy)."""
    import numpy as np

    from oracle import llg
    from paper_1102_3069_gb300 import inputs

    w = inputs.workload("cube_256x256x64", seed=0)
    mat = w["material"]
    shape = (32, 32, 32)
    p = llg.Problem(shape, w["cell"], mat["Ms"], mat["Aex"], mat["alpha"], Ku=mat["Ku"],
                    u=inputs.tilted_axes(shape, 0).astype(np.float64), B=mat["B"], T=mat["temperature"],
                    seed=mat["seed"], pbc=(True, True, False), images=2)
    m = inputs.random_unit(shape, 0).astype(np.float64)
    N = int(np.prod(shape))
    n = 0
    t = time.perf_counter()
    while time.perf_counter() - t < seconds or n < 2:
        p.rhs(m, step=n, dt=w["dt"])
        n += 1
    dt = time.perf_counter() - t
    return {"value": n * N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} H_eff evaluations of a 32^3 crop of cube_256x256x64 (2 images per periodic side)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(METHODS))
    ap.add_argument("--table1", action="store_true",
                    help="Euler-step timing sweep of the paper's Table 1 grids (N^2 and N^3, 4 nm cells)")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="the FP64 oracle's Euler steps on the Table-1 grids (one thread) and on all host cores")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="batched Dormand-Prince steps of an ensemble of this many independent samples")
    ap.add_argument("--relax", type=int, default=0,
                    help="time to relax this many 128 x 128 films from random states (batched and one by one)")
    ap.add_argument("--relax-max-steps", type=int, default=100000)
    ap.add_argument("--relax-ensemble", type=int, default=0,
                    help="time to relax this many ensemble samples (uneven grids) together")
    ap.add_argument("--relax-alpha", type=float, default=0.02)
    ap.add_argument("--warmstart", type=int, default=0,
                    help="learned warm start: relax this many training films, train the operator, compare "
                         "relaxation times on held-out films")
    ap.add_argument("--warmstart-eval", type=int, default=64)
    ap.add_argument("--warmstart-epochs", type=int, default=60)
    ap.add_argument("--min-timed-s", type=float, default=2.0,
                    help="repeat the timed window of --steps steps until this much wall time has passed")
    ap.add_argument("--dft", default="fp32", choices=["fp32", "split-bf16"],
                    help="precision of the 3-D z transforms (split-bf16: tensor-core DFT products)")
    ap.add_argument("--gemm", type=int, nargs=3, default=None, metavar=("M", "N", "K"),
                    help="time the tensor-core bf16 product alone")
    ap.add_argument("--cufft", action="store_true",
                    help="time the film's demag convolution through cuFFT next to the hand-written passes")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps > 5:
            args.steps = 5
        if args.warmup > 1:
            args.warmup = 1
        line = run_reference(args)
        if line:
            print(json.dumps(line))
        return
    import __graft_entry__
    from paper_1102_3069_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        __graft_entry__.build()
    if args.table1:
        print(json.dumps(run_table1(args)))
        return
    if args.cpu_sweep:
        print(json.dumps(run_cpu_sweep(args)))
        return
    if args.ensemble > 0:
        print(json.dumps(run_ensemble(args)))
        return
    if args.relax > 0:
        print(json.dumps(run_relax(args)))
        return
    if args.gemm:
        print(json.dumps(run_gemm(args)))
        return
    if args.relax_ensemble > 0:
        print(json.dumps(run_relax_ensemble(args)))
        return
    if args.warmstart > 0:
        print(json.dumps(run_warmstart(args)))
        return
    if args.cufft:
        print(json.dumps(run_cufft_comparison(args)))
        return
    line = run_gpu(args)
    if line is None:
        return
    ws, _ = _dist()
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample() if args.workload == WORKLOAD else cpu_baseline_cube()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
