#!/usr/bin/env python3
"""Benchmark of the periodic operator (periodizing operator + near-image P2P).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]

One step = one full application of the operator (prep, far field through
the periodizing operator, near-image P2P, combine) to the workload's
synthetic inputs, already resident on the GPU.  Default workload: 2D doubly
periodic Laplace, cell e1 = (16, 0), e2 = (0, 1), 1e5 sources from an
8-component Gaussian mixture (sigma 0.02 per fractional axis), zero net
charge, targets = sources, potential + gradient, mixed precision at
tol 1e-6, far field through the NUFFT path (ES width 8, 8 GL lines).

Metric: targets+sources per second = (N_S + N_T) / time per step, summed over
ranks (each rank runs its own independent cell: weak scaling, no
collective on the data path).  L2 is flushed (256 MiB write) before every
timed step; the flush is outside the timed events.

--impl reference times the FP64 CPU oracle (the plain method of the paper
plus the direct near sum) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "laplace_aspect16_gmm_n1e5"
METRIC = "targets+sources/s of periodic Laplace/Stokes op, mixed vs FP64 at rel err 1e-6"
SM_MAX_MHZ_FALLBACK = 2070.0  # GB300 maximum SM clock, used only if neither nvidia-smi nor MEASURED_PEAKS.json has it


def device_sms(dev):
    """Streaming multiprocessors of the benchmarked device (read from the device)."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def peak_clock_mhz(clocks):
    """SM clock for per-clock peaks: the median SM clock sampled under load
    during the timed region (so a box held below its maximum clock is not
    charged for it), else the maximum SM clock nvidia-smi reports, else the
    measured maximum, else the GB300 maximum."""
    if clocks and clocks.get("sm_mhz"):
        return float(clocks["sm_mhz"]), "median SM clock sampled during the timed region"
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"]), "maximum SM clock (nvidia-smi)"
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["sm_max_mhz"]), "maximum SM clock (MEASURED_PEAKS.json)"
    except Exception:
        return SM_MAX_MHZ_FALLBACK, "GB300 maximum SM clock (fallback)"

# Per-pair work of the near-image P2P, one pair = (target, source, near
# image): (FP32 operations, MUFU operations in units of the 16/clk/SM rate;
# ex2 runs at twice that rate and counts 1/2).  These are the operations of
# the implemented formulation: per-source image sums, then per (target,
# source) one log2 of a product of scaled r^2 and the strength FMAs, shared
# by the nimg images (9 for the doubly periodic 3 x 3 block, 15 with m0 = 2,
# 3 for the singly periodic strip); coordinate differences against a subtile
# centre.
#   Laplace pot + grad: per pair dx, dy, r^2 (2), product (2), sum dx/r^2, dy/r^2 (2) = 8
#                       and rcp; per (t, s) lg2 and 3 FMAs
#   Laplace pot:        per pair dx, dy, r^2 (2), product (2) = 6; per (t, s) lg2, 1 FMA
#   Stokes velocity:    per pair dx, dy, r^2 (2), product (2), dx^2 - dy^2 (2),
#                       sum cos 2t (1), sum sin t cos t (2) = 11 and rcp; per (t, s)
#                       lg2 and ~7 FP32 for the two components
#   mod. Helmholtz K0:  per pair dx, dy, x^2 (2), x, exponent, 7-term fit (6), two
#                       products, image sum = 13 (+3 without the beta scaling and
#                       folded fit variable: 16 counted), 2 rsqrt + ex2 (2.5 units);
#                       per (t, s) nrhs FMAs; with K1: + fit (6), scaling (2),
#                       two sums (2) per pair and 2 nrhs more FMAs per (t, s)
def p2p_work(kernel, nrhs, grad, nimg=9):
    # tree-code leaves (direct sums of neighbouring leaves, one pair per image):
    #   Laplace: dx, dy from hi/lo parts (6), r^2 (2), q lg2, q dx/r^2, q dy/r^2 (5) = 13; lg2 + rcp
    #   Stokes:  dx, dy (6), r^2 (2), d.f / r^2 (3), the two components (6) = 17; lg2 + rcp
    if kernel == "laplace_leaf":
        return (13.0, 2.0)
    if kernel == "stokes_leaf":
        return (17.0, 2.0)
    if kernel == "laplace":
        return (8.0 + 3.0 / nimg, 1.0 + 1.0 / nimg) if grad else (6.0 + 1.0 / nimg, 1.0 / nimg)
    if kernel == "stokes":
        return (11.0 + 7.0 / nimg, 1.0 + 1.0 / nimg)
    if kernel == "mstokes":
        # k_p2p_ms, x = beta r <= 2 branch: hi/lo differences 6, r^2 and x^2 3,
        # I0 / p1 / K0 / q1' polynomials 24, logs and E 5, A and B/r^2 3, the
        # 2 x 2 image sum 6, plus 4 FMAs per source and rhs; MUFU lg2 + rcp
        return (48.0 + 4.0 * nrhs / nimg, 2.0)
    if grad:
        return (26.0 + 3.0 * nrhs / nimg, 2.5)
    return (16.0 + nrhs / nimg, 2.5)


def alu_rates():
    """Results per clock per SM measured on this GPU model by an issue-rate
    probe (recorded in profiles/alu_peaks.json, method in profiles/alu_peaks.md):
    FP32 = scalar FFMA rate, MUFU = the lg2/rcp/rsqrt rate."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "alu_peaks.json")))
        return {"fp32": max(d["ffma"], d["ffma2_packed"]), "mufu": min(d["mufu_lg2"], d["mufu_rcp"], d["mufu_rsqrt"]),
                "source": "profiles/alu_peaks.json (measured)"}
    except Exception:
        return {"fp32": 128.0, "mufu": 16.0, "source": "fallback: nominal 128 FP32 / 16 MUFU per clock per SM"}


def p2p_roofline(kernel, nrhs, grad, pairs, launch_ms, step_ms, name, sms, clocks, traffic=None, nimg=9):
    """Bound = min(FP32 rate / FP32 ops per pair, MUFU rate / MUFU ops per pair)
    x SMs x SM clock (peak_clock_mhz); achieved = pairs per launch / launch time."""
    fp32_ops, mufu_ops = p2p_work(kernel, nrhs, grad, nimg)
    r = alu_rates()
    mhz, mhz_src = peak_clock_mhz(clocks)
    f_fp32 = r["fp32"] / fp32_ops
    f_mufu = r["mufu"] / mufu_ops
    peak = sms * min(f_fp32, f_mufu) * mhz * 1e6 / 1e9
    achieved = pairs / (launch_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_basis": (f"min(FP32 {r['fp32']:.1f}/clk/SM / {fp32_ops:.2f} ops, MUFU {r['mufu']:.1f}/clk/SM / "
                           f"{mufu_ops:.2f} ops) per pair x {sms} SMs x {mhz:.0f} MHz ({mhz_src}); "
                           f"{'FP32' if f_fp32 < f_mufu else 'MUFU'}-bound; rates from {r['source']}"),
            "pairs_per_launch": pairs, "launch_ms": launch_ms, "share_of_step": launch_ms / step_ms}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--path", default=None, help="override far-field path (direct|nufft)")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the FP64-path comparison run")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--scale", type=float, default=1.0, help="scale point counts (profiling on a small case)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--we", default=None, choices=["auto", "axis", "rotated"],
                    help="override the west/east plane-wave direction")
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: skip the batched modified-Helmholtz sub-records")
    ap.add_argument("--near", default="auto", choices=["auto", "direct", "fmm"],
                    help="near-image sum: direct P2P or the tree code (auto: the library's rule)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample), run in a single-threaded subprocess
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, %(root)r)
import workloads
from oracle import ewald, lattice, method, p1
w = workloads.make(%(name)r)
singly = w.get("singly", False)
if singly:
    cell = p1.canonical_strip(w["e1"], w["e2"])
    s, t = p1.wrap_strip(w["src"], cell), p1.wrap_strip(w["trg"], cell)
else:
    cell, s, t = lattice.to_canonical(w["e1"], w["e2"], w["src"], w["trg"])
kernel = w["kernel"]
beta = w.get("beta", 0.0)
vec = kernel in ("stokes", "mstokes")
q = w["q"]
if vec:
    q = np.einsum("ij,rjn->rin", cell["rot"], q)
res = []
rng = np.random.default_rng(%(seed)d)
for nsamp in %(samples)r:
    idx = rng.choice(t.shape[1], nsamp, replace=False)
    tt = t[:, idx]
    t0 = time.perf_counter()
    if singly:
        p1.near_sum(kernel, beta, cell, tt, s, q, want_grad=not vec)
    else:
        ewald.near_sum(kernel, beta, cell, tt, s, q, want_grad=not vec)
    t1 = time.perf_counter()
    if singly:
        p1.far_field(kernel, beta, cell, tt, s, q, eps=%(eps)r, want_grad=not vec)
    else:
        method.far_field(kernel, beta, cell, tt, s, q, eps=%(eps)r, want_grad=not vec)
    # (targets, near-sum seconds, far-field seconds)
    res.append((nsamp, t1 - t0, time.perf_counter() - t1))
print(json.dumps({"samples": res, "ns": int(s.shape[1]), "nt": int(t.shape[1])}))
"""


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def _fit_oracle(d):
    """Time per full workload from two target samples: the near sum has no
    source-side fixed cost (per-target time from the larger sample); the far
    field has one (coefficient formation over all sources): fixed + slope n,
    the slope clamped at >= 0 against timing noise."""
    (n1, a1, f1), (n2, a2, f2) = d["samples"]
    per_near = a2 / n2
    slope = max(0.0, (f2 - f1) / (n2 - n1))
    fixed = max(0.0, f1 - slope * n1)
    return fixed, per_near + slope


def oracle_time(name, samples=(32, 256), eps=1e-6, procs=1):
    """The FP64 oracle (plain method far field at eps + direct near sum), each
    process single-threaded, on `samples` sampled targets and all sources.
    procs > 1 runs that many such processes at once (distinct target samples),
    one per host core: the oracle's work over targets is independent, so the
    all-core time of the workload is fixed + per_target * N_T / procs with the
    per-target and fixed costs measured under the concurrent load."""
    env = _oracle_env()
    runs = []
    for k in range(procs):
        code = ORACLE_SNIPPET % dict(root=ROOT, name=name, samples=list(samples), eps=eps, seed=123 + k)
        runs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                     text=True, env=env))
    t0 = time.perf_counter()
    outs = [r.communicate(timeout=1800) for r in runs]
    wall = time.perf_counter() - t0
    fits, d = [], None
    for r, (out, err) in zip(runs, outs):
        if r.returncode != 0:
            raise RuntimeError(err[-2000:])
        d = json.loads(out.strip().splitlines()[-1])
        fits.append(_fit_oracle(d))
    fixed = statistics.median(f for f, _ in fits)
    per_target = statistics.mean(p for _, p in fits)
    t_full = fixed + per_target * d["nt"] / procs
    return dict(t_full=t_full, per_target=per_target, fixed=fixed, ns=d["ns"], nt=d["nt"], wall=wall,
                samples=list(samples), procs=procs)


def cpu_baseline(name, unit="targets+sources/s"):
    """The oracle timed single-threaded and on all host cores (see oracle_time)."""
    ot1 = oracle_time(name)
    n = host_cores()
    otn = oracle_time(name, procs=n) if n > 1 else None
    return cpu_baseline_obj(name, ot1, unit, otn)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_obj(name, ot1, unit, otn=None):
    """ot1: the oracle single-threaded; otn: on all host cores (or None)."""
    one = (ot1["ns"] + ot1["nt"]) / ot1["t_full"]
    base = (f"FP64 oracle (plain method, eps 1e-6 far field + direct near sum), one thread per process, on all "
            f"{ot1['ns']} sources and {ot1['samples'][0]} / {ot1['samples'][1]} sampled targets; time extrapolated "
            f"linearly to {ot1['nt']} targets (single thread: {ot1['wall']:.1f} s)")
    if otn is None:
        return {"value": one, "unit": unit, "cores": 1, "kind": "oracle", "sample": base,
                "single_thread_value": one}
    alln = (otn["ns"] + otn["nt"]) / otn["t_full"]
    return {"value": alln, "unit": unit, "cores": otn["procs"], "kind": "oracle",
            "sample": base + (f"; all cores: {otn['procs']} such processes at once on distinct target samples "
                              f"({otn['wall']:.1f} s), targets split over the processes"),
            "single_thread_value": one, "all_cores_value": alln, "nproc": host_cores()}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample of the workload (all sources, 4 / 12 sampled targets,
    single-threaded), extrapolated to the whole workload."""
    if rank != 0:
        return 0
    vals = []
    ot = None
    for _ in range(args.warmup + args.steps):
        ot = oracle_time(args.workload, samples=(4, 12))
        vals.append((ot["ns"] + ot["nt"]) / ot["t_full"])
    v = statistics.median(vals[args.warmup:])
    cb = cpu_baseline_obj(args.workload, ot, "targets+sources/s")
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "targets+sources/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ot["t_full"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "targets+sources/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def start_clocks(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def stop_clocks(proc, f, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in open(path):
        p = [x.strip() for x in ln.split(",")]
        if len(p) < 9 or p[0] != str(gpu_index):
            continue
        try:
            sm.append(float(p[1]))
            mx = float(p[2])
        except ValueError:
            continue
        for n, v in zip(names, p[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    loaded = [x for x in sm if x > 0.5 * (mx or SM_MAX_MHZ_FALLBACK)] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel_file, key):
    """DRAM bytes per launch from the committed ncu summary, if it still
    matches the kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_counters.json")
    try:
        d = json.load(open(path))
        rec = d[key]
        h = hashlib.sha256(open(os.path.join(ROOT, kernel_file), "rb").read()).hexdigest()[:16]
        if rec.get("source_sha") != h:
            return None
        return rec.get("dram_bytes_per_launch")
    except Exception:
        return None


BATCH_ORACLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, %(root)r)
import workloads
from oracle import ewald, lattice, method
cells = workloads.batch_cells(ncell=256, seed=3, nrhs=8)
counts = np.array([c["src"].shape[1] for c in cells])
order = np.argsort(counts)
pick = [int(order[int(f * (len(order) - 1))]) for f in %(quantiles)r]
rng = np.random.default_rng(5)
res = []
for c in pick:
    cell = cells[c]
    cl, s, t = lattice.to_canonical(cell["e1"], cell["e2"], cell["src"], cell["src"])
    idx = rng.choice(s.shape[1], %(ntarg)d, replace=False)
    t0 = time.perf_counter()
    ewald.near_sum("modhelm", %(beta)r, cl, t[:, idx], s, cell["q"], want_grad=False)
    method.far_field("modhelm", %(beta)r, cl, t[:, idx], s, cell["q"], eps=1e-7, want_grad=False)
    res.append((int(s.shape[1]), %(ntarg)d, time.perf_counter() - t0))
print(json.dumps({"samples": res, "sum_n2": float(np.sum(counts.astype(float) ** 2)), "sum_n": int(counts.sum())}))
"""


def batch_oracle_time(beta, quantiles=(0.25, 0.5, 0.75, 0.9), ntarg=12):
    """FP64 oracle on a bounded sample of the batch: ntarg targets in each of a
    few cells (quantiles of N), all their sources, 8 rhs; the cost per
    (target, source) is extrapolated to sum_c N_c^2 (targets = sources)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = BATCH_ORACLE_SNIPPET % dict(root=ROOT, quantiles=list(quantiles), ntarg=ntarg, beta=beta)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    work = sum(n * k for n, k, _ in d["samples"])
    wall = sum(t for _, _, t in d["samples"])
    t_full = wall / work * d["sum_n2"]
    return {"value": 2 * d["sum_n"] / t_full, "unit": "targets+sources/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle (near sum + plain far field, 8 rhs) for {ntarg} targets in each of "
                       f"{len(d['samples'])} cells (N = {', '.join(str(n) for n, _, _ in d['samples'])}; "
                       f"{wall:.1f} s); cost per (target, source) extrapolated to sum_c N_c^2")}


def init_dist(world, dev):
    """One process per GPU (torchrun): NCCL for the barrier and the max over
    ranks only; no collective on the data path (every rank runs its own cells)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if dev.type == "cuda":
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, x, dev):
    """The slowest rank's time (the job ends when it does)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, seconds):
    """Whole-job throughput: every rank processes units_per_rank units (weak
    scaling), and the job takes the max-over-ranks time."""
    return world * units_per_rank / seconds


def timed_region(step, args, dist, dev, local, after=None):
    """W untimed steps, then K steps timed with CUDA events on the launching
    stream (L2 flushed by a 256 MiB write before each, outside the events),
    with a barrier + synchronize on both sides; clocks sampled meanwhile.
    after(): called after each timed step, outside the events (reads phase
    events recorded by the step).  Returns (mean ms per step, max over ranks;
    clocks)."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk_path = os.path.join(tempfile.gettempdir(), f"pfmm_clocks_{os.getpid()}.csv")
    proc, fh = start_clocks(clk_path)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
        if after:
            after()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = stop_clocks(proc, fh, clk_path, local)
    return max_over_ranks(dist, sum(ts) / len(ts), dev), clocks


def far_units(kernel, cells, beta, nrhs, tol=1e-6):
    """Far-field work of a batch from each cell's plan (host only): the
    (target, term) pairs of the direct evaluation and the (source, term) pairs
    of the direct formation (the south/north terms of cells on the NUFFT path
    go through the transforms instead), and the number of NUFFT cells."""
    import ctypes
    from paper_2111_01083_gb300 import _lib
    from paper_2111_01083_gb300.periodic import _opts
    L = _lib.lib()
    ev = fo = nnu = 0
    for c in cells:
        n = int(c["src"].shape[1])
        o = _opts(kernel, c["e1"], c["e2"], beta, tol, "mixed", "auto", 0, 0, nrhs, 0)
        h = ctypes.c_void_p()
        _lib.check(L.pfmm_plan_create(ctypes.byref(o), n, n, ctypes.byref(h)))
        d = _lib.PlanDesc()
        try:
            _lib.check(L.pfmm_plan_describe(h, ctypes.byref(d)))
        finally:
            L.pfmm_plan_destroy(h)
        nsn = (d.M - (0 if d.mode0 else 1) + 1) if d.M > 0 else 0
        nufft = d.path == 2
        nterm = 2 * d.Nq + (0 if nufft else 2 * nsn)
        ev += n * nterm
        fo += n * nterm
        nnu += int(nufft)
    return ev, fo, nnu


def time_batch(beta, args, dist, dev, local, scale=1.0):
    """The batched modified-Helmholtz workload at one beta: 256 cells, 8 rhs,
    captured in one CUDA graph; each timed step is one graph.replay().  The
    graph carries external event-record nodes around the per-cell phases and
    the batched P2P, so the P2P time of every timed replay is read from the
    replay itself.  Evaluated pairs and the launch count come from one eager
    execute with pair counting after the timing (the counters add atomics)."""
    import numpy as np
    import torch
    import workloads
    from paper_2111_01083_gb300 import BatchOp
    cells = workloads.batch_cells(ncell=256, seed=3, nrhs=8, scale=scale)
    counts = [c["src"].shape[1] for c in cells]
    S_h = torch.from_numpy(np.ascontiguousarray(np.concatenate([c["src"] for c in cells], axis=1))).pin_memory()
    Q_h = torch.from_numpy(np.ascontiguousarray(np.concatenate([c["q"] for c in cells], axis=1))).pin_memory()
    S = S_h.to(dev)
    Q = Q_h.to(dev)
    op = BatchOp("modhelm", [dict(e1=c["e1"], e2=c["e2"], beta=beta) for c in cells], counts, precision="mixed",
                 nrhs=8, tol=1e-6)
    op.profile(True, count_pairs=False)
    graph, out = op.capture(S, Q, grad=False)
    torch.cuda.synchronize()
    op.status(dev)
    phases = []
    ms, clocks = timed_region(graph.replay, args, dist, dev, local, after=lambda: phases.append(op.phase_ms()))
    cell_ms = statistics.mean(p[0] for p in phases)
    p2p_ms = statistics.mean(p[1] for p in phases)
    op.profile(True, count_pairs=True)
    op(S, Q, out=out, grad=False)
    _, _, nlaunch, evaluated = op.phase_ms()
    # counters off again (an eager execute switches them); profiling stays on:
    # the graph's event nodes record into the profiling events, which must
    # outlive every replay
    op.profile(True, count_pairs=False)
    op(S, Q, out=out, grad=False)
    torch.cuda.synchronize()
    ns = int(sum(counts))
    sms = device_sms(dev)
    # the periodizing operator's direct formation and evaluation work against
    # the FP32 bound: per (point, term) 2 FMAs per rhs and ~6 FP32 operations
    # for the plane wave; the time is that of all per-cell phases (preparation,
    # formation, weights, evaluation, NUFFT stages), so the fraction is a lower
    # bound for the two kernels
    ev_u, fo_u, nnu = far_units("modhelm", cells, beta, 8)
    mhz, _ = peak_clock_mhz(clocks)
    fp32_per_unit = 2.0 * 8 + 6.0
    far_peak = sms * alu_rates()["fp32"] / fp32_per_unit * mhz * 1e6
    far = {"eval_units": ev_u, "form_units": fo_u, "nufft_cells": nnu, "per_cell_phases_ms": cell_ms,
           "units_per_s": (ev_u + fo_u) / (cell_ms * 1e-3) if cell_ms > 0 else None,
           "fp32_bound_units_per_s": far_peak,
           "frac_of_fp32_bound": ((ev_u + fo_u) / (cell_ms * 1e-3) / far_peak) if cell_ms > 0 else None,
           "basis": "units = (target, term) pairs of the direct evaluation + (source, term) pairs of the direct "
                    "formation over all cells; 2 FMA per rhs (8 rhs) + 6 FP32 for the plane wave per unit; "
                    "time = all per-cell phases"}
    rec = {"beta": beta, "ms_per_step": ms, "targets+sources/s": 2 * ns / (ms * 1e-3),
           "phases_ms": {"per_cell_prep_and_far_field": cell_ms, "batched_p2p": p2p_ms,
                         "measured": "CUDA events inside the replayed graph, mean over the timed replays"},
           "near_block_pairs": int(sum(9 * n * n for n in counts)), "near_pairs_evaluated": evaluated,
           "roofline": p2p_roofline("modhelm", 8, False, evaluated, p2p_ms, ms,
                                    "k_p2p_batch (persistent batched near-image P2P, modified Helmholtz; "
                                    "pairs = those evaluated: triples beyond the K0 cutoff are skipped)", sms, clocks),
           "far_field": far, "clocks": clocks, "gpu_launches_per_step": nlaunch, "n_sources_total": ns}
    # the operator owns the graph's workspace and phase events: it must live as
    # long as the graph is replayed
    return rec, dict(S=S, Q=Q, S_h=S_h, Q_h=Q_h, graph=graph, out=out, ns=ns, counts=counts, op=op)


def run_batch(args, rank, world, local):
    """Batched modified Helmholtz: 256 cells (eta = 1, d log-uniform in [1, 64],
    N log-uniform in [500, 5e4]), 8 rhs, one beta per run, the whole batch
    captured in one CUDA graph and replayed per step."""
    import torch
    beta = float(args.workload.split("beta")[-1])
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, dev)
    rec, bufs = time_batch(beta, args, dist, dev, local, scale=args.scale)
    S, Q, S_h, Q_h, graph, out, ns = (bufs[k] for k in ("S", "Q", "S_h", "Q_h", "graph", "out", "ns"))
    counts = bufs["counts"]
    ms, clocks = rec["ms_per_step"], rec["clocks"]
    pairs, evaluated, nlaunch = rec["near_block_pairs"], rec["near_pairs_evaluated"], rec["gpu_launches_per_step"]

    # end to end: pinned host inputs -> device, graph replay, potentials -> pinned host
    pot_h = torch.empty(tuple(out[0].shape), dtype=torch.float64).pin_memory()
    cur = torch.cuda.current_stream(dev)
    e2e_t = []
    for _ in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.copy_(S_h, non_blocking=True)
        Q.copy_(Q_h, non_blocking=True)
        graph.replay()
        pot_h.copy_(out[0], non_blocking=True)
        cur.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(dist, statistics.median(e2e_t[1:]), dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu and args.scale == 1.0:
        try:
            cpu = batch_oracle_time(beta)
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[:200]}
    line = {"metric": METRIC, "value": job_value(world, 2 * ns, ms * 1e-3), "unit": "targets+sources/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc", "data": "synthetic",
            "config": {"workload": args.workload if args.scale == 1.0 else f"{args.workload}@scale{args.scale}",
                       "kernel": "modhelm", "beta": beta, "ncell": 256, "nrhs": 8,
                       "n_sources_total": ns, "targets_are_sources": True, "near_block_pairs": pairs,
                       "near_pairs_evaluated": evaluated,
                       "execution": "one CUDA graph per step (per-cell far field + one persistent P2P kernel)",
                       "l2": "flushed (256 MiB write) before each timed step", "parallelism": f"replicas{world}"},
            "phases_ms": rec["phases_ms"],
            "roofline": rec["roofline"],
            "cpu_baseline": cpu, "clocks": clocks,
            "e2e": {"value": job_value(world, 2 * ns, e2e_s), "unit": "targets+sources/s",
                    "h2d_bytes_per_step": S_h.numel() * 8 + Q_h.numel() * 8, "d2h_bytes_per_step": pot_h.numel() * 8,
                    "api": "BatchOp CUDA-graph replay with pinned host copies in the timed region"},
            "gpu_launches": nlaunch * args.steps}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_adjoint(args, rank, world, local):
    """Differentiation workload: E = 1/2 sum q_i phi(x_i) (Laplace, targets =
    sources); one step = forward operator + backward (dE/dq and the forces
    dE/dx through pfmm_execute_adjoint)."""
    import torch
    import workloads
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, dev)
    w = workloads.make(args.workload, scale=args.scale)
    n = w["src"].shape[1]
    S_h = torch.from_numpy(w["src"]).pin_memory()
    Q_h = torch.from_numpy(w["q"]).pin_memory()
    S = S_h.to(dev).requires_grad_(True)
    Q = Q_h.to(dev).requires_grad_(True)
    op = PeriodicOp("laplace", w["e1"], w["e2"], tol=w["tol"], precision="mixed", ns_max=n, nt_max=n)

    def step():
        S.grad = None
        Q.grad = None
        pot, _ = periodic(op, S, Q)
        (0.5 * (Q * pot).sum()).backward()

    step()
    torch.cuda.synchronize()
    op.status()
    ms, clocks = timed_region(step, args, dist, dev, local)
    # the adjoint execute is the last one of a step: its near-field phase (the
    # direct P2P, or the tree code's leaf kernels and the pairs they sum) and
    # launch count
    op.profile(True)
    p2p, nl, leaves, lpairs = [], [], [], []
    for _ in range(3):
        step()
        ph = op.phase_ms(sub=True)
        p2p.append(ph[2])
        leaves.append(ph[7])
        nl.append(op.describe()["nlaunch"])
        if op.describe()["near_fmm"]:
            lpairs.append(op.pairs())
    op.profile(False)
    desc = op.describe()
    p2p_ms = statistics.median(p2p)
    nimg = 3 * (2 * desc["m0"] + 1)
    if desc["near_fmm"]:
        roof = p2p_roofline("laplace_leaf", 1, True, statistics.median(lpairs), statistics.median(leaves), ms,
                            f"k_fmm_p2p + k_fmm_l2p (tree-code leaves of the adjoint execute: direct sums of "
                            f"neighbouring leaves and L2P, {nimg} images)", device_sms(dev), clocks, nimg=nimg)
    else:
        roof = p2p_roofline("laplace", 1, True, desc["npairs"], p2p_ms, ms,
                            "k_p2p_mixed (near-image P2P of the adjoint execute)", device_sms(dev), clocks, nimg=nimg)
    # end to end: pinned host inputs -> device, forward + backward, gradients -> pinned host
    dq_h = torch.empty((1, n), dtype=torch.float64).pin_memory()
    dx_h = torch.empty((2, n), dtype=torch.float64).pin_memory()
    cur = torch.cuda.current_stream(dev)
    e2e_t = []
    for _ in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.no_grad():
            S.copy_(S_h, non_blocking=True)
            Q.copy_(Q_h, non_blocking=True)
        step()
        dq_h.copy_(Q.grad, non_blocking=True)
        dx_h.copy_(S.grad, non_blocking=True)
        cur.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(dist, statistics.median(e2e_t[1:]), dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu and args.scale == 1.0:
        try:
            cpu = cpu_baseline(args.workload)
            cpu["sample"] += "; one oracle evaluation (potential + gradient) gives dE/dq and dE/dx"
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[:200]}
    line = {"metric": METRIC, "value": job_value(world, 2 * n, ms * 1e-3), "unit": "targets+sources/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc", "data": "synthetic",
            "config": {"workload": args.workload if args.scale == 1.0 else f"{args.workload}@scale{args.scale}",
                       "kernel": "laplace", "n": n, "step": "forward + backward (dE/dq, dE/dx)",
                       "l2": "flushed (256 MiB write) before each timed step", "parallelism": f"replicas{world}"},
            "roofline": roof,
            "cpu_baseline": cpu, "clocks": clocks,
            "e2e": {"value": job_value(world, 2 * n, e2e_s), "unit": "targets+sources/s",
                    "h2d_bytes_per_step": S_h.numel() * 8 + Q_h.numel() * 8,
                    "d2h_bytes_per_step": dq_h.numel() * 8 + dx_h.numel() * 8,
                    "api": "periodic() autograd forward + backward with pinned host copies in the timed region"},
            "gpu_launches": None}
    # forward + adjoint executes per step (the adjoint adds one contraction kernel)
    line["gpu_launches"] = args.steps * (2 * nl[-1] + 1)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload.startswith("batch_modhelm_beta"):
        return run_batch(args, rank, world, local)
    if "adjoint" in args.workload:
        return run_adjoint(args, rank, world, local)

    import numpy as np
    import torch
    import workloads
    from paper_2111_01083_gb300 import PeriodicOp
    from paper_2111_01083_gb300.build import LIB, build_library

    if not os.path.exists(LIB):
        build_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, dev)

    w = workloads.make(args.workload, scale=args.scale)
    cfg = dict(workloads.CONFIGS[args.workload])
    path = args.path or cfg.get("path", "auto")
    kernel = w["kernel"]
    self_t = w["trg"] is w["src"]
    S = torch.tensor(w["src"], device=dev)
    Q = torch.tensor(w["q"], device=dev)
    T = None if self_t else torch.tensor(w["trg"], device=dev)
    ns = S.shape[1]
    nt = ns if self_t else T.shape[1]
    grad = kernel not in ("stokes", "mstokes")
    singly = cfg.get("singly", False)
    we = args.we or cfg.get("we", "auto")
    beta = cfg.get("beta", 0.0)
    nrhs = int(Q.shape[0])
    op = PeriodicOp(kernel, w["e1"], w["e2"], beta=beta, tol=cfg["tol"], precision="mixed", path=path,
                    nufft_w=cfg.get("nufft_w", 0), n_gl=cfg.get("n_gl", 0), ns_max=ns, nt_max=nt, singly=singly,
                    we=we, nrhs=nrhs, near=args.near)
    op.profile(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = op(S, Q, T, grad=grad)
    torch.cuda.synchronize()
    op.status()
    # eager executes (one library call per step), for reference
    eager = []
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        op(S, Q, T, grad=grad, out=out)
        e1.record()
        e1.synchronize()
        eager.append(e0.elapsed_time(e1))
    eager_ms = statistics.median(eager[1:])
    nlaunch_step = op.describe()["nlaunch"]
    # the timed step: one replay of the execute captured in a CUDA graph (the
    # many small launches of the tree code and the far field are replayed
    # without per-launch host overhead); phases from the graph's event nodes
    graph, out = op.capture(S, Q, T, grad=grad, out=out)
    for _ in range(max(0, args.warmup - 1)):
        graph.replay()
    torch.cuda.synchronize()
    op.status()

    clk_path = os.path.join(tempfile.gettempdir(), f"pfmm_clocks_{os.getpid()}.csv")
    proc, fh = start_clocks(clk_path)
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, p2p_ms, far_ms, sub_ms = [], [], [], []
    launches = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ph = op.phase_ms(sub=True)
        far_ms.append(ph[1])
        p2p_ms.append(ph[2])
        sub_ms.append(ph[3:])
        launches += nlaunch_step
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = stop_clocks(proc, fh, clk_path, local)
    op.status()
    ms = max_over_ranks(dist, sum(step_ms) / len(step_ms), dev)
    value = job_value(world, ns + nt, ms * 1e-3)
    desc = op.describe()

    # end to end: host arrays through pfmm_execute_host (pinned), copies inside the timed region
    src_h = torch.from_numpy(w["src"]).pin_memory()
    q_h = torch.from_numpy(w["q"]).pin_memory()
    trg_h = src_h if self_t else torch.from_numpy(w["trg"]).pin_memory()
    pot_h = torch.empty(tuple(out[0].shape), dtype=torch.float64).pin_memory()
    grad_h = torch.empty(tuple(out[1].shape), dtype=torch.float64).pin_memory() if grad else None
    op.execute_host_ptrs(src_h, q_h, trg_h, pot_h, grad_h)
    e2e_t = []
    for _ in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.execute_host_ptrs(src_h, q_h, trg_h, pot_h, grad_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(dist, statistics.median(e2e_t), dev)
    h2d = src_h.numel() * 8 + q_h.numel() * 8 + (0 if self_t else trg_h.numel() * 8)
    d2h = pot_h.numel() * 8 + (grad_h.numel() * 8 if grad else 0)

    # accuracy: mixed vs the FP64 GPU path on the same input (outside the timed region)
    acc = None
    if not args.skip_fp64 and rank == 0:
        op64 = PeriodicOp(kernel, w["e1"], w["e2"], beta=beta, tol=1e-10, precision="fp64", path="direct",
                          ns_max=ns, nt_max=nt, singly=singly, we=we, nrhs=nrhs)
        op64.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ref = op64(S, Q, T, grad=grad)
        e1.record()
        e1.synchronize()
        op64.status()

        def rel(a, b, mc):
            a = a.double()
            b = b.double()
            if mc:
                a = a - a.mean(-1, keepdim=True)
                b = b - b.mean(-1, keepdim=True)
            return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        acc = {"fp64_gpu_ms_per_step": e0.elapsed_time(e1),
               "rel_err_pot_vs_fp64": rel(out[0], ref[0], kernel in ("laplace", "stokes")),
               "rel_err_grad_vs_fp64": rel(out[1], ref[1], False) if grad else None,
               "fp64_gpu_value": (ns + nt) / (e0.elapsed_time(e1) * 1e-3)}
        del op64, ref

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    # roofline of the dominant kernel: pairs per launch / event time
    p2p = sum(p2p_ms) / len(p2p_ms)
    nimg = 3 if singly else 3 * (2 * desc["m0"] + 1)
    near_sub, near_stats = None, None
    if desc["near_fmm"]:
        names = ["tree", "upward", "traversal", "downward", "leaves"]
        near_sub = {k: sum(x[i] for x in sub_ms) / len(sub_ms) for i, k in enumerate(names)}
        near_stats = op.near_stats()
        # the tree code's leaf kernel (L2P + direct sums of neighbouring leaves);
        # its pairs are the ones it sums directly (counted while profiling)
        npairs = op.pairs()
        roof = p2p_roofline(f"{kernel}_leaf", nrhs, grad, npairs, near_sub["leaves"], ms,
                            f"k_fmm_p2p + k_fmm_l2p (tree-code leaves: direct sums of neighbouring leaves and L2P, "
                            f"{nimg} images)",
                            device_sms(dev), clocks, None, nimg=nimg)
    else:
        kname = {"mstokes": "k_p2p_ms", "modhelm": "k_p2p_mixed_mh"}.get(kernel, "k_p2p_mixed")
        # modified Helmholtz skips (target block, source tile, image) triples beyond
        # the K0 cutoff: its roofline counts the pairs it evaluates
        npairs = op.pairs() if kernel == "modhelm" else desc["npairs"]
        roof = p2p_roofline(kernel, nrhs, grad, npairs, p2p, ms, f"{kname} (near-image P2P, {nimg} images)",
                            device_sms(dev), clocks,
                            traffic_for("paper_2111_01083_gb300/csrc/p2p.cu", f"{kname}_{args.workload}"), nimg=nimg)
    cpu = None
    if world == 1 and not args.no_cpu and args.scale == 1.0:
        try:
            cpu = cpu_baseline(args.workload)
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[:200]}
    # the batched workload (256 cells, 8 rhs) at each beta, graph-replay timed,
    # as sub-records of the default line
    batch = None
    if world == 1 and args.workload == WORKLOAD and args.scale == 1.0 and not args.no_batch:
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup = max(3, min(args.steps, 5)), 3
        batch = {"workload": "batch_modhelm (256 cells, N log-uniform in [500, 5e4], aspect log-uniform in [1, 64], "
                             "8 rhs, tol 1e-6, mixed)", "steps": sub.steps, "warmup": sub.warmup,
                 "l2": "flushed (256 MiB write) before each timed replay"}
        for b in (1.0, 10.0, 100.0):
            try:
                rec, bufs = time_batch(b, sub, None, dev, local)
                del bufs
                batch[f"beta{int(b)}"] = rec
            except Exception as e:  # reported, not fatal
                batch[f"beta{int(b)}"] = {"error": str(e)[:300]}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": value, "unit": "targets+sources/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64acc", "data": "synthetic",
        "config": {"workload": args.workload if args.scale == 1.0 else f"{args.workload}@scale{args.scale}",
                   "kernel": kernel, "e1": list(w["e1"]), "e2": list(w["e2"]),
                   "n_sources": ns, "n_targets": nt, "targets_are_sources": self_t, "nrhs": nrhs,
                   "dist": cfg.get("dist"), "tol": cfg["tol"], "path": ["direct", "direct", "nufft"][desc["path"]],
                   "nufft_w": desc["nufft_w"], "n_gl": desc["n_gl"], "M": desc["M"], "Nq": desc["Nq"],
                   "m0": desc["m0"], "outputs": "pot+grad" if grad else "velocity",
                   "periodicity": "singly (e1)" if singly else "doubly",
                   "west_east": "rotated (e2-perp)" if desc["we_rotated"] else "axis (e1)",
                   "l2": "flushed (256 MiB write) before each timed step", "parallelism": f"replicas{world}"},
        "phases_ms": {"far_field": sum(far_ms) / len(far_ms), "near_field": p2p},
        "execution": "CUDA-graph replay of one execute per step (PeriodicOp.capture)",
        "eager_ms_per_step": eager_ms,
        "near_field": {"method": "tree code" if desc["near_fmm"] else "direct P2P", "phases_ms": near_sub,
                       "stats": near_stats, "order": desc["near_order"] if desc["near_fmm"] else None,
                       "leaf": desc["near_leaf"] if desc["near_fmm"] else None},
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "e2e": {"value": job_value(world, ns + nt, e2e_s), "unit": "targets+sources/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "pfmm_execute_host (pinned host buffers)"},
        "gpu_launches": launches, "accuracy": acc,
    }
    if batch is not None:
        line["batch_modhelm"] = batch
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
