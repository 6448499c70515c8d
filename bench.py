#!/usr/bin/env python
"""Benchmark of the GB300 HISQ path: mixed-precision multi-right-hand-side CG on
A = m^2 - D_eo D_oe to the true residual 1e-10 at the production shape, with the roofline of its
dominant kernel measured live and the plain FP64 single-RHS CG beside it.

One step = one `hisq_cg_solve` of 16 Z2-noise right-hand sides on the 64^3 x 16 lattice
(m = 0.002): links and vectors stored in FP16 with FP32 arithmetic, bundles that share every link
read (size from the autotuner), FP64-accurate reliable updates every 10x residual drop (double-
single arithmetic on the FP32 pipe), every right-hand side to the FP64 true residual 1e-10.  Link
reads, both Dslash halves, the fused BLAS-1, the residual recomputations and the per-RHS control
all run inside it.  The line also carries the same figures for the 32^3 x 8 single-RHS solve.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own right-hand sides on its own GPU (independent
replicas: no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HISQ Dslash GFlop/s & HBM GB/s; CG s/RHS to res 1e-10 vs plain FP64 CG"
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
TOL = 1e-10
# lattice and mass of each mode when --dims / --mass are not given
MODE_DEFAULTS = {"cg": ("64,64,64,16", 0.002), "production": ("64,64,64,16", 0.002),
                 "batch": ("48,48,48,12", 0.002), "learned": ("32,32,32,8", 0.005),
                 "sweep": ("32,32,32,8", 0.01), "multishift": ("32,32,32,8", 0.01),
                 "trace": ("32,32,32,8", 0.01), "dslash": ("32,32,32,8", 0.01), "slabs": ("64,64,64,16", 0.002)}
DEFAULT_DELTA = {"fp32": 0.01, "fp16": 0.03, "bf16": 0.1}  # the library's reliable-update threshold by storage
SMALL_DIMS, SMALL_MASS = (32, 32, 32, 8), 0.01   # the single-RHS precision-form solve (extra keys)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="fp16", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--dims", default=None)
    ap.add_argument("--mass", type=float, default=None)
    ap.add_argument("--step-rhs", type=int, default=16, help="cg: right-hand sides solved per step")
    ap.add_argument("--bundle", type=int, default=16,
                    help="cg: right-hand sides per bundle (0: chosen by the autotuner from the Dslash timings)")
    ap.add_argument("--rhs", default="z2", choices=["z2", "gaussian"], help="cg: kind of right-hand side")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="cg: only the timed region and its roofline (no comparators, no small lattice)")
    ap.add_argument("--mode", default="cg",
                    choices=["cg", "sweep", "learned", "batch", "production", "multishift", "trace", "dslash",
                             "slabs"],
                    help="cg: the benchmark line; sweep: Dslash throughput against the number of "
                         "right-hand sides; learned: the learned-preconditioner workload (32^3 x 8); "
                         "batch: bundles with uneven convergence (48^3 x 12); production: a sweep of "
                         "Z2-noise right-hand sides (64^3 x 16); multishift: eight shifted systems "
                         "from one multi-shift solve against separate solves (32^3 x 8); trace: the "
                         "stochastic Tr A^-1 of Eq. (2) from Z2 noise (32^3 x 8); dslash: one Dslash "
                         "configuration (--inner, --nrhs, --dims) launched --steps times (for profiling); slabs: the "
                         "Dslash decomposed into t-slabs with depth-3 halos against the undecomposed one")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--test-rhs", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--nrhs", type=int, default=1500, help="production: right-hand sides in the sweep")
    ap.add_argument("--pc", action="store_true", help="production: also train and apply the network")
    ap.add_argument("--recon", type=int, default=18, choices=[18, 13, 9],
                    help="dslash: reals stored per Naik link (13 and 9: reconstructed from SU(3) times a scale)")
    ap.add_argument("--shape", default=None,
                    help="dslash: launch shape R,threads,lanes (skips the autotuner, so that the only "
                         "Dslash launches are one warm-up and the --steps timed ones)")
    args = ap.parse_args()
    d_dims, d_mass = MODE_DEFAULTS[args.mode]
    if args.dims is None:
        args.dims = d_dims
    if args.mass is None:
        args.mass = d_mass
    return args


def workload(args):
    dims = [int(d) for d in args.dims.split(",")]
    n = args.step_rhs
    kind = "Z2-noise" if args.rhs == "z2" else "Gaussian"
    return dims, {
        "workload": f"{'x'.join(map(str, dims[:3]))}x{dims[3]} even-odd HISQ CG on m^2 - D_eo D_oe, m={args.mass}, "
                    f"{n} {kind} RHS per step in bundles of {args.bundle or 'autotuned size'} sharing every link "
                    f"read, {args.inner} storage / "
                    f"fp32 arithmetic, FP64-accurate reliable updates (delta {DEFAULT_DELTA.get(args.inner)}, double-single arithmetic on the "
                    f"FP32 pipe), FP64 true residual <= 1e-10 per RHS",
        "lattice": dims, "rhs_per_step": n, "rhs": kind, "mass": args.mass, "inner_storage": args.inner,
        "fields": "synthetic SU(3) fat links (eps 0.3, 5% noise) and Naik links, staggered phases and "
                  "antiperiodic t folded in; seeds 1/2/3; RHS seeds 60000+1000*rank+k",
        "l2": "inputs larger than L2 (links and vectors of this lattice: GBs) and L2 flushed between steps "
              "(512 MiB write)",
    }


def rhs_vector(hi, lat, kind, k, rank):
    seed = 60000 + 1000 * rank + k
    return hi.z2_rhs(lat, seed, seed_base=0) if kind == "z2" else hi.gaussian_rhs(lat, seed, seed_base=0)


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.5)
        return self

    def mark(self, start):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            out, _ = self.proc.communicate()
            self.lines = [l.strip() for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
            except ValueError:
                ts = None
            if ts is not None and self.t0 is not None and not (self.t0 - 1.0 <= ts <= self.t1 + 1.0):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(key):
    """DRAM bytes (read + write) per launch of the persistent solve kernel from the committed
    ncu summary, if that summary was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != kernel_source_hash():
        return None
    val = rec.get("per_launch_bytes", {}).get(key)
    return float(val) if val else None


KERNEL_SOURCES = ("cg_persistent.cuh", "cg_persistent_body.cuh", "dslash_kernel.cuh", "link_codec.cuh",
                  "hisq_internal.cuh", "solver_state.cuh", "ds_arith.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1409_1510_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------------------------
def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample(lat, o, b, mass, budget_s):
    """Time the FP64 oracle CG, as it stands, for as many iterations as fit in budget_s."""
    t = time.perf_counter()
    o.cg(b, mass, TOL, max_iter=1)
    per_iter = time.perf_counter() - t
    iters = max(1, min(500, int(budget_s / max(per_iter, 1e-6))))
    t = time.perf_counter()
    _, done, _ = o.cg(b, mass, TOL, max_iter=iters)
    el = time.perf_counter() - t
    if done > 0:  # converged before the budget: count the iterations it ran
        iters = done
    flops = (2 * 1146 + 72) * lat.half_volume * iters
    return flops / el / 1e9, iters, el


def cpu_baseline(lat, X, N, b, mass, budget_s=12.0):
    """The FP64 oracle CG on a bounded sample of the same solve: the OpenMP build on all host
    cores (the line's value) and the single-threaded build."""
    import oracle
    import oracle.build as obuild
    dims = list(lat.dims)
    cores = os.cpu_count() or 1
    o_all = oracle.Oracle(dims, X, N, so_path=obuild.build(output=obuild.LIBRARY_OMP, openmp=True))
    v_all, it_all, el_all = oracle_sample(lat, o_all, b, mass, budget_s)
    o_one = oracle.Oracle(dims, X, N)
    v_one, it_one, el_one = oracle_sample(lat, o_one, b, mass, budget_s)
    return {"value": v_all, "unit": "GFlop/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{it_all} iterations of the FP64 oracle CG on the same {dims} problem, one right-hand "
                      f"side ({el_all:.1f} s, {el_all / it_all * 1e3:.0f} ms/iteration, site loops of the Dslash "
                      f"on {cores} OpenMP threads)",
            "single_thread": {"value": v_one, "unit": "GFlop/s", "cores": 1,
                              "sample": f"{it_one} iterations ({el_one:.1f} s, {el_one / it_one * 1e3:.0f} "
                                        f"ms/iteration, one thread)"}}


def run_reference(args, rank):
    """Reference arm: the FP64 CPU oracle (OpenMP build, all host cores) on this workload's
    lattice, mass and right-hand-side kind, in the same metric and unit."""
    import hisq_inputs as hi
    import oracle
    import oracle.build as obuild
    dims, cfg = workload(args)
    if rank != 0:
        return
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    b = rhs_vector(hi, lat, args.rhs, 0, 0)
    cores = os.cpu_count() or 1
    o = oracle.Oracle(dims, X, N, so_path=obuild.build(output=obuild.LIBRARY_OMP, openmp=True))
    for _ in range(max(1, args.warmup)):
        oracle_sample(lat, o, b, args.mass, 0.0)
    per_step = 60.0 / max(1, args.steps)
    its, secs = 0, 0.0
    for _ in range(args.steps):
        _, i, el = oracle_sample(lat, o, b, args.mass, per_step)
        its += i
        secs += el
    value = its * (2 * 1146 + 72) * lat.half_volume / secs / 1e9
    sample = (f"{its} FP64 oracle CG iterations on the {dims} problem, one right-hand side, over {args.steps} "
              f"steps ({secs:.1f} s, Dslash site loops on {cores} OpenMP threads, {cpu_model()}); one bounded "
              f"sample per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "GFlop/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def combine_ranks(dist, total_ms, flops, launches, device):
    """Whole-job figures of the timed region: the slowest rank's time, and the flops and kernel
    launches summed over ranks (every rank solves its own right-hand sides).  dist = None: one rank."""
    if dist is None:
        return total_ms, flops, launches
    import torch
    t = torch.tensor([total_ms, flops, launches], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1]), float(t[2])


# ---------------------------------------------------------------------------------------------
def event_ms(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def dslash_rate(hisq, torch, hi, lat, fat, naik, prec, n, flush, stream, dev, d64, reps=10):
    """One Dslash of n right-hand sides with the autotuned shape: median CUDA-event time with the
    L2 flushed before every launch; GFlop/s and compulsory-byte GB/s."""
    from paper_1409_1510_gb300 import accounting as acc
    vin = torch.empty(hisq.hisq_vector_bytes(prec, n), dtype=torch.uint8, device=dev)
    hisq.hisq_pack(d64(np.stack([hi.gaussian_rhs(lat, 900 + k) for k in range(n)])), vin, n, prec)
    vout = torch.empty_like(vin)
    shape = hisq.hisq_autotune(fat, naik, n)
    hisq.hisq_dslash(fat, naik, vin, vout, n, 1)
    ts = []
    for i in range(reps):
        flush.zero_()
        ts.append(event_ms(torch, stream, lambda: hisq.hisq_dslash(fat, naik, vin, vout, n, i % 2)))
    sec = statistics.median(ts) / 1e3
    elem = {0: 8, 1: 4, 2: 2, 3: 2}[prec]
    byts = acc.compulsory_bytes(n, elem, elem, 18, 8.0 if prec in (2, 3) else 0.0, 4.0 if prec == 2 else 0.0)
    hbm_peak, _ = peaks()
    gbs = byts * lat.half_volume / sec / 1e9
    return {"nrhs": n, "us": sec * 1e6, "gflops": acc.DSLASH_FLOPS_PER_SITE * n * lat.half_volume / sec / 1e9,
            "hbm_gbs": gbs, "frac_hbm": gbs / hbm_peak, "compulsory_bytes_per_site": byts,
            "shape": {"rhs_per_thread": shape[0], "threads": shape[1], "lanes_per_site": shape[2]}}


def set_params(hisq, prec, driver=2, timing=0, bundle=0):
    # driver: 0 host-driven (CUDA events on every Dslash), 1 CUDA graph, 2 persistent kernel
    p = hisq.hisq_default_solver_params()
    p.inner_prec, p.use_graph, p.time_kernels, p.bundle = prec, driver, timing, bundle  # delta: by precision
    hisq.hisq_set_solver_params(p)


def solve_ms(hisq, torch, stream, fat, naik, bs, xs, mass, flush):
    """One hisq_cg_solve of the right-hand sides bs, L2 flushed before, CUDA events around it."""
    flush.zero_()
    torch.cuda.synchronize()
    ms = event_ms(torch, stream, lambda: hisq.hisq_cg_solve(fat, naik, bs, xs, mass, TOL))
    return ms, hisq.hisq_last_stats()


def small_lattice_figures(hisq, torch, hi, inner, stream, dev, flush):
    """The 32^3 x 8 precision-form solve (m = 0.01, one Gaussian right-hand side): mixed precision
    against plain FP64 CG, and a bundle of 16 right-hand sides against single solves."""
    lat = hi.Lattice(SMALL_DIMS)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    hisq.hisq_init(list(SMALL_DIMS), dev.index or 0, stream)
    try:
        fat = hisq.hisq_links_create(d64(X), False, inner, 18)
        naik = hisq.hisq_links_create(d64(N), True, inner, 18)
        b = [d64(hi.gaussian_rhs(lat, 0))]
        x = [torch.zeros_like(b[0])]
        out = {"lattice": list(SMALL_DIMS), "mass": SMALL_MASS, "rhs": "Gaussian"}
        for name, prec in (("mixed", inner), ("fp64", 0)):
            set_params(hisq, prec, 2, 1)
            for _ in range(3):
                solve_ms(hisq, torch, stream, fat, naik, b, x, SMALL_MASS, flush)
            runs = [solve_ms(hisq, torch, stream, fat, naik, b, x, SMALL_MASS, flush) for _ in range(7)]
            ms = statistics.median(r[0] for r in runs)
            st = runs[-1][1]
            ph = list(st.phase_ms)
            out[name] = {"ms_per_rhs": ms, "iterations": st.max_iterations, "reliable_updates": st.reliable_updates,
                         "recompute_share": ph[3] / st.solve_kernel_ms if st.solve_kernel_ms > 0 else None}
        out["speedup_vs_fp64_cg"] = out["fp64"]["ms_per_rhs"] / out["mixed"]["ms_per_rhs"]
        bs = [d64(hi.gaussian_rhs(lat, 100 + k)) for k in range(16)]
        xs = [torch.zeros_like(v) for v in bs]
        set_params(hisq, inner, 2, 0, 16)
        solve_ms(hisq, torch, stream, fat, naik, bs, xs, SMALL_MASS, flush)
        bms = [solve_ms(hisq, torch, stream, fat, naik, bs, xs, SMALL_MASS, flush)[0] for _ in range(3)]
        out["bundle_of_16"] = {"ms_per_rhs": statistics.median(bms) / 16,
                               "speedup_per_rhs_vs_single": out["mixed"]["ms_per_rhs"] / (statistics.median(bms) / 16)}
    finally:
        hisq.hisq_finalize()
    return out


def run_ours(args, rank, world, local_rank, dist):
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import accounting as acc
    from paper_1409_1510_gb300 import hisq

    dims, cfg = workload(args)
    mass, nstep = args.mass, args.step_rhs
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    lat = hi.Lattice(dims)
    Vh = lat.half_volume
    t0 = time.perf_counter()
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    t_fields = time.perf_counter() - t0

    def d64(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)

    hisq.hisq_init(dims, local_rank, stream)
    inner = PREC[args.inner]
    fat = hisq.hisq_links_create(d64(X), False, inner, 18)
    naik = hisq.hisq_links_create(d64(N), True, inner, 18)
    rhs_host = [rhs_vector(hi, lat, args.rhs, k, rank) for k in range(nstep)]
    bs = [d64(v) for v in rhs_host]
    xs = [torch.zeros_like(v) for v in bs]
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: tunes the Dslash launch shapes (and the bundle size with --bundle 0), first launches
    set_params(hisq, inner, 2, 1, args.bundle)
    for _ in range(args.warmup):
        solve_ms(hisq, torch, stream, fat, naik, bs, xs, mass, flush)

    # ---- the timed region: K steps of nstep right-hand sides (persistent driver; the solve
    # kernels and their phases timed on the solve's stream) ----
    with ClockSampler(local_rank) as clk:
        barrier()
        clk.mark(True)
        t_wall = time.perf_counter()
        ms, stats = [], []
        for _ in range(args.steps):
            m, st = solve_ms(hisq, torch, stream, fat, naik, bs, xs, mass, flush)
            ms.append(m)
            stats.append(st)
        barrier()
        t_wall = time.perf_counter() - t_wall
        clk.mark(False)
    iters = np.zeros(nstep, dtype=np.int32)
    res = np.zeros(nstep)
    last = hisq.hisq_last_stats(iters, res)
    total_ms = sum(ms)
    flops = sum(s.flops for s in stats)
    launches = sum(s.kernel_launches for s in stats)
    total_ms_max, flops_all, launches_all = combine_ranks(dist, total_ms, flops, launches, dev)
    value = flops_all / (total_ms_max / 1e3) / 1e9
    s_per_rhs = total_ms / 1e3 / (args.steps * nstep)

    # ---- roofline of the dominant kernel, the persistent solve kernel: algorithmic flops and
    # bytes of each launch over its CUDA-event duration (recorded by the library inside the timed
    # region), and the phase times from inside the kernel ----
    fp32_peak, fp64_peak = hisq.hisq_measure_fma_peaks()  # TFLOP/s, FMA chains on every SM
    hbm_peak, peak_kind = peaks()
    k_ms = sum(s.solve_kernel_ms for s in stats)
    k_n = sum(s.solve_kernel_launches for s in stats)
    k_flops = sum(s.flops + acc.recompute_flops(Vh, s.reliable_updates) for s in stats)
    k_bytes = sum(acc.bundle_solve_bytes(inner, Vh, s.total_iterations, s.bundle_iterations, s.reliable_updates,
                                         s.recompute_passes, s.nrhs) for s in stats)
    ph = [sum(s.phase_ms[i] for s in stats) for i in range(5)]
    tflops = k_flops / (k_ms / 1e3) / 1e12
    gbs = k_bytes / (k_ms / 1e3) / 1e9
    frac_alu, frac_hbm = tflops / fp32_peak, gbs / hbm_peak
    nb = last.bundle_size
    ds_its = sum(s.bundle_iterations for s in stats)
    ds_flops = sum(s.total_iterations for s in stats) * 2 * acc.DSLASH_FLOPS_PER_SITE * Vh
    phases = {"ms_per_launch": {name: ph[i] / max(k_n, 1) for i, name in
                                enumerate(("dslash_doe", "dslash_aop_dot", "pxr_update", "reliable_recompute"))},
              "dslash_phases_tflops": ds_flops / ((ph[0] + ph[1]) / 1e3) / 1e12 if ph[0] + ph[1] > 0 else None,
              "dslash_phases_gbs": ds_its * 2 * acc.LINK_BYTES_18[inner] * Vh / ((ph[0] + ph[1]) / 1e3) / 1e9
              if ph[0] + ph[1] > 0 else None,
              "recompute_share": ph[3] / k_ms if k_ms > 0 else None,
              "recompute_gflops": sum(acc.recompute_flops(Vh, s.reliable_updates) for s in stats) / (ph[3] / 1e3) / 1e9
              if ph[3] > 0 else None,
              "clock": "%globaltimer read by block 0 after each grid barrier"}
    key = f"cg_persistent_{args.inner}_{'x'.join(map(str, dims))}_n{nb}_delta{DEFAULT_DELTA[args.inner]}"
    traffic = kernel_traffic(key)
    binding = "alu" if frac_alu >= frac_hbm else "hbm"
    roofline = {"bound": binding,
                "achieved": tflops if binding == "alu" else gbs,
                "peak": fp32_peak if binding == "alu" else hbm_peak,
                "unit": "TFLOP/s" if binding == "alu" else "GB/s",
                "frac": frac_alu if binding == "alu" else frac_hbm,
                "traffic": traffic,
                "kernel": f"cg_persistent_kernel<{args.inner}> (whole bundle solve, {k_n} launches in the timed region, "
                          f"bundles of {nb})",
                "peak_source": ("measured FP32 FMA peak (hisq_measure_fma_peaks: independent FMA chains on every SM)"
                                if binding == "alu" else f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"),
                "algorithmic_flops_per_launch": k_flops / max(k_n, 1),
                "algorithmic_bytes_per_launch": k_bytes / max(k_n, 1),
                "launch_ms": k_ms / max(k_n, 1),
                "other_bound": {"unit": "GB/s" if binding == "alu" else "TFLOP/s",
                                "achieved": gbs if binding == "alu" else tflops,
                                "peak": hbm_peak if binding == "alu" else fp32_peak,
                                "frac": frac_hbm if binding == "alu" else frac_alu},
                "phases": phases}

    line = None
    extras = {}
    if not args.no_extras:
        # ---- plain FP64 single-RHS CG on the same field and first right-hand side (the comparator) ----
        set_params(hisq, 0, 2, 1)
        solve_ms(hisq, torch, stream, fat, naik, bs[:1], xs[:1], mass, flush)
        r64 = [solve_ms(hisq, torch, stream, fat, naik, bs[:1], xs[:1], mass, flush) for _ in range(2)]
        fp64_s = statistics.median(r[0] for r in r64) / 1e3
        # ---- the same mixed-precision solve one right-hand side at a time ----
        set_params(hisq, inner, 2, 1, 1)
        solve_ms(hisq, torch, stream, fat, naik, bs[:1], xs[:1], mass, flush)
        r1 = [solve_ms(hisq, torch, stream, fat, naik, bs[:1], xs[:1], mass, flush) for _ in range(2)]
        single_s = statistics.median(r[0] for r in r1) / 1e3
        extras = {
            "fp64_cg_s_per_rhs": fp64_s, "speedup_vs_fp64_cg": fp64_s / s_per_rhs,
            "fp64_cg_iterations": r64[-1][1].max_iterations,
            "single_rhs_mixed": {"s_per_rhs": single_s, "iterations": r1[-1][1].max_iterations,
                                 "bundle_speedup_per_rhs": single_s / s_per_rhs},
            "dslash": {"precision": args.inner,
                       "n1": dslash_rate(hisq, torch, hi, lat, fat, naik, inner, 1, flush, stream, dev, d64),
                       "n16": dslash_rate(hisq, torch, hi, lat, fat, naik, inner, 16, flush, stream, dev, d64)},
            "alu_peaks": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak,
                          "how": "independent FMA chains on every SM, CUDA events (hisq_measure_fma_peaks)"},
        }
        # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region) ----
        bh = [torch.from_numpy(np.ascontiguousarray(v).view(np.float64).copy()).pin_memory() for v in rhs_host]
        xh = [torch.empty_like(v).pin_memory() for v in bh]
        set_params(hisq, inner, 2, 0, args.bundle)
        hisq.hisq_cg_solve(fat, naik, bh, xh, mass, TOL)
        ke = max(2, min(args.steps, 4))
        el, est = [], []
        for _ in range(ke):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            hisq.hisq_cg_solve(fat, naik, bh, xh, mass, TOL)
            el.append(time.perf_counter() - t)
            est.append(hisq.hisq_last_stats())
        vbytes = Vh * 6 * 8 * nstep
        extras["e2e"] = {"value": sum(s.flops for s in est) / sum(el) / 1e9, "unit": "GFlop/s",
                         "h2d_bytes_per_step": vbytes, "d2h_bytes_per_step": vbytes}
    hisq.hisq_finalize()
    if not args.no_extras:
        extras["small_lattice_single_rhs"] = small_lattice_figures(hisq, torch, hi, inner, stream, dev, flush)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(lat, X, N, rhs_host[0], mass)
        line = {
            "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic", "config": cfg,
            "cg_s_per_rhs": s_per_rhs, "iterations_max": int(iters.max()), "iterations_mean": float(iters.mean()),
            "reliable_updates": last.reliable_updates, "recompute_passes": last.recompute_passes,
            "bundle_size": nb, "converged": last.converged, "true_residual_max": float(res.max()),
            "roofline": roofline, "cpu_baseline": cpu,
            "gpu_launches": int(launches_all), "clocks": clk.summary(), "wall_s_timed_region": t_wall,
            "field_generation_s": t_fields, **extras,
        }
        if "e2e" not in line:
            line["e2e"] = None
    return line


def run_sweep(args):
    """Dslash GFlop/s and GB/s against n (Eq. (4)) for each storage precision, 18-real links,
    autotuned launch shape, L2 flushed before every timed launch (CUDA events)."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import accounting as acc
    from paper_1409_1510_gb300 import hisq
    dims, _ = workload(args)
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    hisq.hisq_init(dims, 0, stream)
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    hbm_peak, _ = peaks()
    fp32_peak, fp64_peak = hisq.hisq_measure_fma_peaks()
    print(json.dumps({"fp32_fma_tflops": fp32_peak, "fp64_fma_tflops": fp64_peak}), flush=True)
    rows = []
    for name in ("fp32", "fp16", "bf16", "fp64"):
        prec = PREC[name]
        fat = hisq.hisq_links_create(d64(X), False, prec, 18)
        naik = hisq.hisq_links_create(d64(N), True, prec, 18)
        for n in ((1, 2, 4, 8, 12, 16) if prec else (1, 2, 4)):
            vin = torch.empty(hisq.hisq_vector_bytes(prec, n), dtype=torch.uint8, device=dev)
            hisq.hisq_pack(d64(np.stack([hi.gaussian_rhs(lat, k) for k in range(n)])), vin, n, prec)
            vout = torch.empty_like(vin)
            shape = hisq.hisq_autotune(fat, naik, n)
            ts = []
            for i in range(12):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hisq.hisq_dslash(fat, naik, vin, vout, n, i % 2)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            sec = statistics.median(ts[2:]) / 1e3
            elem = {0: 8, 1: 4, 2: 2, 3: 2}[prec]
            byts = acc.compulsory_bytes(n, elem, elem, 18, 8.0 if prec in (2, 3) else 0.0,
                                        4.0 if prec == 2 else 0.0) * lat.half_volume
            rows.append({"precision": name, "nrhs": n, "us": sec * 1e6,
                         "gflops": acc.DSLASH_FLOPS_PER_SITE * n * lat.half_volume / sec / 1e9,
                         "gbs": byts / sec / 1e9, "frac_hbm": byts / sec / 1e9 / hbm_peak,
                         "frac_fma_peak": acc.DSLASH_FLOPS_PER_SITE * n * lat.half_volume / sec / 1e12
                         / (fp64_peak if prec == 0 else fp32_peak),
                         "shape": {"rhs_per_thread": shape[0], "threads": shape[1], "lanes_per_site": shape[2]}})
            print(json.dumps(rows[-1]), flush=True)
        hisq.hisq_links_destroy(fat)
        hisq.hisq_links_destroy(naik)
    hisq.hisq_finalize()


def run_dslash(args):
    """One Dslash configuration: links and --nrhs right-hand sides (default 16) in --inner
    storage on --dims, launched --steps times with the L2 flushed before each (CUDA events);
    prints the median time, GFlop/s and compulsory GB/s and the launch shape."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import accounting as acc
    from paper_1409_1510_gb300 import hisq
    dims, _ = workload(args)
    n = args.nrhs if args.nrhs != 1500 else 16
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    hisq.hisq_init(dims, 0, stream)
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    prec = PREC[args.inner] if args.inner in PREC else 2
    fat = hisq.hisq_links_create(d64(X), False, prec, 18)
    naik = hisq.hisq_links_create(d64(N), True, prec, args.recon)
    vin = torch.empty(hisq.hisq_vector_bytes(prec, n), dtype=torch.uint8, device=dev)
    hisq.hisq_pack(d64(np.stack([hi.gaussian_rhs(lat, k) for k in range(n)])), vin, n, prec)
    vout = torch.empty_like(vin)
    if args.shape:
        shape = tuple(int(v) for v in args.shape.split(","))
        hisq.hisq_set_launch_shape(prec, args.recon, n, *shape)
    else:
        shape = hisq.hisq_autotune(fat, naik, n)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    hisq.hisq_dslash(fat, naik, vin, vout, n, 1)  # warm-up
    ts = []
    for i in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hisq.hisq_dslash(fat, naik, vin, vout, n, i % 2)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    sec = statistics.median(ts) / 1e3
    elem = {0: 8, 1: 4, 2: 2, 3: 2}[prec]
    # 16-bit records carry a float scale per site for the fat field, and for the Naik field when stored in full
    scales = (4.0 * (1 + (args.recon == 18))) if prec in (2, 3) else 0.0
    byts = acc.compulsory_bytes(n, elem, elem, args.recon, scales, 4.0 if prec == 2 else 0.0) * lat.half_volume
    hbm_peak, _ = peaks()
    print(json.dumps({"mode": "dslash", "lattice": dims, "precision": args.inner, "naik_reals": args.recon,
                      "nrhs": n, "launches": args.steps,
                      "us": sec * 1e6, "gflops": acc.DSLASH_FLOPS_PER_SITE * n * lat.half_volume / sec / 1e9,
                      "gbs": byts / sec / 1e9, "frac_hbm": byts / sec / 1e9 / hbm_peak,
                      "shape_arg": ",".join(str(v) for v in shape)}), flush=True)
    hisq.hisq_finalize()


def run_slabs(args):
    """The Dslash decomposed into 2 and 4 t-slabs with depth-3 ghost planes (all slabs on this GPU)
    against the undecomposed Dslash of the same canonical input, --inner storage, 1 and 16
    right-hand sides: median CUDA-event times of face packing, interior kernels, halo copies and the
    whole decomposed Dslash (scatter and gather excluded), L2 flushed before each launch."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import hisq
    dims, _ = workload(args)
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    hisq.hisq_init(dims, 0, stream)
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    prec = PREC[args.inner]
    Xd, Nd = d64(X), d64(N)
    fat = hisq.hisq_links_create(Xd, False, prec, 18)
    naik = hisq.hisq_links_create(Nd, True, prec, 18)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    out = {"mode": "slabs", "lattice": list(dims), "precision": args.inner, "runs": []}
    for n in (1, 16):
        vin = d64(np.stack([hi.gaussian_rhs(lat, k) for k in range(n)]))
        vout = torch.empty_like(vin)
        packed = torch.empty(hisq.hisq_vector_bytes(prec, n), dtype=torch.uint8, device=dev)
        hisq.hisq_pack(vin, packed, n, prec)
        pout = torch.empty_like(packed)
        hisq.hisq_autotune(fat, naik, n)
        ts = []
        for i in range(max(args.steps, 5)):
            flush.zero_()
            ts.append(event_ms(torch, stream, lambda: hisq.hisq_dslash(fat, naik, packed, pout, n, 0)))
        whole_ms = statistics.median(ts)
        for nslab in (2, 4):
            h = hisq.hisq_slabs_create(Xd, Nd, prec, nslab)
            ms = np.zeros(4)
            hisq.hisq_slabs_dslash(h, vin, vout, n, 0, ms)  # warm-up
            rows = []
            for i in range(max(args.steps, 5)):
                flush.zero_()
                torch.cuda.synchronize()
                hisq.hisq_slabs_dslash(h, vin, vout, n, 0, ms)
                rows.append(ms.copy())
            med = np.median(np.stack(rows), axis=0)
            out["runs"].append({"nrhs": n, "slabs": nslab, "planes_per_slab": dims[3] // nslab,
                                "face_pack_ms": med[0], "interior_ms": med[1], "halo_copy_ms": med[2],
                                "decomposed_ms": med[3], "undecomposed_ms": whole_ms,
                                "overhead": med[3] / whole_ms - 1.0})
            hisq.hisq_slabs_destroy(h)
    print(json.dumps(out), flush=True)
    hisq.hisq_finalize()


def make_pairs(hisq, torch, hi, lat, fat, naik, mass, d64, want):
    """(r, e) training pairs from plain FP32 CG on this gauge field: 16 right-hand sides at a time
    are solved to 1e-10 (x*), then re-solved for k iterations (x_k) at 25 values of k up to 80% of
    the iteration count; e = x* - x_k, r = b - A x_k (so A e = r).  Returns packed FP32 bundles of
    16 pairs (r and e) and the number of pairs."""
    vh = lat.half_volume
    dev = torch.device("cuda", 0)
    p = hisq.hisq_default_solver_params()
    p.inner_prec = 1
    per_rhs = 25
    nrhs = (want + per_rhs - 1) // per_rhs
    bsz = hisq.hisq_vector_bytes(1, 16)
    nb = (want + 15) // 16
    rbuf = torch.empty(nb * bsz, dtype=torch.uint8, device=dev)
    ebuf = torch.empty_like(rbuf)
    pending_r, pending_e, filled = [], [], 0
    canon = lambda v: torch.stack(v).contiguous()
    done = 0
    for j0 in range(0, nrhs, 16):
        bs = [d64(hi.gaussian_rhs(lat, 7000 + j)) for j in range(j0, min(nrhs, j0 + 16))]
        xs = [torch.zeros_like(b) for b in bs]
        p.max_iter = 20000
        p.bundle = len(bs)
        hisq.hisq_set_solver_params(p)
        hisq.hisq_cg_solve(fat, naik, bs, xs, mass, TOL)
        its = hisq.hisq_last_stats().max_iterations
        for k in np.linspace(2, max(3, int(0.8 * its)), per_rhs).astype(int):
            p.max_iter = int(k)
            hisq.hisq_set_solver_params(p)
            xk = [torch.zeros_like(b) for b in bs]
            hisq.hisq_cg_solve(fat, naik, bs, xk, mass, TOL, raise_on_error=False)
            # r_k = b - A x_k on the GPU (A in FP32 through the library)
            xin = torch.empty(hisq.hisq_vector_bytes(1, len(bs)), dtype=torch.uint8, device=dev)
            ax = torch.empty_like(xin)
            hisq.hisq_pack(canon(xk), xin, len(bs), 1)
            hisq.hisq_aop(fat, naik, mass, xin, ax, len(bs))
            axc = torch.empty((len(bs), vh, 3, 2), dtype=torch.float64, device=dev)
            hisq.hisq_unpack(ax, axc, len(bs), 1)
            for q in range(len(bs)):
                if done >= want:
                    break
                pending_r.append(bs[q].view(vh, 3, 2) - axc[q])
                pending_e.append(xs[q].view(vh, 3, 2) - xk[q].view(vh, 3, 2))
                done += 1
                if len(pending_r) == 16:
                    hisq.hisq_pack(canon(pending_r), rbuf[filled * bsz:(filled + 1) * bsz], 16, 1)
                    hisq.hisq_pack(canon(pending_e), ebuf[filled * bsz:(filled + 1) * bsz], 16, 1)
                    filled += 1
                    pending_r, pending_e = [], []
    return rbuf, ebuf, filled * 16


def train_network(hisq, torch, fat, naik, mass, rbuf, ebuf, npairs, epochs, hist=None, validate=None, rounds=1):
    """Adam on the GPU from the identity plus a 2% random perturbation (the identity is a saddle
    point); returns the preconditioner handle.  With `validate` (a function of the handle that
    returns the mean flexible-CG iteration count on validation right-hand sides), training runs
    in `rounds` equal parts and the handle keeps the weights of the best validated part (the
    residual-norm loss does not see the conditioning of the preconditioned operator, which can
    drift while the loss stays flat); returns (handle, validation curve) then."""
    rng = np.random.default_rng(0)
    w0 = np.zeros(408, complex)
    w0[[0, 68, 340]] = 1.0
    w0 += 0.02 * (rng.standard_normal(408) + 1j * rng.standard_normal(408))
    pc = hisq.hisq_pc_create(np.ascontiguousarray(w0).view(np.float64))
    if hist is None:
        hist = np.zeros(epochs)
    if validate is None:
        hisq.hisq_pc_train(pc, fat, naik, mass, rbuf, ebuf, npairs, 16, epochs, 5e-3, hist)
        torch.cuda.synchronize()
        return pc
    per = max(1, epochs // rounds)
    curve, best, best_w = [], None, None
    for k in range(0, epochs, per):
        h = np.zeros(min(per, epochs - k))
        hisq.hisq_pc_train(pc, fat, naik, mass, rbuf, ebuf, npairs, 16, len(h), 5e-3, h)
        hist[k:k + len(h)] = h
        its = validate(pc)
        curve.append({"epochs": k + len(h), "loss": float(h[-1]), "validation_iterations": its})
        print(f"training: {curve[-1]}", file=sys.stderr, flush=True)
        if best is None or its < best:
            best, best_w = its, np.zeros(2 * 408)
            hisq.hisq_pc_get_weights(pc, best_w)
    hisq.hisq_pc_set_weights(pc, best_w)
    torch.cuda.synchronize()
    return pc, curve


def run_learned(args):
    """Learned-preconditioner workload: (r, e) pairs from plain CG iterates on the same gauge
    field, training on the GPU, then flexible CG against plain CG on fresh right-hand sides."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import hisq
    dims, _ = workload(args)
    mass = args.mass
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    hisq.hisq_init(dims, 0, torch.cuda.current_stream())
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    fat = hisq.hisq_links_create(d64(X), False, 1, 18)
    naik = hisq.hisq_links_create(d64(N), True, 1, 18)
    t0 = time.perf_counter()
    rbuf, ebuf, pairs = make_pairs(hisq, torch, hi, lat, fat, naik, mass, d64, args.pairs)
    t_pairs = time.perf_counter() - t0
    print(f"pairs: {pairs} in {t_pairs:.1f} s", file=sys.stderr, flush=True)
    hist = np.zeros(args.epochs)
    valid = [d64(hi.gaussian_rhs(lat, 8000 + k)) for k in range(16)]
    # flexible CG gets at most ten times the iterations plain CG needs (a poor network then ends
    # unconverged, and is reported as such, instead of running to the default limit)
    _, _, its_cg, _ = _solve_set(hisq, torch, fat, naik, valid, mass, inner_prec=1, bundle=16)
    cap = int(10 * its_cg.max())

    def validate(handle):
        _, st, its, _ = _solve_set(hisq, torch, fat, naik, valid, mass, inner_prec=1, bundle=16, pc=handle.value,
                                   max_iter=cap)
        return float(its.mean()) if st.converged == len(valid) else float(cap)

    t0 = time.perf_counter()
    pc, curve = train_network(hisq, torch, fat, naik, mass, rbuf, ebuf, pairs, args.epochs, hist, validate,
                              rounds=6)
    t_train = time.perf_counter() - t0
    # fresh right-hand sides: plain CG against flexible CG with the network (both FP32 inner,
    # FP64 reliable updates, true residual 1e-10 checked in FP64)
    tests = [d64(hi.gaussian_rhs(lat, 9000 + k)) for k in range(args.test_rhs)]
    out = {}
    for name, handle in (("cg", None), ("fcg_learned", pc)):
        hv = handle.value if handle is not None else None
        _solve_set(hisq, torch, fat, naik, tests[:16], mass, inner_prec=1, bundle=16, pc=hv, max_iter=cap)  # warm-up
        sec, st, iters, res = _solve_set(hisq, torch, fat, naik, tests, mass, inner_prec=1, bundle=16, pc=hv,
                                         max_iter=cap)
        out[name] = {"s_per_rhs": sec / len(tests), "mean_iterations": float(iters.mean()),
                     "max_true_residual": float(res.max()), "converged": st.converged,
                     "fallbacks": st.fallbacks}
        print(f"test {name}: {out[name]}", file=sys.stderr, flush=True)
    line = {"mode": "learned", "lattice": dims, "mass": mass, "pairs": pairs, "pair_seconds": t_pairs,
            "train_seconds": t_train, "epochs": args.epochs, "loss_first": float(hist[0]),
            "loss_last": float(hist[-1]), "form": "normal (M^dag M)", "validation": curve, "max_iter": cap,
            "validation_rhs": len(valid), "test_rhs": len(tests), **out,
            "iteration_ratio": out["fcg_learned"]["mean_iterations"] / out["cg"]["mean_iterations"],
            "time_ratio": out["fcg_learned"]["s_per_rhs"] / out["cg"]["s_per_rhs"]}
    print(json.dumps(line), flush=True)
    hisq.hisq_finalize()


def _solve_set(hisq, torch, fat, naik, bs, mass, **params):
    """Solve the right-hand sides bs (device canonical) with the given solver parameters; returns
    (seconds by CUDA events, stats, iterations, true residuals)."""
    p = hisq.hisq_default_solver_params()
    for k, v in params.items():
        setattr(p, k, v)
    hisq.hisq_set_solver_params(p)
    xs = [torch.zeros_like(b) for b in bs]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    # a right-hand side that misses tol within max_iter is reported through the stats
    hisq.hisq_cg_solve(fat, naik, bs, xs, mass, TOL, raise_on_error=False)
    e1.record(stream)
    e1.synchronize()
    iters = np.zeros(len(bs), dtype=np.int32)
    res = np.zeros(len(bs))
    st = hisq.hisq_last_stats(iters, res)
    return e0.elapsed_time(e1) / 1e3, st, iters, res


def run_batch(args):
    """Batching form on 48^3 x 12, m = 0.002, FP32 storage: 16 Gaussian right-hand sides with
    norms log-uniform in 1e-3..1e3 and spectral shaping (b_k = s_k A^{q_k} g_k / |.|, q_k = k mod 3,
    A applied in FP64 by the library), solved in bundles of n = 1, 2, 4, 8, 12, 16 by the persistent
    kernel and by the captured CUDA graph, and with the bundle size chosen by the autotuner."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import hisq
    dims = tuple(int(x) for x in args.dims.split(","))
    mass = args.mass
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    hisq.hisq_init(dims, 0, torch.cuda.current_stream())
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    vh, nrhs = lat.half_volume, 16
    # the shaped right-hand sides (FP64 A through the library)
    f64 = hisq.hisq_links_create(d64(X), False, 0, 18)
    n64 = hisq.hisq_links_create(d64(N), True, 0, 18)
    scales = 10.0 ** np.random.default_rng(2000).uniform(-3.0, 3.0, nrhs)
    bs = []
    vin = torch.empty(hisq.hisq_vector_bytes(0, 1), dtype=torch.uint8, device=dev)
    vout = torch.empty_like(vin)
    for k in range(nrhs):
        g = d64(hi.gaussian_rhs(lat, 2000 + k))
        for _ in range(k % 3):
            hisq.hisq_pack(g, vin, 1, 0)
            hisq.hisq_aop(f64, n64, mass, vin, vout, 1)
            g = torch.empty_like(g)
            hisq.hisq_unpack(vout, g, 1, 0)
        bs.append((g * (scales[k] / torch.linalg.vector_norm(g))).contiguous())
    hisq.hisq_links_destroy(f64)
    hisq.hisq_links_destroy(n64)
    fat = hisq.hisq_links_create(d64(X), False, 1, 18)
    naik = hisq.hisq_links_create(d64(N), True, 1, 18)
    rows = []
    for n in (1, 2, 4, 8, 12, 16):
        row = {"bundle": n}
        for name, driver in (("persistent", 2), ("graph", 1)):
            _solve_set(hisq, torch, fat, naik, bs[:n], mass, inner_prec=1, bundle=n, use_graph=driver)  # warm-up
            sec, st, iters, res = _solve_set(hisq, torch, fat, naik, bs, mass, inner_prec=1, bundle=n, use_graph=driver)
            # right-hand-side iterations a bundle's Dslash phases spend on converged (masked) lanes
            idle = sum(int(iters[k0:k0 + n].max()) * len(iters[k0:k0 + n]) - int(iters[k0:k0 + n].sum())
                       for k0 in range(0, nrhs, n))
            row[name] = {"s_per_rhs": sec / nrhs, "iterations_min": int(iters.min()), "iterations_max": int(iters.max()),
                         "iterations_sum": int(iters.sum()), "bundle_iterations": int(st.bundle_iterations),
                         "masked_lane_fraction": idle / (idle + int(iters.sum())), "converged": int(st.converged),
                         "max_true_residual": float(res.max())}
        rows.append(row)
        print(json.dumps(row), flush=True)
    sec, st, iters, res = _solve_set(hisq, torch, fat, naik, bs, mass, inner_prec=1, bundle=0)
    auto = {"bundle_chosen": int(st.bundle_size), "s_per_rhs": sec / nrhs, "converged": int(st.converged),
            "max_true_residual": float(res.max())}
    line = {"mode": "batch", "lattice": list(dims), "mass": mass, "nrhs": nrhs, "storage": "fp32",
            "rhs": "Gaussian, norms log-uniform 1e-3..1e3, spectral shaping A^(k mod 3)",
            "bundles": rows, "autotuned": auto,
            "speedup_16_vs_1": rows[0]["persistent"]["s_per_rhs"] / rows[-1]["persistent"]["s_per_rhs"]}
    print(json.dumps(line), flush=True)
    hisq.hisq_finalize()


def run_production(args):
    """Production-shaped sweep on 64^3 x 16, m = 0.002: args.nrhs Z2-noise right-hand sides,
    FP16 storage with FP64 reliable updates, bundle size from the autotuner, every right-hand side
    to the FP64 true residual 1e-10; the Dslash phases' HBM rate from the persistent kernel's
    phase clock.  With --pc, the network is trained on this gauge field (FP32) and flexible CG is
    compared with plain FP32 CG on a sample of the right-hand sides."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import accounting as acc
    from paper_1409_1510_gb300 import hisq
    dims = tuple(int(x) for x in args.dims.split(","))
    mass = args.mass
    lat = hi.Lattice(dims)
    t0 = time.perf_counter()
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    t_fields = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    hisq.hisq_init(dims, 0, torch.cuda.current_stream())
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    fat = hisq.hisq_links_create(d64(X), False, 2, 18)
    naik = hisq.hisq_links_create(d64(N), True, 2, 18)
    vh = lat.half_volume
    hbm_peak, _ = peaks()
    chunk = 96  # right-hand sides per call (the library splits them into tuned bundles)
    _solve_set(hisq, torch, fat, naik, [d64(hi.z2_rhs(lat, 50000 + k)) for k in range(16)], mass,
               inner_prec=2, bundle=0)  # warm-up: tuning and first launches
    tot_s, its, ups, conv, worst, ph, kms, bits, nb = 0.0, [], 0, 0, 0.0, np.zeros(5), 0.0, 0, 0
    t_wall = time.perf_counter()
    for k0 in range(0, args.nrhs, chunk):
        bs = [d64(hi.z2_rhs(lat, 60000 + k)) for k in range(k0, min(args.nrhs, k0 + chunk))]
        sec, st, iters, res = _solve_set(hisq, torch, fat, naik, bs, mass, inner_prec=2, bundle=0, time_kernels=1)
        tot_s += sec
        its += iters.tolist()
        ups += st.reliable_updates
        conv += st.converged
        worst = max(worst, float(res.max()))
        ph += np.array(list(st.phase_ms))
        kms += st.solve_kernel_ms
        bits += st.bundle_iterations
        nb = st.bundle_size
    t_wall = time.perf_counter() - t_wall
    P_b = acc.VECTOR_BYTES[2]
    ds_bytes = bits * (2 * acc.LINK_BYTES_18[2] + 5 * P_b * nb) * vh
    line = {"mode": "production", "lattice": list(dims), "mass": mass, "nrhs": args.nrhs, "storage": "fp16",
            "bundle_chosen": nb, "sweep_seconds_gpu": tot_s, "sweep_seconds_wall": t_wall,
            "s_per_rhs": tot_s / args.nrhs, "converged": conv, "max_true_residual": worst,
            "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
            "reliable_updates": int(ups),
            "dslash_phases_gbs": ds_bytes / (ph[0] + ph[1]) * 1e3 / 1e9 if ph[0] + ph[1] > 0 else None,
            "fp64_reliable_share": ph[3] / kms if kms > 0 else None, "field_generation_s": t_fields}
    line["dslash_phases_frac"] = line["dslash_phases_gbs"] / hbm_peak if line["dslash_phases_gbs"] else None
    if args.pc:
        line["learned"] = production_pc(args, hisq, torch, hi, lat, X, N, mass, d64)
    print(json.dumps(line), flush=True)
    hisq.hisq_finalize()


def production_pc(args, hisq, torch, hi, lat, X, N, mass, d64):
    """Train the network on (r, e) pairs of this gauge field (FP32 links) and compare flexible CG
    with plain CG on a sample of Z2 right-hand sides."""
    fat = hisq.hisq_links_create(d64(X), False, 1, 18)
    naik = hisq.hisq_links_create(d64(N), True, 1, 18)
    pairs = make_pairs(hisq, torch, hi, lat, fat, naik, mass, d64, args.pairs)
    rbuf, ebuf, npairs = pairs
    valid = [d64(hi.z2_rhs(lat, 59000 + k)) for k in range(16)]
    _, _, its_cg, _ = _solve_set(hisq, torch, fat, naik, valid, mass, inner_prec=1, bundle=16)
    cap = int(10 * its_cg.max())

    def validate(handle):
        _, st, its, _ = _solve_set(hisq, torch, fat, naik, valid, mass, inner_prec=1, bundle=16, pc=handle.value,
                                   max_iter=cap)
        return float(its.mean()) if st.converged == len(valid) else float(cap)

    pc, curve = train_network(hisq, torch, fat, naik, mass, rbuf, ebuf, npairs, args.epochs, None, validate,
                              rounds=max(1, min(args.epochs, 4)))
    sample = [d64(hi.z2_rhs(lat, 60000 + k)) for k in range(args.test_rhs)]
    out = {"pairs": npairs, "epochs": args.epochs, "validation": curve}
    for name, handle in (("cg", None), ("fcg_learned", pc)):
        _solve_set(hisq, torch, fat, naik, sample[:16], mass, inner_prec=1, bundle=16,
                   pc=handle.value if handle is not None else None, max_iter=cap)
        sec, st, iters, res = _solve_set(hisq, torch, fat, naik, sample, mass, inner_prec=1, bundle=16,
                                         pc=handle.value if handle is not None else None, max_iter=cap)
        out[name] = {"s_per_rhs": sec / len(sample), "mean_iterations": float(iters.mean()),
                     "max_true_residual": float(res.max()), "converged": int(st.converged),
                     "fallbacks": int(st.fallbacks)}
    hisq.hisq_pc_destroy(pc)
    hisq.hisq_links_destroy(fat)
    hisq.hisq_links_destroy(naik)
    return out


MS_SHIFTS = (0.0,) + tuple(float(v) for v in 10.0 ** np.linspace(-4.0, 0.0, 7))


def _multishift(hisq, torch, fat, naik, b, shifts, mass, **params):
    """One hisq_cg_multishift call: (wall seconds around the synchronous call, stats, per-shift
    iterations, per-shift FP64 true residuals)."""
    p = hisq.hisq_default_solver_params()
    for k, v in params.items():
        setattr(p, k, v)
    hisq.hisq_set_solver_params(p)
    xs = [torch.zeros_like(b) for _ in shifts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hisq.hisq_cg_multishift(fat, naik, b, xs, shifts, mass, TOL, raise_on_error=False)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    iters = np.zeros(len(shifts), dtype=np.int32)
    res = np.zeros(len(shifts))
    st = hisq.hisq_last_stats(iters, res)
    return sec, st, iters, res


def run_multishift(args):
    """Eight shifted systems (A + sigma_j) x_j = b on 32^3 x 8, m = 0.01, sigma = 0 and 1e-4..1
    (log-spaced, the spread of a rational approximation's poles), one Gaussian right-hand side,
    every shift to the FP64 true residual 1e-10: one multi-shift solve (low-precision shared
    iteration plus per-shift FP64 refinement, for each storage precision and shared tolerance;
    and all in FP64) against eight separate mixed-precision CG solves."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import hisq
    dims = tuple(int(x) for x in args.dims.split(","))
    mass = args.mass
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    hisq.hisq_init(dims, 0, torch.cuda.current_stream())
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    b = d64(hi.gaussian_rhs(lat, 7000))
    shifts = MS_SHIFTS
    rows = []
    for prec_name in ("fp16", "fp32", "fp64"):
        prec = PREC[prec_name]
        fat = hisq.hisq_links_create(d64(X), False, prec, 18)
        naik = hisq.hisq_links_create(d64(N), True, prec, 18)
        tols = (1e-3, 1e-4, 1e-5) if prec in (2, 3) else (1e-5, 1e-6, 1e-7) if prec == 1 else (None,)
        for tol_ms in tols:
            extra = {"multishift_tol": tol_ms} if tol_ms else {}
            _multishift(hisq, torch, fat, naik, b, shifts, mass, inner_prec=prec, **extra)  # warm-up, capture
            runs = [_multishift(hisq, torch, fat, naik, b, shifts, mass, inner_prec=prec, **extra) for _ in range(3)]
            sec, st, iters, res = sorted(runs, key=lambda r: r[0])[1]
            rows.append({"solver": "multishift", "storage": prec_name, "shared_tol": tol_ms, "seconds": sec,
                         "shared_seconds": st.shared_seconds, "shared_iterations": int(st.shared_iterations),
                         "refine_iterations": int(st.refine_iterations), "iterations": iters.tolist(),
                         "converged": int(st.converged), "max_true_residual": float(res.max())})
            print(json.dumps(rows[-1]), flush=True)
            if tol_ms in (1e-7, None):
                # the same solve with the shared iteration as the captured graph (use_graph = 1)
                _multishift(hisq, torch, fat, naik, b, shifts, mass, inner_prec=prec, use_graph=1, **extra)
                runs = [_multishift(hisq, torch, fat, naik, b, shifts, mass, inner_prec=prec, use_graph=1, **extra)
                        for _ in range(3)]
                sec, st, iters, res = sorted(runs, key=lambda r: r[0])[1]
                rows.append({"solver": "multishift_graph", "storage": prec_name, "shared_tol": tol_ms, "seconds": sec,
                             "shared_seconds": st.shared_seconds, "shared_iterations": int(st.shared_iterations),
                             "refine_iterations": int(st.refine_iterations), "converged": int(st.converged),
                             "max_true_residual": float(res.max())})
                print(json.dumps(rows[-1]), flush=True)
        if prec != 0:
            # the same eight systems as separate mixed-precision CG solves (mass sqrt(m^2 + sigma))
            tot, its, conv, worst = 0.0, [], 0, 0.0
            for sg in shifts:
                m_j = float(np.sqrt(mass * mass + sg))
                _solve_set(hisq, torch, fat, naik, [b], m_j, inner_prec=prec, bundle=1)
                sec, st, it, res = _solve_set(hisq, torch, fat, naik, [b], m_j, inner_prec=prec, bundle=1)
                tot += sec
                its.append(int(it[0]))
                conv += st.converged
                worst = max(worst, float(res[0]))
            rows.append({"solver": "separate_cg", "storage": prec_name, "seconds": tot, "iterations": its,
                         "converged": conv, "max_true_residual": worst})
            print(json.dumps(rows[-1]), flush=True)
        hisq.hisq_links_destroy(fat)
        hisq.hisq_links_destroy(naik)
    best = min((r for r in rows if r["solver"] == "multishift" and r["converged"] == len(shifts)),
               key=lambda r: r["seconds"])
    sep = min((r for r in rows if r["solver"] == "separate_cg"), key=lambda r: r["seconds"])
    line = {"mode": "multishift", "lattice": list(dims), "mass": mass, "shifts": list(shifts), "runs": rows,
            "best_multishift": {k: best[k] for k in ("storage", "shared_tol", "seconds")},
            "best_separate_cg": {k: sep[k] for k in ("storage", "seconds")},
            "speedup_vs_separate_cg": sep["seconds"] / best["seconds"]}
    print(json.dumps(line), flush=True)
    hisq.hisq_finalize()


def run_trace(args):
    """Eq. (2) without derivative factors on 32^3 x 8, m = 0.01: Tr A^{-1} over the even sites from
    --nrhs Z2 noise vectors (default 64), FP16 storage with FP64 reliable updates, bundles chosen
    by the autotuner, every solve to the FP64 true residual 1e-10; reports the estimate, its
    standard error, Tr M^{-1} / V = 2 m Tr A^{-1} / V for M = m + D, and the time per noise vector."""
    import torch
    import hisq_inputs as hi
    from paper_1409_1510_gb300 import hisq
    dims = tuple(int(x) for x in args.dims.split(","))
    mass = args.mass
    nnoise = args.nrhs if args.nrhs != 1500 else 64
    lat = hi.Lattice(dims)
    X, N = hi.fat_links(lat), hi.naik_links(lat)
    dev = torch.device("cuda", 0)
    hisq.hisq_init(dims, 0, torch.cuda.current_stream())
    d64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).to(dev)
    prec = PREC[args.inner]
    fat = hisq.hisq_links_create(d64(X), False, prec, 18)
    naik = hisq.hisq_links_create(d64(N), True, prec, 18)
    p = hisq.hisq_default_solver_params()
    p.inner_prec = prec
    hisq.hisq_set_solver_params(p)
    hisq.hisq_trace_inverse(fat, naik, mass, 16, 1, TOL)  # warm-up: tuning, first launches
    samples = np.zeros(nnoise)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    est, err, _ = hisq.hisq_trace_inverse(fat, naik, mass, nnoise, 2026, TOL, samples)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    res = np.zeros(nnoise)
    st = hisq.hisq_last_stats(None, res)
    V = int(np.prod(dims))
    line = {"mode": "trace", "lattice": list(dims), "mass": mass, "storage": args.inner, "nnoise": nnoise,
            "seconds": sec, "s_per_noise": sec / nnoise, "trace_A_inv": est, "std_error": err,
            "condensate_TrMinv_over_V": 2 * mass * est / V, "condensate_error": 2 * mass * err / V,
            "bundle": int(st.bundle_size), "mean_iterations": st.total_iterations / nnoise,
            "converged": int(st.converged), "max_true_residual": float(res.max())}
    print(json.dumps(line), flush=True)
    hisq.hisq_finalize()


def main():
    args = parse()
    if args.mode == "trace":
        run_trace(args)
        return
    if args.mode == "multishift":
        run_multishift(args)
        return
    if args.mode == "sweep":
        run_sweep(args)
        return
    if args.mode == "dslash":
        run_dslash(args)
        return
    if args.mode == "learned":
        run_learned(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    if args.mode == "production":
        run_production(args)
        return
    if args.mode == "slabs":
        run_slabs(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist = tdist
    line = run_ours(args, rank, world, local_rank, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
