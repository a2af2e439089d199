"""Benchmark: HISQ stencil bandwidth and time-to-1e-10 of the mixed-precision CG.

One step = one complete even/odd CG solve, (4m^2 - D_eo D_oe) x = b, to a
1e-10 FP64 true residual on a 32^3 x 64 lattice (m = 0.01, delta = 0.1) with
the sloppy iteration in the paper's 16-bit gauge / 20-bit fermion / FP32
triplet and FP64 reliable updates, from a right-hand side already resident in
HBM.  ``value`` is the solve's algorithmic HBM traffic (every kernel's arrays
counted once per launch) divided by the step time; ``roofline`` reports the
stencil kernel alone from CUDA events around each of its launches in the
timed region; ``time_to_solution`` compares the same solve with the plain FP64
GPU CG.  ``e2e`` repeats the step through the C ABI with host buffers (the
right-hand side uploaded and the solution read back inside the timed region).

``--impl reference`` times the FP64 CPU oracle (the only other implementation
of this method here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HISQ Dslash HBM GB/s (% of peak); time-to-1e-10 solve, custom fmt vs FP64 GPU"
DIMS = (32, 32, 32, 64)
MASS = 0.01
TOL = 1e-10
DELTA = 0.1
PROF_EVERY = 8  # timed solves: stencil event pairs in one block of iterations out of eight
SLOPPY = "int20"
# the stencil's flop convention (16 complex 3x3 matrix-vector products of 66 flop plus 15 six-real adds)
FLOP_PER_SITE = 16 * 66 + 15 * 6
WORKLOAD = ("mixed-precision even/odd CG to 1e-10 (16-bit gauge / 20-bit fermion / FP32 sloppy, r12 long links, "
            "FP64 x, true residuals and reductions, delta 0.1) on a 32^3x64 lattice, m=0.01, seeded near-identity "
            "SU(3) links (eps 0.3, fat x0.8, staggered phases), Gaussian source")


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the stencil's code (comments and blank lines ignored)."""
    h = hashlib.sha256()
    for name in ("dslash.cuh", "codecs.cuh", "reduce.cuh", "finish.cuh", "ff.cuh"):
        with open(os.path.join(ROOT, "paper_2302_09224_gb300", "csrc", name)) as f:
            for line in f:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic():
    """Per-launch DRAM bytes of the stencil from the committed ncu summary, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "stencil_int20_32x32x32x64.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source hash:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram bytes per launch \(32\^3x64, mean of both passes\):\s*([0-9.eE+]+)", text)
    if not (m_hash and m_b) or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def aggregate(pg, ms, bytes_local, device):
    """Whole-job figures of N replicas: the slowest rank's time and every rank's bytes (weak scaling)."""
    ms_max = max_over_ranks(pg, ms, device)
    total = sum_over_ranks(pg, bytes_local, device)
    return ms_max, total / (ms_max / 1e3) / 1e9


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v, device):
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v, device):
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def config_dict(args, world=1):
    """The workload's description, identical in both arms' lines."""
    return {"workload": WORKLOAD, "lattice": list(DIMS), "mass": MASS, "tol": TOL, "delta": DELTA,
            "sloppy": "fix16/int20/f32 r12", "l2": "no flush: every step streams >1 GB per iteration "
            "(links 0.5 GB per stencil pass), far above the 129 MB L2",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "m_ee": "one fused pass" if getattr(args, "fused", False) else "two stencil passes",
            "kernel_chain": "sequential launches" if getattr(args, "no_pdl", False)
            else "programmatic dependent launch",
            "cg_scalars": "one-block sums" if getattr(args, "no_split", False)
            else "summed by every block of the kernel that uses them"}


def oracle_sample(fat_h, lng_h, b_h, iters):
    """Time `iters` FP64 CG iterations of the oracle on the host cores."""
    import oracle

    t0 = time.perf_counter()
    x, st, it, tr = oracle.cg(DIMS, fat_h, lng_h, MASS, b_h, TOL, maxiter=iters)
    dt = time.perf_counter() - t0
    return dt, it, oracle.get_threads()


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    from paper_2302_09224_gb300 import synth

    oracle.build()
    fat, lng = synth.gauge_pair(DIMS, seed=0)
    b = synth.spinor(DIMS, synth.rhs_seed(0))
    fat_h, lng_h, b_h = fat.numpy(), lng.numpy(), b.numpy()
    sample_iters = args.ref_iters
    # one step = a bounded sample of the workload: `sample_iters` iterations of the oracle's CG on the same
    # system, timed whole (the initial and final residual operator applications included); its value counts
    # the headline solve's algorithmic bytes per iteration for each iteration done
    bytes_per_iter = args.solve_bytes / args.solve_iters
    steps_s, iters_done, cores = [], [], 1
    for s in range(args.warmup + args.steps):
        dt, it, cores = oracle_sample(fat_h, lng_h, b_h, sample_iters)
        if s >= args.warmup:
            steps_s.append(dt)
            iters_done.append(it)
    total_s = sum(steps_s)
    value = bytes_per_iter * sum(iters_done) / total_s / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / len(steps_s) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {sample_iters} FP64 CG iterations of the C oracle (OpenMP) on "
                                       f"the full 32^3x64 system, {bytes_per_iter / 1e9:.3f} GB of the GPU solve's "
                                       f"algorithmic traffic per iteration"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    force_shapes(args)
    if args.fused:
        hisq.hisq_mee_fused(1)
    if args.no_pdl:
        hisq.hisq_programmatic_launch(0)
    if args.no_split:
        hisq.hisq_cg_split_scalars(0)
    ctx = hisq.hisq_create(local)
    fat, lng = synth.gauge_pair(DIMS, seed=0, device=dev)
    g = hisq.hisq_load_gauge(ctx, DIMS, fat, lng)
    b = synth.spinor(DIMS, synth.rhs_seed(rank), device=dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.Stream(device=dev)

    def params(name, delta, on_device=1, graph=1, recon=None):
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.delta, p.on_device = MASS, TOL, delta, on_device
        p.sloppy = hisq.prec(name, recon or (12 if name != "f64" else 18))
        p.use_graph = graph
        p.stream = stream.cuda_stream
        p.maxiter = 100000
        return p

    p = params(SLOPPY, DELTA)
    # one untimed solve with per-launch accounting: algorithmic bytes per step
    hisq.hisq_profile_reset(ctx)
    hisq.hisq_profile_enable(ctx, True)
    with torch.cuda.stream(stream):
        st, info0 = hisq.hisq_cg(ctx, g, p, b, x)
    bytes_per_step = sum(hisq.hisq_profile_read(ctx, k).bytes for k in range(3))
    blas0 = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_BLAS)  # every class timed in this untimed solve
    for _ in range(max(0, args.warmup - 1)):
        x.zero_()
        with torch.cuda.stream(stream):
            hisq.hisq_cg(ctx, g, p, b, x)
    shapes = {"plain": hisq.hisq_stencil_config_in_use(g, p.sloppy, False),
              "reducing": hisq.hisq_stencil_config_in_use(g, p.sloppy, True)}
    hisq.hisq_profile_reset(ctx)
    # the timed solves carry event pairs around the stencil launches only (one pair around the two
    # passes of each M_ee, counted as two launches), in one block of iterations out of PROF_EVERY (each
    # pair costs device time; the other blocks run an identical graph without them)
    hisq.hisq_profile_select(ctx, 1 << hisq.HISQ_PROF_STENCIL)
    hisq.hisq_profile_sample(ctx, PROF_EVERY)
    torch.cuda.synchronize()
    barrier(pg)
    l0 = hisq.hisq_launch_count(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            x.zero_()  # start each solve from x = 0 (on the default stream, ordered by the sync below)
            torch.cuda.current_stream().synchronize()
            with torch.cuda.stream(stream):
                st, info = hisq.hisq_cg(ctx, g, p, b, x)
            infos.append((st, info.iters, info.true_residual, info.reliable_updates))
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = hisq.hisq_launch_count(ctx) - l0
    stencil = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
    hisq.hisq_profile_enable(ctx, False)
    hisq.hisq_profile_select(ctx, 0xFFFFFFFF)
    hisq.hisq_profile_sample(ctx, 1)
    barrier(pg)
    ms_max, value = aggregate(pg, ms, bytes_per_step * args.steps, dev)

    # the CPU baseline: the oracle's FP64 CG on the host cores, a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        oracle.build()
        fat_h, lng_h, b_h = fat.cpu().numpy(), lng.cpu().numpy(), b.cpu().numpy()
        dt, it, cores = oracle_sample(fat_h, lng_h, b_h, args.ref_iters)
        per_iter = dt / (it + 2)
        cpu_step = per_iter * info.iters
        # one stencil pass on all cores and on one thread, and one thread's CG iteration
        xo = synth.spinor(DIMS, synth.rhs_seed(1)).numpy()
        t0 = time.perf_counter()
        oracle.dslash(DIMS, fat_h, lng_h, 0, xo)
        pass_all = time.perf_counter() - t0
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.dslash(DIMS, fat_h, lng_h, 0, xo)
        pass_one = time.perf_counter() - t0
        dt1, it1, _ = oracle_sample(fat_h, lng_h, b_h, 1)
        oracle.set_threads(cores)
        cpu = {"value": bytes_per_step / cpu_step / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.ref_iters} FP64 CG iterations of the C oracle (OpenMP) on the full 32^3x64 "
                         f"lattice, {dt:.1f} s, extrapolated to the GPU solve's {info.iters} iterations",
               "cg_iteration_s": per_iter, "cg_iteration_s_1_thread": dt1 / (it1 + 2),
               "stencil_pass_s": pass_all, "stencil_pass_s_1_thread": pass_one}

    # end to end through the ABI with host buffers
    # the right-hand side and the solution in pinned host memory (the copies run at full link speed)
    bh = b.cpu().pin_memory().numpy()
    xh = torch.zeros(tuple(b.shape), dtype=torch.float64).pin_memory().numpy()
    ph = params(SLOPPY, DELTA, on_device=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        xh[:] = 0
        hisq.hisq_cg(ctx, g, ph, bh, xh)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(pg, e2e_s, dev)
    e2e_value = sum_over_ranks(pg, bytes_per_step, dev) / e2e_s / 1e9

    # plain FP64 GPU CG on the same system (time-to-solution comparison)
    p64 = params("f64", 0.0)
    x64 = torch.zeros_like(b)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    with torch.cuda.stream(stream):
        st64, info64 = hisq.hisq_cg(ctx, g, p64, b, x64)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_s = f0.elapsed_time(f1) / 1e3

    # the same solve with every other sloppy storage triplet of Sec. 4 (one warm-up solve each: the
    # gauge copy in that format and the launch-shape tuning happen there), and BiCGStab(4) on the
    # full M = 2m + D; each timed with events on the solver's stream
    def timed(fn):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        with torch.cuda.stream(stream):
            res = fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return res, a0.elapsed_time(a1) / 1e3

    formats = {}
    if not args.no_formats:
        # the FP64-class 30-bit triplet computes in FP32 pairs, where rebuilding the third row of a
        # 12-real link costs more than reading 18 reals: it is timed with 18-real long links
        for name in ("f32", "half", "int30f32", "int30", "int14", "int20se"):
            pf = params(name, DELTA, recon=18 if name == "int30" else None)
            xf = torch.zeros_like(b)
            with torch.cuda.stream(stream):
                hisq.hisq_cg(ctx, g, pf, b, xf)
            xf.zero_()
            (stf, inff), sec = timed(lambda: hisq.hisq_cg(ctx, g, pf, b, xf))
            formats[name] = {"s": sec, "speedup_vs_fp64": fp64_s / sec, "iters": inff.iters,
                             "long_links": "r18" if name == "int30" else "r12",
                             "reliable_updates": inff.reliable_updates, "true_residual": inff.true_residual,
                             "status": hisq.STATUS_NAMES[stf]}
        formats["int20"] = {"s": ms / args.steps / 1e3, "speedup_vs_fp64": fp64_s / (ms / args.steps / 1e3),
                            "iters": infos[-1][1], "reliable_updates": infos[-1][3],
                            "true_residual": infos[-1][2], "status": hisq.STATUS_NAMES[infos[-1][0]]}
        # the same int20 solve with the error-estimate reliable-update trigger instead of delta = 0.1
        pd = params(SLOPPY, DELTA)
        pd.ru_trigger = 1
        xd = torch.zeros_like(b)
        with torch.cuda.stream(stream):
            hisq.hisq_cg(ctx, g, pd, b, xd)
        xd.zero_()
        (std, infd), secd = timed(lambda: hisq.hisq_cg(ctx, g, pd, b, xd))
        formats["int20_error_estimate_trigger"] = {"s": secd, "iters": infd.iters,
                                                   "reliable_updates": infd.reliable_updates,
                                                   "true_residual": infd.true_residual,
                                                   "status": hisq.STATUS_NAMES[std]}
        # the full-lattice system (2m + D) x = b by even/odd reduction around the same CG
        bf = synth.spinor(DIMS, synth.rhs_seed(rank), full=True, device=dev)
        xs = torch.zeros_like(bf)
        with torch.cuda.stream(stream):
            hisq.hisq_solve_full(ctx, g, params(SLOPPY, DELTA), bf, xs)
        xs.zero_()
        (stf2, inf2), secf = timed(lambda: hisq.hisq_solve_full(ctx, g, params(SLOPPY, DELTA), bf, xs))
        formats["full_system_int20"] = {"s": secf, "iters": inf2.iters, "reliable_updates": inf2.reliable_updates,
                                        "true_residual_full": inf2.true_residual, "status": hisq.STATUS_NAMES[stf2]}
        xb = torch.zeros_like(bf)
        pb = params(SLOPPY, DELTA)
        pb.l = 4
        with torch.cuda.stream(stream):
            hisq.hisq_bicgstabl(ctx, g, pb, bf, xb)
        xb.zero_()
        (stb, infb), secb = timed(lambda: hisq.hisq_bicgstabl(ctx, g, pb, bf, xb))
        formats["bicgstab4_int20_full_M"] = {"s": secb, "cycles": infb.iters, "matvecs": infb.matvecs,
                                            "reliable_updates": infb.reliable_updates,
                                            "true_residual": infb.true_residual, "status": hisq.STATUS_NAMES[stb]}
        # the headline solve with the long links in the other storages (Sec. 1: 18 reals, 8 reals; 13 reals
        # for U(3) links): time to solution, and the stencil's passes in a short profiled solve
        for recon in (18, 13, 8):
            pr = params(SLOPPY, DELTA, recon=recon)
            xr = torch.zeros_like(b)
            with torch.cuda.stream(stream):
                hisq.hisq_cg(ctx, g, pr, b, xr)
            xr.zero_()
            (str_, infr), secr = timed(lambda: hisq.hisq_cg(ctx, g, pr, b, xr))
            hisq.hisq_profile_reset(ctx)
            hisq.hisq_profile_select(ctx, 1 << hisq.HISQ_PROF_STENCIL)
            hisq.hisq_profile_enable(ctx, True)
            ps = params(SLOPPY, DELTA, recon=recon)
            ps.maxiter = 64
            xr.zero_()
            with torch.cuda.stream(stream):
                hisq.hisq_cg(ctx, g, ps, b, xr)
            sr = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
            hisq.hisq_profile_enable(ctx, False)
            hisq.hisq_profile_select(ctx, 0xFFFFFFFF)
            formats[f"int20_long_r{recon}"] = {
                "s": secr, "iters": infr.iters, "reliable_updates": infr.reliable_updates,
                "true_residual": infr.true_residual, "status": hisq.STATUS_NAMES[str_],
                "stencil_us_per_pass": 1e3 * sr.ms / max(sr.launches, 1),
                "stencil_gbs": sr.bytes / max(sr.ms, 1e-9) / 1e6}

    # the FP64 baseline's stencil alone: a short profiled FP64 solve (its passes timed by events)
    hisq.hisq_profile_reset(ctx)
    hisq.hisq_profile_select(ctx, 1 << hisq.HISQ_PROF_STENCIL)
    hisq.hisq_profile_enable(ctx, True)
    p64s = params("f64", 0.0)
    p64s.maxiter = 64
    x64.zero_()
    with torch.cuda.stream(stream):
        hisq.hisq_cg(ctx, g, p64s, b, x64)
    s64 = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
    hisq.hisq_profile_enable(ctx, False)
    hisq.hisq_profile_select(ctx, 0xFFFFFFFF)
    vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
    fp64_stencil = {"us_per_pass": 1e3 * s64.ms / max(s64.launches, 1),
                    "gbs": s64.bytes / max(s64.ms, 1e-9) / 1e6,
                    "tflops": FLOP_PER_SITE * vh * s64.launches / max(s64.ms, 1e-9) / 1e9,
                    "launches": s64.launches, "note": "FP64/FP64/FP64 triplet, 18-real links, in a 64-iteration "
                                                      "profiled solve"}

    # the task's other configurations, at sizes that keep the default run within a few minutes
    extras = {}
    if not args.no_extras:
        extras["multishift_12_shifts_32x32x32x64"] = multishift_results(ctx, g, b, args.ms_pairs.split(","))
        extras["batched_16rhs_32x32x32x64"] = batched_results(ctx, g, DIMS, MASS, 16, ["int20"])
        reqs = synth.poisson_requests(args.serve_requests, rate_hz=200.0, seed=1, volumes=SERVE_VOLUMES)
        gauges, mine = load_volumes(ctx, reqs, {DIMS: g})
        extras["serving"] = serve_results(ctx, gauges, reqs, True)
        extras["serving"]["workload"] = (f"{args.serve_requests} Poisson requests at 200/s (seed 1), volumes "
                                         "8^4/16^4/24^3x48/32^3x64, 30% multi-shift (8 shifts), against the same "
                                         "requests solved one after another")
        for gm in mine:
            hisq.hisq_free_gauge(ctx, gm)

    peak, peak_kind = measured_peak()
    achieved = stencil.bytes / (stencil.ms / 1e3) / 1e9 if stencil.ms > 0 else 0.0
    per_launch_bytes = stencil.bytes / max(1, stencil.launches)
    traffic = profiled_traffic()
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(args, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": ("mee_fused_kernel<FIX16, INT20, float, r12> (M_ee in one pass, links once)"
                                if args.fused else "dslash_kernel<FIX16, INT20, float, r12> (both passes of M_ee)"),
                     "bytes_per_launch": per_launch_bytes, "launches": stencil.launches,
                     "sampling": f"one event pair around the two stencil launches of each M_ee (their mean: half "
                                 f"the span) in one block of iterations in {PROF_EVERY} of the timed solves",
                     "launch_shapes": shapes,
                     "ms_per_launch": stencil.ms / max(1, stencil.launches)},
        "blas": {"achieved_gbs": blas0.bytes / (blas0.ms / 1e3) / 1e9 if blas0.ms > 0 else 0.0,
                 "share_of_step": blas0.ms / (ms / args.steps) if ms > 0 else 0.0,
                 "note": "from the untimed profiled solve (every kernel class timed)"},
        "time_to_solution": {"custom_s": ms / args.steps / 1e3, "fp64_s": fp64_s,
                             "speedup_vs_fp64": fp64_s / (ms / args.steps / 1e3),
                             "iters_custom": infos[-1][1], "iters_fp64": info64.iters,
                             "reliable_updates": infos[-1][3],
                             "true_residual_custom": infos[-1][2], "true_residual_fp64": info64.true_residual,
                             "status": [hisq.STATUS_NAMES[i[0]] for i in infos] + [hisq.STATUS_NAMES[st64]]},
        "stencil_gflops": FLOP_PER_SITE * (DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2) * stencil.launches
                          / (stencil.ms / 1e3) / 1e9 if stencil.ms > 0 else 0.0,
        "formats_time_to_solution": formats,
        "fp64_stencil": fp64_stencil,
        "configs": extras,
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": int(bh.nbytes),
                "d2h_bytes_per_step": int(xh.nbytes), "s_per_step": e2e_s},
        "gpu_launches": int(sum_over_ranks(pg, launches, dev)),
        "clocks": clk.summary(),
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def force_shapes(args):
    """Apply --stencil-config (before any stencil launch)."""
    from paper_2302_09224_gb300 import hisq

    if not args.stencil_config:
        return
    v = [int(t) for t in args.stencil_config.split(",")]
    hisq.hisq_stencil_config(v[0])
    if len(v) > 1:
        hisq.hisq_stencil_config_reduce(v[1])


def run_stencil_only(args):
    """A few stencil applications on one lattice (the small case for ncu captures)."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    dims = tuple(int(v) for v in args.stencil.split(","))
    force_shapes(args)
    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    del fat, lng
    x = synth.spinor(dims, 1000, device="cuda")
    out = torch.empty_like(x)
    for _ in range(args.launches):
        hisq.hisq_dslash(ctx, g, hisq.prec(args.prec, 12), 0, 0.0, None, x, out, True)
    torch.cuda.synchronize()
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    print(json.dumps({"stencil": list(dims), "prec": args.prec, "launches": args.launches}))
    return 0


def run_solve_only(args):
    """One short mixed-precision solve (CG, or BiCGStab(4) with --solver bicgstab) on a given lattice: the case for
    ncu captures of the solver's kernels."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    dims = tuple(int(v) for v in args.solve.split(","))
    force_shapes(args)
    if args.no_split:
        hisq.hisq_cg_split_scalars(0)
    if args.fused:
        hisq.hisq_mee_fused(1)
    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    del fat, lng
    bicg = args.solver == "bicgstab"
    b = synth.spinor(dims, synth.rhs_seed(0), full=bicg, device="cuda")
    x = torch.zeros_like(b)
    p = hisq.hisq_default_params()
    p.mass, p.tol, p.delta, p.on_device = MASS, TOL, DELTA, 1
    p.sloppy = hisq.prec(args.prec, args.recon)
    p.maxiter = args.maxiter
    if bicg:  # BiCGStab(4) on the full M; maxiter counts operator applications
        p.l = 4
        st, info = hisq.hisq_bicgstabl(ctx, g, p, b, x)
    else:
        st, info = hisq.hisq_cg(ctx, g, p, b, x)
    torch.cuda.synchronize()
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    print(json.dumps({"solve": list(dims), "solver": args.solver, "prec": args.prec, "maxiter": args.maxiter,
                      "status": hisq.STATUS_NAMES.get(st, st), "iters": info.iters}))
    return 0


def run_batched_solve(args):
    """Short batched CG solves on one lattice for every (tile, kernel) pair: the batched stencil's time per
    launch and its algorithmic bandwidth (profiler events on the solver's stream), the small case for ncu
    captures of the batched kernels, and the sweep behind the tile tuner."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    dims = tuple(int(v) for v in args.batched_solve.split(","))
    nr = args.nrhs
    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    del fat, lng
    b = torch.stack([synth.spinor(dims, synth.rhs_seed(k), device="cuda") for k in range(nr)]).contiguous()
    tiles = [int(v) for v in args.rhs_tiles.split(",")]
    kernels = [int(v) for v in args.rhs_kernels.split(",")]
    out = []
    for T in tiles:
        for kern in kernels:
            p = hisq.hisq_default_params()
            p.mass, p.tol, p.delta, p.on_device = MASS, TOL, DELTA, 1
            p.sloppy = hisq.prec(args.prec, 12)
            p.maxiter = args.maxiter
            p.nrhs, p.rhs_tile, p.rhs_kernel = nr, T, kern
            x = torch.zeros_like(b)
            hisq.hisq_cg(ctx, g, p, b, x)  # tuning and warm-up
            x.zero_()
            hisq.hisq_profile_reset(ctx)
            hisq.hisq_profile_enable(ctx, True)
            st, info = hisq.hisq_cg(ctx, g, p, b, x)
            torch.cuda.synchronize()
            sten = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
            blas = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_BLAS)
            hisq.hisq_profile_enable(ctx, False)
            passes = max(sten.launches, 1)
            out.append({"tile": T, "kernel": ["tuned", "registers", "staged"][kern], "status": hisq.STATUS_NAMES.get(st, st),
                        "iters": info.iters, "stencil_ms_per_pass": sten.ms / passes,
                        "stencil_us_per_rhs_pass": 1e3 * sten.ms / passes / nr,
                        "stencil_gbs": sten.bytes / max(sten.ms, 1e-9) / 1e6,
                        "blas_us_per_rhs_iter": 1e3 * blas.ms / max(info.iters, 1) / nr})
            print(json.dumps(out[-1]), flush=True)
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    return 0


MS_SHIFTS, MS_MASS = 12, 0.005


def multishift_results(ctx, g, b, pairs):
    """Config 3: 12 shifts log-spaced in [1e-4, 1] on g's lattice, base m = 0.005, per-shift targets
    1e-10..1e-7; the multi-shift stage (all shifts in one fused update kernel per iteration) plus refinement,
    per (stage / refinement) format pair.  Each pair runs once untimed (gauge copy, tuning), then timed."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    sig = synth.shifts_logspaced(MS_SHIFTS, 1e-4, 1.0)
    tols = synth.shift_tolerances(MS_SHIFTS, 1e-10, 1e-7)
    res = {}
    # Table 3 pairs a higher-precision multi-shift stage with a lower-precision refinement (single/half
    # and 30-bit/20-bit), plus 20-bit for both; the FP64-class 30-bit triplet runs with 18-real long links
    for pair in pairs:
        ms_name, ref_name = pair.split("/")
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.delta, p.on_device = MS_MASS, min(tols), DELTA, 1
        p.sloppy = hisq.prec(ms_name, 18 if ms_name in ("f64", "int30") else 12)
        p.refine = hisq.prec(ref_name, 18 if ref_name in ("f64", "int30") else 12)
        p.maxiter = 100000
        xs = [torch.zeros_like(b) for _ in sig]
        hisq.hisq_multishift_cg(ctx, g, p, sig, tols, b, xs)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = hisq.hisq_multishift_cg(ctx, g, p, sig, tols, b, xs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tr = list(info.shift_resid)[:MS_SHIFTS]  # FP64 true residuals computed on the GPU after refinement
        res[pair] = {"s": dt, "status": hisq.STATUS_NAMES[st], "iters_multishift": info.iters,
                     "refine_iters_total": int(sum(list(info.refine_iters)[:MS_SHIFTS])),
                     "shift_iters": list(info.shift_iters)[:MS_SHIFTS],
                     "refine_iters": list(info.refine_iters)[:MS_SHIFTS],
                     "residual_after_multishift": list(info.shift_resid_ms)[:MS_SHIFTS], "true_residual": tr,
                     "targets_met": all(r <= t for r, t in zip(tr, tols))}
    return res


def batched_results(ctx, g, dims, m, nr, names, profile_iters=200):
    """Config 4's batched CG: nr Gaussian right-hand sides solved together (autotuned tile; each stencil
    launch loads every link once per tile) against the same systems solved one after another; the batched
    stencil's time per right-hand side and pass comes from a short profiled batched solve."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    b = torch.stack([synth.spinor(dims, synth.rhs_seed(k), device="cuda") for k in range(nr)]).contiguous()
    res = {}
    for name in names:
        def params(n, maxiter=100000):
            p = hisq.hisq_default_params()
            p.mass, p.tol, p.delta, p.on_device = m, TOL, DELTA, 1
            p.sloppy = hisq.prec(name, 12)
            p.maxiter = maxiter
            p.nrhs = n
            return p

        x = torch.zeros_like(b)
        hisq.hisq_cg(ctx, g, params(nr, 16), b, x)  # untimed: gauge copy, tile and shape tuning
        x.zero_()
        hisq.hisq_profile_reset(ctx)
        hisq.hisq_profile_enable(ctx, True)
        hisq.hisq_cg(ctx, g, params(nr, profile_iters), b, x)
        sten = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
        hisq.hisq_profile_enable(ctx, False)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = hisq.hisq_cg(ctx, g, params(nr), b, x)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        x1 = torch.zeros_like(b[0])
        iters1 = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nr):
            x1.zero_()
            _, i1 = hisq.hisq_cg(ctx, g, params(1), b[k], x1)
            iters1.append(i1.iters)
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t0
        res[name] = {"batched_s": t_batch, "sequential_s": t_single, "speedup": t_single / t_batch,
                     "status": hisq.STATUS_NAMES[st], "iters_max_batched": info.iters, "iters_single": iters1,
                     "true_residual_max": info.true_residual,
                     "stencil_us_per_rhs_pass": 1e3 * sten.ms / max(sten.launches, 1) / nr,
                     "stencil_gbs": sten.bytes / max(sten.ms, 1e-9) / 1e6}
    return res


def serve_results(ctx, gauges, reqs, sequential):
    """Config 5: the seeded Poisson stream submitted at its arrival times to the library's request loop
    (continuous batching); latency percentiles, throughput and, optionally, the same requests solved one
    after another on one stream."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    live = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        b = synth.spinor(r["dims"], r["rhs_seed"], device="cuda")
        if r["multishift"]:
            xs = torch.zeros((len(r["shifts"]),) + tuple(b.shape), dtype=torch.float64, device="cuda")
            t = hisq.hisq_submit(ctx, gauges[r["dims"]], hisq.HISQ_REQ_MULTISHIFT, r["mass"], b, xs, True,
                                 sigma=r["shifts"], shift_tol=[r["tol"]] * len(r["shifts"]))
        else:
            xs = torch.zeros_like(b)
            t = hisq.hisq_submit(ctx, gauges[r["dims"]], hisq.HISQ_REQ_CG, r["mass"], b, xs, True, tol=r["tol"])
        live.append((t, b, xs))
    statuses = {}
    for t, b, xs in live:
        st, _ = hisq.hisq_wait(ctx, t, 3600.0)
        statuses[hisq.STATUS_NAMES[st]] = statuses.get(hisq.STATUS_NAMES[st], 0) + 1
    wall = time.perf_counter() - t0
    s = hisq.hisq_serve_stats(ctx)
    line = {"requests": len(reqs), "completed": s.completed, "statuses": statuses,
            "latency_p50_s": s.latency_p50_s, "latency_p99_s": s.latency_p99_s, "solves_per_s": s.solves_per_s,
            "wall_s": wall}
    if sequential:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for r in reqs:
            b = synth.spinor(r["dims"], r["rhs_seed"], device="cuda")
            p = hisq.hisq_default_params()
            p.mass, p.tol, p.on_device = r["mass"], r["tol"], 1
            if r["multishift"]:
                xs = [torch.zeros_like(b) for _ in r["shifts"]]
                hisq.hisq_multishift_cg(ctx, gauges[r["dims"]], p, r["shifts"], [r["tol"]] * len(r["shifts"]), b,
                                        xs)
            else:
                hisq.hisq_cg(ctx, gauges[r["dims"]], p, b, torch.zeros_like(b))
        torch.cuda.synchronize()
        seq = time.perf_counter() - t1
        line.update({"sequential_s": seq, "throughput_vs_sequential": seq / wall})
    return line


SERVE_VOLUMES = ((8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64))


def load_volumes(ctx, reqs, have=None):
    """Resident gauge fields for the requests' volumes (reusing `have`: {dims: gauge})."""
    from paper_2302_09224_gb300 import hisq, synth

    gauges, mine = dict(have or {}), []
    for d in sorted({r["dims"] for r in reqs}):
        if d not in gauges:
            fat, lng = synth.gauge_pair(d, seed=0, device="cuda")
            gauges[d] = hisq.hisq_load_gauge(ctx, d, fat, lng)
            mine.append(gauges[d])
            del fat, lng
    return gauges, mine


def run_multishift(args):
    """Config 3 alone, every pair of --ms-pairs (the default run reports it too)."""
    from paper_2302_09224_gb300 import hisq, synth

    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(DIMS, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, DIMS, fat, lng)
    b = synth.spinor(DIMS, synth.rhs_seed(0), device="cuda")
    res = multishift_results(ctx, g, b, args.ms_pairs.split(","))
    print(json.dumps({"workload": "multi-shift CG, 12 shifts log-spaced 1e-4..1, 32^3x64, m=0.005, "
                      "targets 1e-10..1e-7; results per (multi-shift stage / refinement) format pair",
                      "results": res}))
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    return 0


def run_batched(args):
    """Config 4: 16 right-hand sides on 48^3x96 (m = 0.002), batched against one after another."""
    import torch

    from paper_2302_09224_gb300 import hisq, synth

    dims, m, nr = (48, 48, 48, 96), 0.002, 16
    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    del fat, lng
    torch.cuda.empty_cache()
    res = batched_results(ctx, g, dims, m, nr, args.formats.split(","))
    print(json.dumps({"workload": "batched CG, 16 Gaussian RHS on 48^3x96, m=0.002, tol 1e-10, autotuned tile",
                      "results": res}))
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    return 0


def run_serve(args):
    """Config 5 with --requests requests (the default run reports a shorter stream)."""
    from paper_2302_09224_gb300 import hisq, synth

    reqs = synth.poisson_requests(args.requests, rate_hz=200.0, seed=1, volumes=SERVE_VOLUMES)
    ctx = hisq.hisq_create(0)
    gauges, mine = load_volumes(ctx, reqs)
    line = serve_results(ctx, gauges, reqs, args.serve_sequential)
    line["workload"] = (f"serving: {args.requests} Poisson requests at 200/s (seed 1), volumes "
                        "8^4/16^4/24^3x48/32^3x64, 30% multi-shift (8 shifts)")
    print(json.dumps(line))
    for g in mine:
        hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-iters", type=int, default=12, help="oracle CG iterations per CPU sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-formats", action="store_true", help="skip the other storage formats' solves")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the multi-shift, batched and serving configurations of the default line")
    ap.add_argument("--serve-requests", type=int, default=30, help="requests of the default line's serving stream")
    ap.add_argument("--fused", action="store_true", help="M_ee as one fused pass (hisq_mee_fused)")
    ap.add_argument("--no-pdl", action="store_true", help="launch the solver kernels without programmatic "
                    "dependent launch (hisq_programmatic_launch(0))")
    ap.add_argument("--no-split", action="store_true", help="sum the CG iteration's alpha and beta once, in a "
                    "one-block launch and a last block (hisq_cg_split_scalars(0))")
    ap.add_argument("--solve-iters", type=int, default=2866,
                    help="reference arm: iterations of one GPU solve (extrapolation unit)")
    ap.add_argument("--solve-bytes", type=float, default=3.605e12,
                    help="reference arm: algorithmic bytes of one GPU solve")
    ap.add_argument("--stencil", default=None, help="LX,LY,LZ,LT: only run stencil applications (profiling)")
    ap.add_argument("--prec", default="int20")
    ap.add_argument("--recon", type=int, default=12, help="long-link storage (18, 13, 12 or 8 reals) of --solve")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--stencil-config", default="",
                    help="force the stencil launch shapes: A (both passes) or A,B (plain, reducing), each 0..4")
    ap.add_argument("--solve", default=None, help="LX,LY,LZ,LT: only one short CG solve (profiling)")
    ap.add_argument("--solver", default="cg", choices=["cg", "bicgstab"],
                    help="solver of --solve: CG on M_ee, or BiCGStab(4) on the full M")
    ap.add_argument("--workload", default="solve", choices=["solve", "multishift", "batched", "serve"],
                    help="solve: the headline line; the others print their own measurement line")
    ap.add_argument("--formats", default="int20,half", help="sloppy formats for --workload batched")
    ap.add_argument("--ms-pairs", default="f32/half,int30/int20,int20/int20",
                    help="multi-shift stage / refinement formats for --workload multishift")
    ap.add_argument("--requests", type=int, default=100, help="requests of --workload serve")
    ap.add_argument("--serve-sequential", action="store_true",
                    help="--workload serve: also solve the requests one after another for comparison")
    ap.add_argument("--maxiter", type=int, default=20)
    ap.add_argument("--batched-solve", default=None,
                    help="LX,LY,LZ,LT: short batched CG solves per (tile, kernel), batched stencil timing (profiling)")
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--rhs-tiles", default="1,2,4,8,16")
    ap.add_argument("--rhs-kernels", default="1,2", help="1 registers, 2 staged neighbour loads, 0 tuned")
    args = ap.parse_args()
    if args.stencil:
        return run_stencil_only(args)
    if args.solve:
        return run_solve_only(args)
    if args.batched_solve:
        return run_batched_solve(args)
    if args.workload == "multishift":
        return run_multishift(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
