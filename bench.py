#!/usr/bin/env python
"""Benchmark of the complex-coordinate FMM hot path on GB300.

Workload (the 2D Helmholtz configuration): k = 20, N = 100,000 points on the
complexified bump curve t in [-40, 40] (bump height drawn in [0.3, 1.0],
imaginary part 0.5*sign(t)*max(|t|-4, 0)), single + double layer with the
curve's analytic normals, complex Gaussian densities, eps = 1e-6, leaf size
64. Inputs are synthetic (seeded, cfmm_inputs.curve2d_long). The headline runs in
MIXED precision (near field in complex64 arithmetic, translations FP64); the
same pass in FP64 is reported beside it, and both are checked against the
direct sum on 100 sampled targets.

One step = one pass of the whole hot path on inputs resident in HBM:
cfmm_plan (bounding box, Morton keys, radix sort, tree, level restriction,
centres, Lists 1-4, expansion orders, translation tables) + cfmm_apply
(P2M, M2M, M2L, P2L, L2L, P2P, M2P, L2P, un-permute) + cfmm_destroy.
value = points per second of that pass; apply_only = the same for the apply
alone on a resident plan (the GMRES matvec).

Other lines (--workload): helm3d / lap3d, the 3D Helmholtz (k=10) and Laplace
surface workloads at N = 1e6; batch3d, one 3D Helmholtz surface (k=15, N=2e5)
with 64 right-hand sides plus 32 uneven surfaces, replayed as one CUDA graph;
serve, the serving loop on a Poisson stream of 2D and 3D requests (points/s
with p50/p99 latency). --n, --sep and --leaf override the workload for
profiler captures and parameter sweeps (not bench lines).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
Multi-GPU: replicas (each rank runs its own copy of the workload), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KAPPA, EPS, LEAF, N_POINTS = 20.0, 1e-6, 64, 100_000
METRIC = "complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 2D Helmholtz SLP+DLP, k=20, N=1e5)"
WORKLOAD = "2D Helmholtz SLP+DLP k=20, N=1e5 complexified curve t in [-40,40], eps=1e-6, leaf 64"
SEP, DIM, DLP = 1, 2, True
KERNEL = 1            # 1 = Helmholtz, 0 = Laplace
LEAF_FP64 = 64
# --workload helm3d: the 3D Helmholtz surface configuration (a second bench line,
# not the headline)
W3D = dict(KAPPA=10.0, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=1_000_000, SEP=2, DIM=3, DLP=False,
           METRIC="complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 3D Helmholtz SLP, k=10, N=1e6)",
           WORKLOAD="3D Helmholtz SLP k=10, N=1e6 complexified plane with bump (Halton in [-20,20]^2, "
                    "Im = 0.4 max(rho-6,0) (x,y)/rho), eps=1e-6, separation k=2, leaf 256 (MIXED) / 128 (FP64) "
                    "as picked by the leaf-size autotuner")
# --workload batch3d: the batched 3D Helmholtz configuration (one geometry with
# 64 right-hand sides plus 32 uneven geometries, all replayed as one CUDA graph)
W4 = dict(KAPPA=15.0, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=200_000, SEP=2, DIM=3, DLP=False,
          METRIC="complex-FMM pts/s at rel.err<=1e-6 (batched 3D Helmholtz SLP, k=15: N=2e5 x 64 RHS "
                 "+ 32 uneven geometries, one CUDA graph)",
          WORKLOAD="batched 3D Helmholtz SLP k=15, eps=1e-6: plane-with-bump surface N=2e5 (Halton in "
                   "[-20,20]^2, slope 0.4) with 64 RHS, plus 32 surfaces of N log-uniform in [1e4, 2e5], "
                   "bump widths U[0.5,3], imaginary slopes U[0.2,0.8], 1 RHS each; separation k=2; "
                   "leaf sizes from the autotuner per geometry")
# --workload lap3d: the 3D Laplace surface configuration (same surface as helm3d)
WL3D = dict(KAPPA=0.0, KERNEL=0, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=1_000_000, SEP=2, DIM=3, DLP=False,
            METRIC="complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 3D Laplace SLP, N=1e6)",
            WORKLOAD="3D Laplace SLP, N=1e6 complexified plane with bump (Halton in [-20,20]^2, "
                     "Im = 0.4 max(rho-6,0) (x,y)/rho), eps=1e-6, separation k=2, leaf 256 (MIXED) / 128 (FP64)")
STEP_NAMES = ["permute", "P2M", "M2M", "M2L", "P2L", "L2L", "P2P", "M2P+L2P", "unpermute"]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2509_05458_gb300 as cf
    from cfmm_inputs import curve2d_long, plane3d, densities

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    g = curve2d_long(N_POINTS, seed=0) if DIM == 2 else plane3d(N_POINTS, seed=0)
    dens_np = densities(g.n, seed=1, nrhs=1, ncomp=2 if DLP else 1)
    re, im = torch.from_numpy(g.re).to(dev), torch.from_numpy(g.im).to(dev)
    nre = torch.from_numpy(g.nrm_re).to(dev) if DLP else None
    nim = torch.from_numpy(g.nrm_im).to(dev) if DLP else None
    dens = torch.from_numpy(dens_np).to(dev)
    out = torch.empty((1, g.n), dtype=torch.complex128, device=dev)
    kernel = (cf.HELMHOLTZ if KERNEL else cf.LAPLACE) | cf.SLP | (cf.DLP if DLP else 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # work model of the workload (host bookkeeping, outside the timed regions)
    wp = cf.plan(DIM, kernel, KAPPA, EPS, re, im, nre, nim, leaf_size=LEAF, sep=SEP, stream=stream)
    work = work_model(wp)
    wp.destroy()

    def measure(precision, check):
        leaf = LEAF if precision == cf.MIXED else LEAF_FP64

        def step(timing=False):
            p = cf.plan(DIM, kernel, KAPPA, EPS, re, im, nre, nim, leaf_size=leaf, sep=SEP, stream=stream,
                        precision=precision)
            if timing:
                p.set_timing(True)
            p.apply(dens, out=out)
            t = p.timings() if timing else None
            info = p.info()
            p.destroy()
            return t, info

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        acc = None
        if check:
            from oracle.direct import direct
            idx = np.random.default_rng(1).choice(g.n, 100, replace=False)
            pts = g.re + 1j * g.im
            u0 = direct(DIM, KERNEL, KAPPA, pts, pts[idx], sigma=dens_np[0, 0],
                        tau=dens_np[0, 1] if DLP else None, nrm=(g.nrm_re + 1j * g.nrm_im) if DLP else None)
            u = out.cpu().numpy()[0, idx]
            acc = float(np.linalg.norm(u - u0) / np.linalg.norm(u0))
        clocks = ClockSampler(local)
        n0 = cf.launch_count()
        step_ms, kern = [], []
        _barrier(ws)
        torch.cuda.synchronize()
        clocks.start()
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            t, info = step(timing=True)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            kern.append(t)
        torch.cuda.synchronize()
        _barrier(ws)
        wall = time.perf_counter() - wall0
        clk = clocks.stop()
        launches = cf.launch_count() - n0
        ms = _max_over_ranks(statistics.mean(step_ms), ws, dev)
        # apply alone on a resident plan (the GMRES matvec)
        p = cf.plan(DIM, kernel, KAPPA, EPS, re, im, nre, nim, leaf_size=leaf, sep=SEP, stream=stream,
                    precision=precision)
        for _ in range(3):
            p.apply(dens, out=out)
        torch.cuda.synchronize()
        ap = []
        for _ in range(max(5, args.steps)):
            flush.zero_()
            ev0.record(stream)
            p.apply(dens, out=out)
            ev1.record(stream)
            ev1.synchronize()
            ap.append(ev0.elapsed_time(ev1))
        p.destroy()
        kt = np.mean(np.array(kern), axis=0)
        return dict(ms=ms, apply_ms=statistics.median(ap), kt=kt, acc=acc, clk=clk, wall=wall,
                    launches=launches // max(1, args.steps), info=info)

    if args.precision == "fp64":
        mixed = fp64 = measure(cf.FP64, rank == 0 and not args.skip_check)
    elif args.precision == "mixed":
        mixed = fp64 = measure(cf.MIXED, rank == 0 and not args.skip_check)
    else:
        mixed = measure(cf.MIXED, rank == 0 and not args.skip_check)
        fp64 = measure(cf.FP64, rank == 0 and not args.skip_check)

    # end to end through the C ABI with host buffers (copies inside the timed region), MIXED
    hre, him = g.re, g.im
    hnre, hnim = (g.nrm_re, g.nrm_im) if DLP else (None, None)
    hd = np.ascontiguousarray(dens_np)
    ho = np.empty((1, g.n), dtype=np.complex128)
    e2e = []
    for i in range(max(3, args.steps) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ph = cf.plan(DIM, kernel, KAPPA, EPS, hre, him, hnre, hnim, leaf_size=LEAF, sep=SEP, precision=cf.MIXED)
        ph.apply(hd, out=ho)
        ph.destroy()
        t1 = time.perf_counter()
        if i > 0:
            e2e.append(t1 - t0)
    e2e_s = statistics.median(e2e)
    h2d = (4 if DLP else 2) * hre.nbytes + hd.nbytes
    d2h = ho.nbytes

    if rank != 0:
        return
    kt = mixed["kt"]
    # roofline of the M2L (the dominant FP64 translation step, with an exact
    # algorithmic count); the near field runs beside the far field on its own
    # stream, so step times overlap and the longest one is reported beside it
    dom = int(np.argmax(kt))
    fp64_peak = 1250.0   # GFLOP/s: nominal dense FP64 of GB300 (no measured FP64 peak is provided)
    roof = dominant_roofline("M2L", kt[3], work, fp64_peak)
    roof["longest_step"] = {"step": STEP_NAMES[dom], "ms": float(kt[dom])}
    if M2L_TRAFFIC_BYTES is not None and DIM == 2 and N_POINTS == 100_000 and LEAF == 64:
        roof["traffic"] = M2L_TRAFFIC_BYTES
        roof["traffic_source"] = "profiles/ncu_m2l_helm2d_k20_n1e5.txt (k_m2l_chunk, one apply, DRAM read+write)"
    info = mixed["info"]
    line = {
        "metric": METRIC,
        "value": g.n * ws / (mixed["ms"] / 1e3),
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": g.n, "kappa": KAPPA, "eps": EPS, "leaf_size": LEAF,
                   "leaf_size_fp64": LEAF_FP64, "sep": SEP,
                   "layers": "SLP+DLP" if DLP else "SLP",
                   "precision": "MIXED (near field complex64, translations FP64)",
                   "parallelism": f"replicas{ws}",
                   "l2": "flushed (256 MB write) before every timed step",
                   "tree": {k: info[k] for k in ("nlevels", "nboxes", "nleaves", "l0", "p2p_pairs", "m2l_pairs")}},
        "apply_only": {"value": g.n / (mixed["apply_ms"] / 1e3), "unit": "points/s", "ms": mixed["apply_ms"]},
        "accuracy": {"rel_l2_vs_direct_100_targets": mixed["acc"], "eps": EPS},
        "fp64": {"value": g.n / (fp64["ms"] / 1e3), "ms_per_step": fp64["ms"],
                 "apply_only": g.n / (fp64["apply_ms"] / 1e3), "apply_ms": fp64["apply_ms"],
                 "accuracy": fp64["acc"],
                 "step_breakdown_ms": {STEP_NAMES[i]: float(fp64["kt"][i]) for i in range(9)}},
        "step_breakdown_ms": {STEP_NAMES[i]: float(kt[i]) for i in range(9)},
        # the near field (slot 6) runs on its own stream beside the far field
        "plan_ms": float(mixed["ms"] - (float(np.sum(kt)) - float(kt[6]))),
        "work": work,
        "roofline": roof,
        "e2e": {"value": g.n / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clk"],
        "clocks_fp64": fp64["clk"],
        "wall_s": mixed["wall"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)


def run_batch(args):
    """--workload batch3d: one step = one replay of the batch graph (every
    geometry's apply on its resident plan); value = point evaluations (points x
    right-hand sides, summed over the geometries) per second."""
    import numpy as np
    import torch

    import paper_2509_05458_gb300 as cf
    from paper_2509_05458_gb300.autotune import tune_leaf_size
    from cfmm_inputs import plane3d, plane3d_uneven, densities

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    geoms = [plane3d(N_POINTS, seed=0)] + plane3d_uneven()
    nrhs = [64] + [1] * (len(geoms) - 1)
    kernel = cf.HELMHOLTZ | cf.SLP
    main = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pts_re = [torch.from_numpy(g.re).to(dev) for g in geoms]
    pts_im = [torch.from_numpy(g.im).to(dev) for g in geoms]
    dens_np = [densities(g.n, seed=100 + i, nrhs=nrhs[i], ncomp=1) for i, g in enumerate(geoms)]
    dens = [torch.from_numpy(d).to(dev) for d in dens_np]
    evals = sum(g.n * r for g, r in zip(geoms, nrhs))

    def build(precision):
        cands = (128, 192, 256, 384) if precision == cf.MIXED else (64, 96, 128, 192)
        plans, outs, leaves, streams = [], [], [], []
        for i, g in enumerate(geoms):
            s = torch.cuda.Stream(device=dev)
            leaf, _ = tune_leaf_size(3, kernel, KAPPA, EPS, pts_re[i], pts_im[i], precision=precision,
                                     candidates=cands, reps=2, stream=s, sep=SEP)
            p = cf.plan(3, kernel, KAPPA, EPS, pts_re[i], pts_im[i], leaf_size=leaf, sep=SEP,
                        precision=precision, stream=s)
            plans.append(p)
            outs.append(torch.empty((nrhs[i], g.n), dtype=torch.complex128, device=dev))
            leaves.append(leaf)
            streams.append(s)
        torch.cuda.synchronize()
        b = cf.Batch([(plans[i], dens[i], outs[i]) for i in range(len(geoms))], main)
        main.synchronize()
        return plans, outs, leaves, streams, b

    def timed(fn, warmup, steps):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(main):
                flush.zero_()
            ev0.record(main)
            fn()
            ev1.record(main)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return ms

    def measure(precision, check):
        plans, outs, leaves, streams, b = build(precision)
        acc = None
        if check:
            from oracle.direct import direct
            errs = []
            rng = np.random.default_rng(1)
            for i, g in enumerate(geoms):
                nt = 60 if i == 0 else 20
                idx = rng.choice(g.n, nt, replace=False)
                pts = g.re + 1j * g.im
                for r in ((0, nrhs[i] - 1) if nrhs[i] > 1 else (0,)):
                    u0 = direct(3, 1, KAPPA, pts, pts[idx], sigma=dens_np[i][r, 0])
                    u = outs[i][r].cpu().numpy()[idx]
                    errs.append(float(np.linalg.norm(u - u0) / np.linalg.norm(u0)))
            acc = {"max_rel_l2": max(errs), "median_rel_l2": float(np.median(errs)),
                   "per_geometry_rhs0": [errs[0]] + errs[2:]}
        clocks = ClockSampler(local)
        n0 = cf.launch_count()
        _barrier(ws)
        torch.cuda.synchronize()
        clocks.start()
        ms = timed(b.replay, args.warmup, args.steps)
        torch.cuda.synchronize()
        _barrier(ws)
        clk = clocks.stop()
        launches = (cf.launch_count() - n0) // max(1, args.steps + args.warmup)

        # the same applies issued eagerly (host launches, one stream per geometry)
        def eager():
            for i, p in enumerate(plans):
                streams[i].wait_event(ev0)
                p.apply(dens[i], out=outs[i])
                main.wait_stream(streams[i])
        ems = timed(eager, 0, 1)   # one pass: a step of this workload takes seconds
        # per-step breakdown of the 64-RHS geometry (dominant kernel)
        plans[0].set_timing(True)
        plans[0].apply(dens[0], out=outs[0])
        kt = np.array(plans[0].timings())
        plans[0].set_timing(False)
        work = work_model(plans[0])
        # end to end: pinned host densities in, results out, around one replay
        hd = [torch.from_numpy(d).pin_memory() for d in dens_np]
        ho = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        e2e = []
        for k in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(main):
                for i in range(len(geoms)):
                    dens[i].copy_(hd[i], non_blocking=True)
                b.replay()
                for i in range(len(geoms)):
                    ho[i].copy_(outs[i], non_blocking=True)
            main.synchronize()
            if k > 0:
                e2e.append(time.perf_counter() - t0)
        out = dict(ms=_max_over_ranks(statistics.mean(ms), ws, dev), eager_ms=statistics.mean(ems), acc=acc,
                   clk=clk, launches=launches, kernels=b.kernels, leaves=leaves, kt=kt, work=work,
                   e2e_s=statistics.median(e2e), h2d=sum(d.nbytes for d in dens_np),
                   d2h=sum(o.numel() * 16 for o in outs), info=plans[0].info())
        b.destroy()
        for p in plans:
            p.destroy()
        return out

    check = rank == 0 and not args.skip_check
    mixed = measure(cf.MIXED, check)
    fp64 = measure(cf.FP64, check) if args.precision == "both" else None
    if rank != 0:
        return
    kt = mixed["kt"]
    dom = int(np.argmax(kt))
    work = dict(mixed["work"])
    work["m2l_flops"] *= nrhs[0]
    work["p2p_pairs"] *= nrhs[0]
    roof = dominant_roofline("M2L", kt[3], work, 1250.0)
    roof["longest_step"] = {"step": STEP_NAMES[dom], "ms": float(kt[dom])}
    roof["scope"] = "the 64-RHS geometry's apply, timed alone with per-step events"
    line = {
        "metric": METRIC,
        "value": evals * ws / (mixed["ms"] / 1e3),
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "geometries": len(geoms), "points": [g.n for g in geoms],
                   "nrhs": nrhs, "point_evaluations_per_step": evals, "kappa": KAPPA, "eps": EPS, "sep": SEP,
                   "leaf_sizes": mixed["leaves"], "precision": "MIXED (near field complex64, translations FP64)",
                   "parallelism": f"replicas{ws}", "l2": "flushed (256 MB write) before every timed step"},
        "accuracy": mixed["acc"],
        "eager_same_applies": {"value": evals / (mixed["eager_ms"] / 1e3), "unit": "points/s",
                               "ms": mixed["eager_ms"]},
        "step_breakdown_ms_64rhs": {STEP_NAMES[i]: float(kt[i]) for i in range(9)},
        "work_64rhs": work,
        "roofline": roof,
        "e2e": {"value": evals / mixed["e2e_s"], "unit": "points/s", "h2d_bytes_per_step": int(mixed["h2d"]),
                "d2h_bytes_per_step": int(mixed["d2h"])},
        "gpu_launches": int(mixed["kernels"]),
        "gpu_launches_counted": int(mixed["launches"]),
        "clocks": mixed["clk"],
    }
    if fp64:
        line["fp64"] = {"value": evals / (fp64["ms"] / 1e3), "ms_per_step": fp64["ms"], "accuracy": fp64["acc"],
                        "leaf_sizes": fp64["leaves"], "clocks": fp64["clk"]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)


def run_serve(args):
    """--workload serve: the serving loop on a Poisson stream of apply requests
    (dims 2 and 3, Laplace or Helmholtz, N log-uniform in [1e3, nmax], eps in
    {1e-3, 1e-6, 1e-9}, 1-20 matvecs each). One step = one whole stream; value
    = point evaluations completed per second of wall time; p50/p99 request
    latency (arrival to last result on the host) beside it. A short stream of
    small requests runs first, untimed."""
    import torch

    from paper_2509_05458_gb300.serving import Server, make_stream, summarize

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    srv = Server(slots=args.slots, device=local)
    warm = make_stream(max(4, args.warmup), seed=99 + rank, rate_hz=100.0, nmin=1000, nmax=20000, dims=(2, 3))
    srv.run(warm, realtime=False)
    runs = []
    clocks = ClockSampler(local)
    _barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        reqs = make_stream(args.requests, seed=7 + 1000 * k + rank, rate_hz=args.rate, nmin=1000,
                           nmax=args.nmax, dims=(2, 3))
        t0 = time.perf_counter()
        res = srv.run(reqs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = summarize(res, wall)
        st["evaluations"] = sum(len(r.rhs) * r.n for r in reqs)
        runs.append(st)
    _barrier(ws)
    clk = clocks.stop()
    wall = _max_over_ranks(sum(r["wall_s"] for r in runs), ws, dev)
    if rank != 0:
        return
    evals = sum(r["evaluations"] for r in runs)
    line = {
        "metric": "complex-FMM serving: points/s and p50/p99 solve latency (Poisson stream, dims 2+3)",
        "value": evals * ws / wall,
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / max(1, args.steps),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"serving loop: Poisson stream of {args.requests} apply requests at "
                               f"{args.rate} Hz, dim in {{2,3}}, Laplace or Helmholtz (k in [1,50], 3D mapped "
                               f"to [1,10]), N log-uniform in [1e3, {args.nmax:.0e}], eps in {{1e-3,1e-6,1e-9}}, "
                               "1-20 matvecs per request on a resident plan, admission by free HBM",
                   "slots": args.slots, "requests_per_step": args.requests, "rate_hz": args.rate,
                   "nmax": args.nmax, "parallelism": f"replicas{ws}",
                   "timing": "host wall clock per stream (latency is arrival to result on the host)"},
        "p50_s": runs[-1]["p50_s"], "p99_s": runs[-1]["p99_s"], "mean_s": runs[-1]["mean_s"],
        "errors": sum(r["errors"] for r in runs),
        "error_kinds": runs[-1]["error_kinds"],
        "streams": runs,
        "e2e": {"value": evals * ws / wall, "unit": "points/s",
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "the stream itself is end to end: host points and densities in, host results out"},
        "roofline": None,
        "gpu_launches": None,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def work_model(p):
    """Algorithmic work of one apply: List-2 pairs and M2L flops (8 flops per
    complex multiply-add, (2P+1)^2 per pair at the pair's level), List-1 pairs."""
    import numpy as np
    inf = p.info()
    t = p.export_tree()
    P = p.orders()
    off, _ = p.export_list(2)
    cnt = np.diff(off)
    m2l_flops = 0
    pairs_per_level = {}
    for l in range(inf["nlevels"]):
        npairs = int(cnt[t["level"] == l].sum())
        if npairs:
            pairs_per_level[int(l)] = npairs
            if DIM == 2:
                m2l_flops += npairs * 8 * (2 * int(P[l]) + 1) ** 2
            else:
                m2l_flops += npairs * (m2l_flops_pair_3d(int(P[l])) if KERNEL else m2l_flops_pair_lap3d(int(P[l])))
    return {"p2p_pairs": int(inf["p2p_pairs"]), "m2l_pairs": int(inf["m2l_pairs"]),
            "m2l_pairs_per_level": pairs_per_level, "orders": [int(x) for x in P],
            "m2l_flops": int(m2l_flops), "p2p_flops_per_pair": P2P_FLOPS_PER_PAIR}


def m2l_flops_pair_3d(P):
    """FP64 flops of one 3D Helmholtz point-and-shoot M2L at order P as the CUDA
    path computes it: four fixed-rotation products (sum_n n(n+1) real x complex
    multiply-adds each, 4 flops), the coaxial recurrence (sum_j j^2 rows, three
    real x complex multiply-adds, 12 flops) and the coaxial product
    (sum_m (1 + [m > 0]) (P - m + 1)^2 complex multiply-adds, 8 flops)."""
    rot = 4 * 4 * P * (P + 1) * (P + 2) // 3
    rec = 12 * P * (P + 1) * (2 * P + 1) // 6
    app = 8 * sum((1 + (m > 0)) * (P - m + 1) ** 2 for m in range(P + 1))
    return rot + rec + app


def m2l_flops_pair_lap3d(P):
    """FP64 flops of one 3D Laplace point-and-shoot M2L at order P: the four
    fixed-rotation products (as for Helmholtz) and the z-axis solid-harmonic
    shift (sum_m (1 + [m > 0]) (P - m + 1)^2 complex multiply-adds, 8 flops)."""
    rot = 4 * 4 * P * (P + 1) * (P + 2) // 3
    app = 8 * sum((1 + (m > 0)) * (P - m + 1) ** 2 for m in range(P + 1))
    return rot + app


def dominant_roofline(name, ms, work, fp64_peak_gflops):
    """Roofline of the dominant kernel of the apply, FP64-ALU bound:
    M2L: work["m2l_flops"]; P2P: List-1 pairs x FP64 flops per pair."""
    flops = None
    if name == "M2L":
        flops = work["m2l_flops"]
    elif name == "P2P" and P2P_FLOPS_PER_PAIR:
        flops = work["p2p_pairs"] * P2P_FLOPS_PER_PAIR
    base = {"bound": "alu", "peak": fp64_peak_gflops, "unit": "GFLOP/s", "traffic": None, "kernel": name,
            "ms": float(ms),
            "peak_source": "nominal GB300 dense FP64, 1.25 TFLOP/s (MEASURED_PEAKS.json has no FP64 figure)"}
    if not flops:
        return dict(base, achieved=None, frac=None)
    ach = flops / (ms / 1e3) / 1e9
    return dict(base, achieved=ach, frac=ach / fp64_peak_gflops)


# FP64 operations of one near-field pair (2D Helmholtz SLP+DLP); 0 = not yet counted
P2P_FLOPS_PER_PAIR = 0
# DRAM bytes of the 2D Helmholtz M2L launches of one apply on the headline workload,
# from one ncu capture (profiles/ncu_m2l_helm2d_k20_n1e5.txt); None once the kernel changes
M2L_TRAFFIC_BYTES = 27_990_784


def cpu_baseline(args):
    """The oracle, as it stands, on a bounded sample of the workload, one core:
    2D, its FMM on 20,000 points of the same curve family (same k, eps, leaf
    size); 3D, its direct sum for 200 targets against all N sources (the oracle
    FMM's top level alone takes minutes there)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    if DIM == 3:
        code = ("import sys,time,json; sys.path.insert(0, %r)\n"
                "import numpy as np\n"
                "from cfmm_inputs import plane3d, densities\n"
                "from oracle.direct import direct\n"
                "g = plane3d(%d, seed=0); d = densities(g.n, seed=1, nrhs=1, ncomp=1)\n"
                "pts = g.re + 1j * g.im; idx = np.arange(200)\n"
                "t=time.perf_counter(); direct(3, %d, %r, pts, pts[idx], sigma=d[0,0]); t=time.perf_counter()-t\n"
                "print(json.dumps({'n': g.n, 's': t}))\n") % (ROOT, N_POINTS, KERNEL, KAPPA)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        if r.returncode != 0:
            return {"value": None, "unit": "points/s", "cores": 1, "kind": "oracle",
                    "sample": "failed: " + r.stderr.strip()[-200:]}
        o = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": 200 / o["s"], "unit": "points/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle direct sum (numpy), 200 targets against all {o['n']} sources: {o['s']:.1f} s; "
                          "points/s = targets evaluated per second"}
    code = ("import sys,time,json; sys.path.insert(0, %r)\n"
            "from cfmm_inputs import curve2d_long, densities\n"
            "from oracle import fmm2d\n"
            "g = curve2d_long(%d, seed=0); d = densities(g.n, seed=1, nrhs=1, ncomp=2)\n"
            "t=time.perf_counter(); fmm2d.apply(g.re, g.im, 1, %r, %r, %d, sigma=d[0,0], tau=d[0,1], "
            "nrm_re=g.nrm_re, nrm_im=g.nrm_im); t=time.perf_counter()-t\n"
            "print(json.dumps({'n': g.n, 's': t}))\n") % (ROOT, args.cpu_n, KAPPA, EPS, LEAF)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "points/s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr.strip()[-200:]}
    o = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": o["n"] / o["s"], "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle FMM (numpy/scipy) on {o['n']} points of the same curve family, "
                      f"same k/eps/leaf, SLP+DLP, one pass: {o['s']:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle, as it stands, on the host cores (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    times = []
    res = None
    for i in range(args.warmup + args.steps):
        res = cpu_baseline(args)
        if i >= args.warmup and res["value"]:
            times.append(res["value"])
    val = statistics.mean(times) if times else None
    line = {"metric": METRIC, "value": val, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": N_POINTS, "kappa": KAPPA, "eps": EPS, "leaf_size": LEAF,
                       "sep": SEP, "layers": "SLP+DLP" if DLP else "SLP", "precision": "FP64",
                       "parallelism": "cpu"},
            "cpu_baseline": {"value": val, "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": res["sample"] if res else None},
            "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-n", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"],
                    help="which passes to run (the headline needs both)")
    ap.add_argument("--workload", default="helm2d", choices=["helm2d", "helm3d", "lap3d", "batch3d", "serve"],
                    help="helm2d: the 2D Helmholtz headline; helm3d / lap3d: the 3D Helmholtz / Laplace "
                         "surface lines; batch3d: the batched 3D Helmholtz line; serve: the serving loop")
    ap.add_argument("--requests", type=int, default=60, help="serve: requests per stream")
    ap.add_argument("--rate", type=float, default=1.0, help="serve: Poisson arrival rate (Hz)")
    ap.add_argument("--nmax", type=int, default=1_000_000, help="serve: largest request size")
    ap.add_argument("--slots", type=int, default=4, help="serve: requests in flight")
    ap.add_argument("--n", type=int, default=0,
                    help="override the point count (small cases for profiler captures; not a bench line)")
    ap.add_argument("--sep", type=int, default=0, help="override the separation k (parameter sweeps)")
    ap.add_argument("--leaf", type=int, default=0, help="override the leaf size of both passes (parameter sweeps)")
    args = ap.parse_args()
    if args.workload == "helm3d":
        globals().update(W3D)
    elif args.workload == "lap3d":
        globals().update(WL3D)
    elif args.workload == "batch3d":
        globals().update(W4)
    if args.n > 0:
        globals()["N_POINTS"] = args.n
    if args.sep > 0:
        globals()["SEP"] = args.sep
    if args.leaf > 0:
        globals()["LEAF"] = globals()["LEAF_FP64"] = args.leaf
    if args.impl == "reference":
        args.warmup = max(0, min(args.warmup, 1))
        args.steps = max(1, min(args.steps, 2))
        run_reference(args)
    elif args.workload == "batch3d":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
