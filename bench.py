#!/usr/bin/env python
"""Benchmark of the complex-coordinate FMM hot path on GB300.

Headline workload (the 3D surface configuration): 3D Helmholtz single layer,
k = 10, N = 1,000,000 Halton points of the complexified plane with a bump
((x, y) in [-20, 20]^2, z = 0.5 exp(-(x^2 + y^2)), Im = 0.4 max(rho - 6, 0)
(x, y)/rho), complex Gaussian densities, eps = 1e-6, separation k = 2, leaf
256 (MIXED) / 128 (FP64). Inputs are synthetic (seeded, cfmm_inputs.plane3d).
The headline runs in MIXED precision (near field and L2P in complex64
arithmetic, translations FP64); the same pass in FP64 is reported beside it.
Both are checked against the library's FP64 direct sum on 1,000 sampled
targets, and, when the CPU baseline runs, against the oracle's direct sum on
its sample.

One step = one pass of the whole hot path on inputs resident in HBM:
cfmm_plan (bounding box, Morton keys, radix sort, tree, level restriction,
centres, Lists 1-4, expansion orders, translation tables) + cfmm_apply
(P2M, M2M, M2L, P2L, L2L, P2P, M2P, L2P, un-permute) + cfmm_destroy.
value = points per second of that pass; apply_only = the same for the apply
alone on a resident plan (the GMRES matvec).

Beside the headline, the same line carries the 3D Laplace pass on the same
surface and the 2D Helmholtz curve configuration (k = 20, N = 1e5, SLP+DLP,
eps = 1e-6, leaf 64), each MIXED and FP64 (--no-extras skips them).

Other lines (--workload): lap3d / helm2d alone; wobble, the paper's own wobbly curve and surface (Sec. 7.1)
at eps 1e-6 and 1e-12; batch3d, one 3D Helmholtz
surface (k=15, N=2e5) with 64 right-hand sides plus 32 uneven surfaces,
replayed as one CUDA graph; serve, the serving loop on a Poisson stream of 2D
and 3D requests (points/s with p50/p99 latency). --n, --sep and --leaf
override the workload for profiler captures and parameter sweeps (not bench
lines).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
Multi-GPU: replicas (each rank runs its own copy of the workload), weak scaling.
"""
from __future__ import annotations

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

WORKLOADS = {
    # the 3D surface configuration (the headline)
    "helm3d": dict(KAPPA=10.0, KERNEL=1, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=1_000_000, SEP=2, DIM=3,
                   DLP=False,
                   METRIC="complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 3D Helmholtz SLP, k=10, N=1e6)",
                   WORKLOAD="3D Helmholtz SLP k=10, N=1e6 complexified plane with bump (Halton in [-20,20]^2, "
                            "Im = 0.4 max(rho-6,0) (x,y)/rho), eps=1e-6, separation k=2, leaf 256 (MIXED) / "
                            "128 (FP64)"),
    # the 3D Laplace pass on the same surface
    "lap3d": dict(KAPPA=0.0, KERNEL=0, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=1_000_000, SEP=2, DIM=3,
                  DLP=False,
                  METRIC="complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 3D Laplace SLP, N=1e6)",
                  WORKLOAD="3D Laplace SLP, N=1e6 complexified plane with bump (Halton in [-20,20]^2, "
                           "Im = 0.4 max(rho-6,0) (x,y)/rho), eps=1e-6, separation k=2, leaf 256 (MIXED) / "
                           "128 (FP64)"),
    # the 2D curve configuration
    "helm2d": dict(KAPPA=20.0, KERNEL=1, EPS=1e-6, LEAF=64, LEAF_FP64=64, N_POINTS=100_000, SEP=1, DIM=2,
                   DLP=True,
                   METRIC="complex-FMM pts/s at rel.err<=1e-6 (mixed vs FP64 GPU; 2D Helmholtz SLP+DLP, k=20, "
                          "N=1e5)",
                   WORKLOAD="2D Helmholtz SLP+DLP k=20, N=1e5 complexified curve t in [-40,40], eps=1e-6, leaf 64"),
    # the batched 3D Helmholtz configuration (one geometry with 64 right-hand
    # sides plus 32 uneven geometries, all replayed as one CUDA graph)
    "batch3d": dict(KAPPA=15.0, KERNEL=1, EPS=1e-6, LEAF=256, LEAF_FP64=128, N_POINTS=200_000, SEP=-1, DIM=3,
                    DLP=False,
                    METRIC="complex-FMM pts/s at rel.err<=1e-6 (batched 3D Helmholtz SLP, k=15: N=2e5 x 64 RHS "
                           "+ 32 uneven geometries, one CUDA graph)",
                    WORKLOAD="batched 3D Helmholtz SLP k=15, eps=1e-6: plane-with-bump surface N=2e5 (Halton in "
                             "[-20,20]^2, slope 0.4) with 64 RHS, plus 32 surfaces of N log-uniform in [1e4, 2e5], "
                             "bump widths U[0.5,3], imaginary slopes U[0.2,0.8], 1 RHS each; separation per "
                             "geometry from its Lipschitz estimate; top level moved down where the rule's order "
                             "exceeds 63; leaf sizes from the autotuner per geometry"),
}
globals().update(WORKLOADS["helm3d"])
STEP_NAMES = ["permute", "P2M", "M2M", "M2L", "P2L", "L2L", "P2P", "M2P+L2P", "unpermute"]
# GB300 ALU peaks derived from unit counts and the maximum SM clock (2.07 GHz):
# 152 SMs x 2 FP64 FMA/clk x 2 flops, and 152 SMs x 128 FP32 FMA/clk x 2 flops
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07
CSRC = os.path.join(ROOT, "paper_2509_05458_gb300", "csrc")


def source_hash(files):
    """sha256 (first 16 hex digits) of the named CUDA sources: the build a
    profile summary under profiles/ was taken on."""
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def profile_figures(name, files):
    """key: value lines of profiles/<name>.txt, or None when the summary is
    missing or was taken on other sources than the current ones."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    d = {}
    for l in lines:
        if ":" in l and not l.startswith(("#", " ")):
            k, v = l.split(":", 1)
            d[k.strip()] = v.strip()
    if d.get("source_sha256") != source_hash(files):
        return None
    d["_path"] = "profiles/" + name
    return d


# the source file of each profiled kernel (a summary is used only while its
# recorded hash matches this file)
P2P_SOURCES = ("p2p.cu",)
TR3H_SOURCES = ("helm3d.cu",)


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


def _geometry(W, n=None):
    from cfmm_inputs import curve2d_long, plane3d
    n = n or W["N_POINTS"]
    return curve2d_long(n, seed=0) if W["DIM"] == 2 else plane3d(n, seed=0)


def measure_workload(args, W, dev, ws, rank, local, steps, warmup, check_targets=1000, e2e=True):
    """MIXED and FP64 passes of workload W: plan+apply steps (the bench step),
    the apply alone on a resident plan, per-step kernel times from a serialised
    apply (near field in line), accuracy against the library's FP64 direct sum
    on sampled targets, and (e2e) the same pass through the C ABI with host
    buffers."""
    import numpy as np
    import torch

    import paper_2509_05458_gb300 as cf
    from cfmm_inputs import densities

    DIM, DLP, KAPPA, EPS, SEP = W["DIM"], W["DLP"], W["KAPPA"], W["EPS"], W["SEP"]
    g = _geometry(W)
    dens_np = densities(g.n, seed=1, nrhs=1, ncomp=2 if DLP else 1)
    re, im = torch.from_numpy(g.re).to(dev), torch.from_numpy(g.im).to(dev)
    nre = torch.from_numpy(g.nrm_re).to(dev) if DLP else None
    nim = torch.from_numpy(g.nrm_im).to(dev) if DLP else None
    dens = torch.from_numpy(dens_np).to(dev)
    out = torch.empty((1, g.n), dtype=torch.complex128, device=dev)
    kernel = (cf.HELMHOLTZ if W["KERNEL"] else cf.LAPLACE) | cf.SLP | (cf.DLP if DLP else 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # reference values at sampled targets: the library's FP64 direct sum
    idx = np.sort(np.random.default_rng(1).choice(g.n, min(check_targets, g.n), replace=False))
    ref = None
    if check_targets:
        ti = torch.from_numpy(idx).to(dev)
        ref = cf.direct(DIM, kernel, KAPPA, re, im, re[ti].contiguous(), im[ti].contiguous(), dens, nre, nim,
                        precision=cf.FP64, stream=stream).cpu().numpy()[0]

    def plan(precision, leaf):
        return cf.plan(DIM, kernel, KAPPA, EPS, re, im, nre, nim, leaf_size=leaf, sep=SEP, stream=stream,
                       precision=precision)

    def measure(precision):
        leaf = W["LEAF"] if precision == cf.MIXED else W["LEAF_FP64"]

        def step():
            p = plan(precision, leaf)
            p.apply(dens, out=out)
            info = p.info()
            p.destroy()
            return info

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        n0 = cf.launch_count()
        step_ms = []
        _barrier(ws)
        torch.cuda.synchronize()
        clocks.start()
        wall0 = time.perf_counter()
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            info = step()
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize()
        _barrier(ws)
        wall = time.perf_counter() - wall0
        clk = clocks.stop()
        launches = cf.launch_count() - n0
        ms = _max_over_ranks(statistics.mean(step_ms), ws, dev)
        acc = None
        u_all = out.cpu().numpy()[0].copy()
        if ref is not None:
            u = u_all[idx]
            acc = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
        # the apply alone on a resident plan (the GMRES matvec)
        p = plan(precision, leaf)
        for _ in range(3):
            p.apply(dens, out=out)
        torch.cuda.synchronize()
        ap = []
        for _ in range(max(5, steps)):
            flush.zero_()
            ev0.record(stream)
            p.apply(dens, out=out)
            ev1.record(stream)
            ev1.synchronize()
            ap.append(ev0.elapsed_time(ev1))
        # per-step kernel times: the near field in line (timing mode 2), so no
        # step's events absorb the other stream's kernels; median of 3
        p.set_timing(2)
        kts = []
        for _ in range(3):
            flush.zero_()
            p.apply(dens, out=out)
            kts.append(p.timings())
        p.set_timing(0)
        kt = np.median(np.array(kts), axis=0)
        work = work_model(p, W)
        p.destroy()
        return dict(ms=ms, apply_ms=statistics.median(ap), kt=kt, acc=acc, clk=clk, wall=wall,
                    launches=launches // max(1, steps), info=info, work=work, leaf=leaf, u=u_all)

    # --precision fp64 / mixed measure one precision only (the headline slot
    # then holds that precision and the line has no FP64 entry beside it)
    if args.precision == "fp64":
        mixed, fp64 = measure(cf.FP64), None
    elif args.precision == "mixed":
        mixed, fp64 = measure(cf.MIXED), None
    else:
        mixed = measure(cf.MIXED)
        fp64 = measure(cf.FP64)

    e2e_line = None
    if e2e:
        # end to end through the C ABI with host buffers (copies inside the timed region), MIXED
        hre, him = g.re, g.im
        hnre, hnim = (g.nrm_re, g.nrm_im) if DLP else (None, None)
        hd = np.ascontiguousarray(dens_np)
        ho = np.empty((1, g.n), dtype=np.complex128)
        e2e_t = []
        for i in range(max(3, steps) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ph = cf.plan(DIM, kernel, KAPPA, EPS, hre, him, hnre, hnim, leaf_size=W["LEAF"], sep=SEP,
                         precision=cf.MIXED)
            ph.apply(hd, out=ho)
            ph.destroy()
            t1 = time.perf_counter()
            if i > 0:
                e2e_t.append(t1 - t0)
        e2e_s = _max_over_ranks(statistics.median(e2e_t), ws, dev)
        h2d = (4 if DLP else 2) * hre.nbytes + hd.nbytes
        e2e_line = {"value": g.n * ws / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(ho.nbytes)}
    return dict(g=g, dens_np=dens_np, idx=idx, out_mixed=None, mixed=mixed, fp64=fp64, e2e=e2e_line,
                precision=args.precision)


def summarize(W, r, ws):
    """The per-workload part of a bench line."""
    mixed, fp64 = r["mixed"], r["fp64"]
    n = r["g"].n
    kt = mixed["kt"]
    info = mixed["info"]
    out = {
        "value": n * ws / (mixed["ms"] / 1e3),
        "ms_per_step": mixed["ms"],
        "config": {"workload": W["WORKLOAD"], "n": n, "kappa": W["KAPPA"], "eps": W["EPS"],
                   "leaf_size": W["LEAF"], "leaf_size_fp64": W["LEAF_FP64"], "sep": W["SEP"],
                   "layers": "SLP+DLP" if W["DLP"] else "SLP",
                   "precision": ("FP64" if r["precision"] == "fp64" else
                                 "MIXED (near field and L2P complex64, translations FP64)"),
                   "tree": {k: info[k] for k in ("nlevels", "nboxes", "nleaves", "l0", "p2p_pairs", "m2l_pairs")}},
        "apply_only": {"value": n / (mixed["apply_ms"] / 1e3), "unit": "points/s", "ms": mixed["apply_ms"]},
        "accuracy": {"rel_l2_vs_fp64_direct_sampled": mixed["acc"], "targets": int(len(r["idx"])),
                     "eps": W["EPS"]},
        "fp64": None if fp64 is None else {
            "value": n / (fp64["ms"] / 1e3), "ms_per_step": fp64["ms"],
            "apply_only": n / (fp64["apply_ms"] / 1e3), "apply_ms": fp64["apply_ms"],
            "accuracy": fp64["acc"],
            "step_breakdown_ms_serialised": {STEP_NAMES[i]: float(fp64["kt"][i]) for i in range(9)}},
        "step_breakdown_ms_serialised": {STEP_NAMES[i]: float(kt[i]) for i in range(9)},
        "plan_ms": float(mixed["ms"] - mixed["apply_ms"]),
        "work": mixed["work"],
    }
    return out


def rooflines(W, r):
    """Rooflines of the M2L (FP64 translations, exact algorithmic flop count)
    and of the near field (flops per pair from an instruction-count capture
    under profiles/, used only while it matches the current sources), from the
    serialised per-step kernel times of the MIXED apply. The dominant one
    (longer time) comes first."""
    mixed = r["mixed"]
    kt, work = mixed["kt"], mixed["work"]
    out = []
    m2l = {"kernel": "M2L" + (" (k_tr3h, modes M2L)" if W["DIM"] == 3 and W["KERNEL"] else ""),
           "bound": "alu", "unit": "GFLOP/s", "ms": float(kt[3]), "peak": FP64_PEAK_GFLOPS,
           "peak_source": "FP64 FMA units x max SM clock (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz); "
                          "MEASURED_PEAKS.json has no FP64 figure",
           "flops_per_apply": work["m2l_flops"], "traffic": None}
    m2l["achieved"] = work["m2l_flops"] / (kt[3] / 1e3) / 1e9 if kt[3] > 0 else None
    m2l["frac"] = m2l["achieved"] / FP64_PEAK_GFLOPS if m2l["achieved"] else None
    if W["DIM"] == 3 and W["KERNEL"]:
        prof = profile_figures("m2l_traffic_helm3d_k10_n1e6.txt", TR3H_SOURCES)
        if prof and "dram_bytes_per_apply" in prof:
            m2l["traffic"] = int(float(prof["dram_bytes_per_apply"]))
            m2l["traffic_source"] = prof["_path"]
    out.append(m2l)
    name = "p2p_flops_%s.txt" % ("helm3d_k10_mixed" if W["DIM"] == 3 and W["KERNEL"] else
                                 "lap3d_mixed" if W["DIM"] == 3 else "helm2d_k20_mixed")
    prof = profile_figures(name, P2P_SOURCES)
    p2p = {"kernel": "P2P (k_p2p32, List 1)", "bound": "alu", "unit": "GFLOP/s", "ms": float(kt[6]),
           "pairs_per_apply": work["p2p_pairs"], "traffic": None}
    if prof:
        f32 = float(prof["fp32_flops_per_pair"])
        f64 = float(prof.get("fp64_flops_per_pair", 0.0))
        p2p.update({"flops_per_pair_fp32": f32, "flops_per_pair_fp64": f64, "counts_source": prof["_path"],
                    "peak": FP32_PEAK_GFLOPS,
                    "peak_source": "FP32 FMA units x max SM clock (152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz)"})
        ach = work["p2p_pairs"] * f32 / (kt[6] / 1e3) / 1e9 if kt[6] > 0 else None
        p2p["achieved"] = ach
        p2p["frac"] = ach / FP32_PEAK_GFLOPS if ach else None
        p2p["fp64_frac"] = (work["p2p_pairs"] * f64 / (kt[6] / 1e3) / 1e9 / FP64_PEAK_GFLOPS
                            if kt[6] > 0 and f64 else None)
        if "dram_bytes_per_launch" in prof and "points_per_launch" in prof:
            # captured on a smaller case with the same leaf geometry: the near
            # field reads each source leaf once per neighbouring target leaf, so
            # its DRAM traffic grows with the number of points
            p2p["traffic"] = int(float(prof["dram_bytes_per_launch"]) * r["g"].n / float(prof["points_per_launch"]))
            p2p["traffic_source"] = prof["_path"] + " (scaled by the point count)"
    else:
        p2p.update({"achieved": None, "frac": None, "peak": FP32_PEAK_GFLOPS,
                    "note": "no instruction-count summary matching the current near-field sources"})
    out.append(p2p)
    out.sort(key=lambda x: -x["ms"])
    return out


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    r = measure_workload(args, W, dev, ws, rank, local, args.steps, args.warmup)
    extras = {}
    if args.workload == "helm3d" and not args.no_extras and args.n == 0:
        for name in ("lap3d", "helm2d"):
            rx = measure_workload(args, WORKLOADS[name], dev, ws, rank, local, min(args.steps, 5),
                                  max(3, min(args.warmup, 3)), check_targets=200, e2e=False)
            sx = summarize(WORKLOADS[name], rx, ws)
            sx["roofline"] = rooflines(WORKLOADS[name], rx)
            extras[name] = sx
    if rank != 0:
        return
    s = summarize(W, r, ws)
    roofs = rooflines(W, r)
    mixed = r["mixed"]
    line = {
        "metric": W["METRIC"],
        "value": s["value"],
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": s["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": dict(s["config"], parallelism=f"replicas{ws}",
                       l2="flushed (256 MB write) before every timed step"),
        "apply_only": s["apply_only"],
        "accuracy": s["accuracy"],
        "fp64": s["fp64"],
        "step_breakdown_ms_serialised": s["step_breakdown_ms_serialised"],
        "plan_ms": s["plan_ms"],
        "work": s["work"],
        "roofline": roofs[0],
        "roofline_kernels": roofs,
        "e2e": r["e2e"],
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clk"],
        "clocks_fp64": r["fp64"]["clk"] if r["fp64"] is not None else None,
        "wall_s": mixed["wall"],
    }
    if extras:
        line["extras"] = extras
    if not args.no_cpu_baseline:
        cb = cpu_baseline(args, W, r)
        line["cpu_baseline"] = cb
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
    # the plans at the workload's eps (one digit of headroom, eps / 10, costs a
    # third of the throughput and leaves the complex64 near field's error on the
    # steepest surfaces where it is)
    PLAN_EPS = EPS
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
        # leaf sizes above 256 make the complex64 near field's error grow past
        # eps on the steepest surfaces, so the mixed candidates stop there
        cands = (128, 192, 256) if precision == cf.MIXED else (64, 96, 128, 192)
        plans, outs, leaves, streams = [], [], [], []
        for i, g in enumerate(geoms):
            s = torch.cuda.Stream(device=dev)
            # separation from each geometry's Lipschitz estimate; the top level
            # moved down where the rule's level needs an order above the
            # translation kernels' limit (low slopes over 40 x 40 at k = 15)
            leaf, _ = tune_leaf_size(3, kernel, KAPPA, PLAN_EPS, pts_re[i], pts_im[i], precision=precision,
                                     candidates=cands, reps=2, stream=s, sep=SEP, top_level=cf.TOP_FIT)
            p = cf.plan(3, kernel, KAPPA, PLAN_EPS, pts_re[i], pts_im[i], leaf_size=leaf, sep=SEP,
                        precision=precision, stream=s, top_level=cf.TOP_FIT)
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
            # against the library's FP64 direct sum at sampled targets
            errs = []
            rng = np.random.default_rng(1)
            for i, g in enumerate(geoms):
                nt = 200 if i == 0 else 100
                idx = torch.from_numpy(np.sort(rng.choice(g.n, nt, replace=False))).to(dev)
                ref = cf.direct(3, kernel, KAPPA, pts_re[i], pts_im[i], pts_re[i][idx].contiguous(),
                                pts_im[i][idx].contiguous(), dens[i], precision=cf.FP64).cpu().numpy()
                for r in ((0, nrhs[i] - 1) if nrhs[i] > 1 else (0,)):
                    u = outs[i][r][idx].cpu().numpy()
                    errs.append(float(np.linalg.norm(u - ref[r]) / np.linalg.norm(ref[r])))
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
        plans[0].set_timing(2)
        plans[0].apply(dens[0], out=outs[0])
        kt = np.array(plans[0].timings())
        plans[0].set_timing(False)
        work = work_model(plans[0], WORKLOADS["batch3d"])
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

    check = rank == 0
    mixed = measure(cf.MIXED, check)
    fp64 = measure(cf.FP64, check) if args.precision == "both" else None
    if rank != 0:
        return
    kt = mixed["kt"]
    dom = int(np.argmax(kt))
    work = dict(mixed["work"])
    # right-hand-side work times nrhs; the per-pair operators once
    work["m2l_flops"] = (work["m2l_flops"] - work["m2l_flops_shared"]) * nrhs[0] + work["m2l_flops_shared"]
    work["p2p_pairs"] *= nrhs[0]
    roof = dominant_roofline("M2L", kt[3], work, FP64_PEAK_GFLOPS)
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
                   "nrhs": nrhs, "point_evaluations_per_step": evals, "kappa": KAPPA, "eps": EPS, "plan_eps": PLAN_EPS, "sep": SEP,
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
        line["cpu_baseline"] = cpu_baseline(args, WORKLOADS["batch3d"])
    print(json.dumps(line), flush=True)


def _serve_summary(runs):
    """points/s over a pass's streams and the last stream's latency quantiles."""
    return {"value": sum(r["evaluations"] for r in runs) / sum(r["wall_s"] for r in runs),
            "p50_s": runs[-1]["p50_s"], "p99_s": runs[-1]["p99_s"]}


def run_serve(args):
    """--workload serve: the serving loop on a Poisson stream of apply requests
    (dims 2 and 3, Laplace or Helmholtz with k ~ U[1, 50], N log-uniform in
    [1e3, nmax], eps in {1e-3, 1e-6, 1e-9}, 1-20 matvecs each on a resident
    plan, admission by free HBM). The arrival rate loads the GPU to about 80%:
    0.8 over the mean service time of a calibration sample of the same
    distribution served one at a time (unless --rate is given). The stream is
    served with precision AUTO (mixed where eps >= 1e-5) and, for comparison,
    the same stream in plain FP64. value = point evaluations per second of wall
    time (AUTO pass); p50/p99 latency = arrival to last result on the host."""
    import torch

    from paper_2509_05458_gb300 import AUTO, FP64
    from paper_2509_05458_gb300.serving import Server, make_stream, summarize

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    dims = (2, 3)
    srv = Server(slots=args.slots, device=local)
    warm = make_stream(max(4, args.warmup), seed=99 + rank, rate_hz=100.0, nmin=1000, nmax=20000, dims=dims)
    srv.run(warm, realtime=False)
    rate = args.rate
    calib = None
    if rate <= 0:
        sample = make_stream(24, seed=1234 + rank, rate_hz=1.0, nmin=1000, nmax=args.nmax, dims=dims, lazy=True)
        one = Server(slots=1, device=local)
        t0 = time.perf_counter()
        one.run(sample, realtime=False, keep_outputs=False)
        torch.cuda.synchronize()
        svc = (time.perf_counter() - t0) / len(sample)
        rate = 0.8 / svc
        calib = {"sample_requests": len(sample), "mean_service_s": svc, "rate_hz": rate}
        # progress on stderr (a stream at 80% load runs about 1.25 x its total
        # service time, so a cut-off run still leaves these figures)
        print(json.dumps({"serve_calibration": calib}), file=sys.stderr, flush=True)
    passes = {}
    clocks = ClockSampler(local)
    _barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    # the full stream in AUTO; the comparison with plain FP64 on its first
    # fp64_requests requests (the same requests and arrival times), with AUTO
    # re-run on that prefix, so both throughputs cover the same work
    nfp = args.requests if args.fp64_requests <= 0 else min(args.fp64_requests, args.requests)
    legs = [("auto", AUTO, args.requests)]
    if args.precision != "mixed":
        if nfp < args.requests:
            legs.append(("auto_prefix", AUTO, nfp))
        legs.append(("fp64", FP64, nfp))
    for name, prec, nreq in legs:
        runs = []
        for k in range(args.steps):
            reqs = make_stream(args.requests, seed=7 + 1000 * k + rank, rate_hz=rate, nmin=1000, nmax=args.nmax,
                               dims=dims, lazy=True, precision=prec)[:nreq]
            t0 = time.perf_counter()
            res = srv.run(reqs, keep_outputs=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            st = summarize(res, wall)
            st["evaluations"] = sum(r.points for r in res if r.error is None)
            st["evaluations_requested"] = sum(r.n * r.nrhs for r in reqs)
            runs.append(st)
            print(json.dumps({"serve_pass": name, "requests": nreq, "wall_s": wall,
                              "points_per_s": st["evaluations"] / wall if wall > 0 else None,
                              "p50_s": st.get("p50_s"), "p99_s": st.get("p99_s")}), file=sys.stderr, flush=True)
        passes[name] = runs
    _barrier(ws)
    clk = clocks.stop()
    main = passes["auto"]
    wall = _max_over_ranks(sum(r["wall_s"] for r in main), ws, dev)
    if rank != 0:
        return
    evals = sum(r["evaluations"] for r in main)
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
                               f"{rate:.3g} Hz, dim in {{2,3}}, Laplace or Helmholtz (k ~ U[1,50] in both "
                               f"dimensions), N log-uniform in [1e3, {args.nmax:.0e}], eps in {{1e-3,1e-6,1e-9}}, "
                               "1-20 matvecs per request on a resident plan, admission by free HBM, precision "
                               "AUTO (mixed where eps >= 1e-5)",
                   "slots": args.slots, "requests_per_step": args.requests, "rate_hz": rate,
                   "rate_calibration": calib, "nmax": args.nmax, "parallelism": f"replicas{ws}",
                   "timing": "host wall clock per stream (latency is arrival to result on the host)"},
        "p50_s": main[-1]["p50_s"], "p99_s": main[-1]["p99_s"], "mean_s": main[-1]["mean_s"],
        "errors": sum(r["errors"] for r in main),
        "error_kinds": main[-1]["error_kinds"],
        "streams": main,
        "fp64_same_stream": ({"requests": nfp,
                              "value": sum(r["evaluations"] for r in passes["fp64"]) /
                              sum(r["wall_s"] for r in passes["fp64"]),
                              "p50_s": passes["fp64"][-1]["p50_s"], "p99_s": passes["fp64"][-1]["p99_s"],
                              "errors": sum(r["errors"] for r in passes["fp64"]), "streams": passes["fp64"],
                              "auto_on_same_requests": _serve_summary(passes["auto_prefix" if "auto_prefix" in passes
                                                                          else "auto"])}
                             if "fp64" in passes else None),
        "e2e": {"value": evals * ws / wall, "unit": "points/s",
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "the stream itself is end to end: host points and densities in, host results out"},
        "roofline": None,
        "gpu_launches": None,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_wobble(args):
    """--workload wobble: the paper's own test interfaces (Sec. 7.1, Eqs.
    wobble_2D_cplx and complex_wobble), single layer, N = 1e6 each: 2D and 3D
    Laplace and Helmholtz (kappa = 2 pi), FP64 at eps = 1e-6 and 1e-12 (the
    paper's two accuracies) and MIXED at 1e-6; one plan+apply pass per step,
    accuracy against the library's FP64 direct sum on 200 sampled targets.
    value = all cases' points over their summed plan+apply times."""
    import numpy as np
    import torch

    import paper_2509_05458_gb300 as cf
    from cfmm_inputs import wobble2d, wobble3d, densities

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    n = args.n or 1_000_000
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cases = []
    clocks = ClockSampler(local)
    clocks.start()
    tot_pts, tot_ms = 0, 0.0
    for dim in (2, 3):
        g = wobble2d(n, seed=0) if dim == 2 else wobble3d(n)
        re, im = torch.from_numpy(g.re).to(dev), torch.from_numpy(g.im).to(dev)
        dens = torch.from_numpy(densities(g.n, seed=1)).to(dev)
        out = torch.empty((1, g.n), dtype=torch.complex128, device=dev)
        idx = torch.from_numpy(np.sort(np.random.default_rng(1).choice(g.n, 200, replace=False))).to(dev)
        for ker in (cf.LAPLACE, cf.HELMHOLTZ):
            kap = 2 * np.pi if ker == cf.HELMHOLTZ else 0.0
            ref = cf.direct(dim, ker | cf.SLP, kap, re, im, re[idx].contiguous(), im[idx].contiguous(), dens,
                            stream=stream).cpu().numpy()[0]
            for eps, prec in ((1e-6, cf.FP64), (1e-6, cf.MIXED), (1e-12, cf.FP64)):
                sep = 2 if dim == 3 else 1
                case = {"dim": dim, "kernel": "helmholtz" if ker else "laplace", "kappa": kap, "eps": eps,
                        "precision": "MIXED" if prec == cf.MIXED else "FP64", "sep": sep, "n": g.n}

                def step():
                    p = cf.plan(dim, ker | cf.SLP, kap, eps, re, im, leaf_size=64, sep=sep, stream=stream,
                                precision=prec)
                    p.apply(dens, out=out)
                    p.destroy()
                try:
                    for _ in range(max(1, args.warmup)):
                        step()
                    ms = []
                    for _ in range(max(1, min(args.steps, 5))):
                        flush.zero_()
                        ev0.record(stream)
                        step()
                        ev1.record(stream)
                        ev1.synchronize()
                        ms.append(ev0.elapsed_time(ev1))
                except cf.CfmmError as e:
                    case["unsupported"] = str(e)
                    cases.append(case)
                    continue
                m = statistics.median(ms)
                u = out[0][idx].cpu().numpy()
                case.update({"ms": m, "points_per_s": g.n / (m / 1e3),
                             "rel_l2_vs_fp64_direct_200_targets": float(np.linalg.norm(u - ref) / np.linalg.norm(ref))})
                tot_pts += g.n
                tot_ms += m
                cases.append(case)
    clk = clocks.stop()
    if rank != 0:
        return
    line = {"metric": "complex-FMM pts/s on the paper's wobbly interfaces (Sec. 7.1), single layer",
            "value": tot_pts * ws / (tot_ms / 1e3), "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 / f32+f64", "data": "synthetic",
            "config": {"workload": "wobble_2D_cplx (t uniform in [-20,20]) and complex_wobble ((t1,t2) Halton in "
                                   "[-25,25]^2), N = %d each, SLP, leaf 64, sep 1 (2D) / 2 (3D)" % n,
                       "parallelism": f"replicas{ws}", "l2": "flushed (256 MB write) before every timed step"},
            "cases": cases, "clocks": clk, "roofline": None, "gpu_launches": None,
            "e2e": None}
    print(json.dumps(line), flush=True)


def work_model(p, W=None):
    """Algorithmic work of one apply: List-2 pairs and M2L flops at each pair's
    level (2D: 8 flops per complex multiply-add, (2P+1)^2 per pair; 3D: the
    point-and-shoot counts below), List-1 pairs."""
    import numpy as np
    W = W or WORKLOADS["helm3d"]
    inf = p.info()
    t = p.export_tree()
    P = p.orders()
    off, _ = p.export_list(2)
    cnt = np.diff(off)
    m2l_flops = 0
    m2l_shared = 0          # per-pair work done once for every right-hand side
    pairs_per_level = {}
    for l in range(inf["nlevels"]):
        npairs = int(cnt[t["level"] == l].sum())
        if npairs:
            pairs_per_level[int(l)] = npairs
            if W["DIM"] == 2:
                m2l_flops += npairs * 8 * (2 * int(P[l]) + 1) ** 2
            else:
                m2l_flops += npairs * (m2l_flops_pair_3d(int(P[l])) if W["KERNEL"]
                                       else m2l_flops_pair_lap3d(int(P[l])))
                if W["KERNEL"] and int(P[l]) <= 40:
                    # the coaxial operators of these pairs are built once (k_tr3h_tri)
                    m2l_shared += npairs * m2l_flops_coax_3d(int(P[l]))
    return {"p2p_pairs": int(inf["p2p_pairs"]), "m2l_pairs": int(inf["m2l_pairs"]),
            "m2l_pairs_per_level": pairs_per_level, "orders": [int(x) for x in P],
            "m2l_flops": int(m2l_flops), "m2l_flops_shared": int(m2l_shared)}


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


def m2l_flops_coax_3d(P):
    """The coaxial-recurrence part of m2l_flops_pair_3d (the per-pair operators,
    independent of the right-hand side)."""
    return 12 * P * (P + 1) * (2 * P + 1) // 6


def m2l_flops_pair_lap3d(P):
    """FP64 flops of one 3D Laplace point-and-shoot M2L at order P: the four
    fixed-rotation products (as for Helmholtz) and the z-axis solid-harmonic
    shift (sum_m (1 + [m > 0]) (P - m + 1)^2 complex multiply-adds, 8 flops)."""
    rot = 4 * 4 * P * (P + 1) * (P + 2) // 3
    app = 8 * sum((1 + (m > 0)) * (P - m + 1) ** 2 for m in range(P + 1))
    return rot + app


def dominant_roofline(name, ms, work, fp64_peak_gflops):
    """Roofline of the M2L of an apply, FP64-ALU bound (work["m2l_flops"])."""
    base = {"bound": "alu", "peak": fp64_peak_gflops, "unit": "GFLOP/s", "traffic": None, "kernel": name,
            "ms": float(ms),
            "peak_source": "FP64 FMA units x max SM clock (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz)"}
    flops = work["m2l_flops"]
    if not flops or ms <= 0:
        return dict(base, achieved=None, frac=None)
    ach = flops / (ms / 1e3) / 1e9
    return dict(base, achieved=ach, frac=ach / fp64_peak_gflops)


# ---- the CPU baseline: the oracle, as it stands, on the host cores ----------

def _oracle_direct_chunk(job):
    """One worker's share of the oracle's direct sum (runs in a spawned process)."""
    sys.path.insert(0, ROOT)
    from oracle.direct import direct
    dim, ker, kap, pts, trg, sigma, tau, nrm = job
    t = time.perf_counter()
    u = direct(dim, ker, kap, pts, trg, sigma=sigma, tau=tau, nrm=nrm)
    return u, time.perf_counter() - t


def oracle_direct_sample(W, g, dens_np, idx, workers):
    """The oracle's direct sum at targets idx against all points, split over
    `workers` spawned processes (each single-threaded). Returns (u, wall s)."""
    import concurrent.futures as fut
    import multiprocessing as mp
    import numpy as np
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    pts = g.re + 1j * g.im
    nrm = (g.nrm_re + 1j * g.nrm_im) if W["DLP"] else None
    sigma = dens_np[0, 0]
    tau = dens_np[0, 1] if W["DLP"] else None
    parts = [p for p in np.array_split(idx, workers) if len(p)]
    jobs = [(W["DIM"], W["KERNEL"], W["KAPPA"], pts, pts[p], sigma, tau, nrm) for p in parts]
    t0 = time.perf_counter()
    with fut.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_direct_chunk, jobs))
    wall = time.perf_counter() - t0
    return np.concatenate([u for u, _ in res]), wall


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(args, W, r=None):
    """The oracle's direct sum (numpy/scipy, as it stands) on a bounded sample
    of the workload: `--cpu-targets` seeded targets against all N sources,
    split over every host core; points/s = targets evaluated per second. When
    the GPU result r is given, its error on the same targets is reported."""
    import numpy as np
    from cfmm_inputs import densities
    g = r["g"] if r else _geometry(W)
    dens_np = r["dens_np"] if r else densities(g.n, seed=1, nrhs=1, ncomp=2 if W["DLP"] else 1)
    nt = min(args.cpu_targets, g.n)
    idx = np.sort(np.random.default_rng(7).choice(g.n, nt, replace=False))
    cores = cpu_cores()
    u0, wall = oracle_direct_sample(W, g, dens_np, idx, cores)
    out = {"value": nt / wall, "unit": "points/s", "cores": cores, "kind": "oracle",
           "sample": f"oracle direct sum (numpy/scipy, FP64), {nt} seeded targets against all {g.n} sources, "
                     f"split over {cores} processes: {wall:.1f} s wall; points/s = targets evaluated per second"}
    if r:
        # the GPU passes' error against the oracle on the same targets
        err = lambda u: float(np.linalg.norm(u[idx] - u0) / np.linalg.norm(u0))
        out["gpu_rel_l2_vs_oracle_on_sample"] = {
            "mixed": err(r["mixed"]["u"]), "fp64": err(r["fp64"]["u"]) if r["fp64"] is not None else None}
    return out


def run_reference(args):
    """--impl reference: the oracle, as it stands, on the host cores (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload if args.workload in ("helm3d", "lap3d", "helm2d") else "helm3d"]
    vals = []
    res = None
    for i in range(args.warmup + args.steps):
        res = cpu_baseline(args, W)
        if i >= args.warmup:
            vals.append(res["value"])
    val = statistics.mean(vals) if vals else None
    line = {"metric": W["METRIC"], "value": val, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": W["WORKLOAD"], "n": W["N_POINTS"], "kappa": W["KAPPA"], "eps": W["EPS"],
                       "leaf_size": W["LEAF"], "sep": W["SEP"], "layers": "SLP+DLP" if W["DLP"] else "SLP",
                       "precision": "FP64", "parallelism": "cpu"},
            "cpu_baseline": {"value": val, "unit": "points/s", "cores": res["cores"] if res else None,
                             "kind": "oracle", "sample": res["sample"] if res else None},
            "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-targets", type=int, default=1000,
                    help="targets of the CPU baseline's sample (against all sources)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 3D Laplace and 2D lines of the default run")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"],
                    help="which passes to run (the headline needs both)")
    ap.add_argument("--workload", default="helm3d",
                    choices=["helm3d", "lap3d", "helm2d", "batch3d", "serve", "wobble"],
                    help="helm3d: the 3D Helmholtz surface headline (with the 3D Laplace and 2D lines); lap3d / "
                         "helm2d: those alone; batch3d: the batched 3D Helmholtz line; serve: the serving loop")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests per stream")
    ap.add_argument("--fp64-requests", type=int, default=0,
                    help="serve: the FP64 comparison on the first N requests of the stream (0 = all)")
    ap.add_argument("--rate", type=float, default=0.0, help="serve: Poisson arrival rate (Hz); 0 = calibrated")
    ap.add_argument("--nmax", type=int, default=1_000_000, help="serve: largest request size")
    ap.add_argument("--slots", type=int, default=4, help="serve: requests in flight")
    ap.add_argument("--n", type=int, default=0,
                    help="override the point count (small cases for profiler captures; not a bench line)")
    ap.add_argument("--sep", type=int, default=0, help="override the separation k (parameter sweeps)")
    ap.add_argument("--leaf", type=int, default=0, help="override the leaf size of both passes (parameter sweeps)")
    args = ap.parse_args()
    if args.workload in WORKLOADS:
        W = WORKLOADS[args.workload]
        if args.n > 0:
            W["N_POINTS"] = args.n
        if args.sep > 0:
            W["SEP"] = args.sep
        if args.leaf > 0:
            W["LEAF"] = W["LEAF_FP64"] = args.leaf
        globals().update(W)
    if args.impl == "reference":
        args.warmup = max(0, min(args.warmup, 1))
        args.steps = max(1, min(args.steps, 2))
        run_reference(args)
    elif args.workload == "batch3d":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "wobble":
        run_wobble(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
