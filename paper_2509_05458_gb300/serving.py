"""Continuous-batching server for complex-coordinate FMM apply requests.

A request carries one geometry (points, optional normals), a kernel, a
wavenumber, an accuracy and one or more right-hand sides to apply in turn (the
matvecs of an iterative solve on a resident plan). The server keeps `slots`
requests in flight at once, each on its own CUDA stream and host worker
thread (the C library releases the GIL for every call), and admits a waiting
request as soon as a slot is free and its estimated device-memory footprint
fits the budget (the free HBM reported by the driver minus a reserve, or a
caller-given budget). Requests that arrive while others run are admitted as
slots and memory free up, so their work overlaps on the device.

Every kernel of the library is deterministic per plan (no atomics across
targets, fixed reduction orders) and plans share no device state, so a result
does not depend on what else is in flight: `tests/test_gpu_serving.py` checks
that each result is bitwise the same alone and in the mix.

Latency of a request = time from its arrival to its last result copied back
to the host; the run reports p50/p99 latency and points/s. Requests the
library cannot serve (for instance a 3D Helmholtz geometry whose top-level
expansion order exceeds the translation kernels' limit, CFMM_EUNSUPPORTED)
fail alone and are counted by error kind.

Large streams are generated lazily: a request may carry only the parameters
of its synthetic geometry and densities, and a producer thread materialises
the next few requests ahead of their arrival (so the host-side generation is
not part of a request's latency unless the producer falls behind).
"""
from __future__ import annotations

import concurrent.futures as cfut
import dataclasses
import statistics
import threading
import time
from typing import List, Optional

import numpy as np

from . import FP64, MIXED, AUTO, SLP, DLP, plan as make_plan

__all__ = ["Request", "Result", "Server", "estimate_bytes"]


@dataclasses.dataclass
class Request:
    rid: int
    dim: int
    kernel: int                     # LAPLACE/HELMHOLTZ or-ed with SLP/DLP
    kappa: float
    eps: float
    pts_re: Optional[np.ndarray]    # [n, dim] float64 (host); None until materialised
    pts_im: Optional[np.ndarray]
    rhs: Optional[List[np.ndarray]]  # each [ncomp, n] complex128 (host)
    nrm_re: Optional[np.ndarray] = None
    nrm_im: Optional[np.ndarray] = None
    arrival: float = 0.0            # seconds from the start of the run
    leaf_size: int = 64
    precision: int = AUTO
    sep: int = 1                    # well-separatedness k (Sec. 6.2)
    spec: Optional[dict] = None     # parameters of a lazily generated request

    @property
    def n(self):
        return self.pts_re.shape[0] if self.pts_re is not None else int(self.spec["n"])

    @property
    def nrhs(self):
        return len(self.rhs) if self.rhs is not None else int(self.spec["nmv"])

    def materialize(self):
        """Generate the geometry and densities of a lazily specified request."""
        if self.pts_re is not None:
            return self
        from cfmm_inputs import curve2d, surface3d, densities
        sp = self.spec
        if self.dim == 2:
            g = curve2d(sp["n"], seed=sp["gseed"], t_half=sp["t_half"], height=sp["height"])
        else:
            g = surface3d(sp["n"], seed=sp["gseed"], half=20.0, random_shape=True)
        dens = densities(sp["n"], seed=sp["gseed"] + 1, nrhs=sp["nmv"], ncomp=1)
        self.pts_re, self.pts_im = g.re, g.im
        self.rhs = [dens[i] for i in range(sp["nmv"])]
        return self

    def release(self):
        """Drop the host data of a lazily specified request once it is served."""
        if self.spec is not None:
            self.pts_re = self.pts_im = self.rhs = None


@dataclasses.dataclass
class Result:
    rid: int
    outputs: List[np.ndarray]       # each [n] complex128 (empty when outputs are not kept)
    arrival: float
    admitted: float
    done: float
    error: Optional[str] = None
    points: int = 0                 # point evaluations delivered (n per right-hand side)
    checksums: Optional[List[complex]] = None   # sum of each output (when outputs are not kept)

    @property
    def latency(self):
        return self.done - self.arrival


def estimate_bytes(req: Request) -> int:
    """Conservative device-memory footprint of a request's plan and workspaces."""
    n, dim = req.n, req.dim
    per_point = 8 * 4 * dim + 12 + 16 * 4          # points/normals, keys/perm, densities, results
    helm = (req.kernel & 0xF) == 1
    per_point += 2500 if helm else 400               # expansions and translation tables
    extra = 0
    if helm and dim == 3:
        # M2L coaxial operators built ahead for a level (about 4.4 kB per point
        # at leaf 256, growing as the leaves shrink), capped by the library's
        # per-launch operator budget
        extra = min(6 << 30, int(n * 4500 * 256 / max(req.leaf_size, 1)))
    return int(n * per_point + extra + (96 << 20))   # + plan-construction scratch


class Server:
    """Runs requests with up to `slots` in flight on separate streams."""

    def __init__(self, slots=4, budget_bytes=None, reserve_bytes=2 << 30, device=0):
        import torch
        self.torch = torch
        self.dev = torch.device(f"cuda:{device}")
        self.slots = slots
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            budget_bytes = max(0, free - reserve_bytes)
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.cv = threading.Condition()
        self.active = 0

    def _run_one(self, req: Request, stream, t0: float, admitted: float, keep=True) -> Result:
        torch = self.torch
        outs, sums = [], []
        points = 0
        try:
            req.materialize()
            with torch.cuda.stream(stream):
                re = torch.from_numpy(np.ascontiguousarray(req.pts_re)).to(self.dev, non_blocking=True)
                im = torch.from_numpy(np.ascontiguousarray(req.pts_im)).to(self.dev, non_blocking=True)
                nre = nim = None
                if req.kernel & DLP:
                    nre = torch.from_numpy(np.ascontiguousarray(req.nrm_re)).to(self.dev, non_blocking=True)
                    nim = torch.from_numpy(np.ascontiguousarray(req.nrm_im)).to(self.dev, non_blocking=True)
                p = make_plan(req.dim, req.kernel, req.kappa, req.eps, re, im, nre, nim,
                              leaf_size=req.leaf_size, sep=req.sep, precision=req.precision, stream=stream)
                out = torch.empty((1, req.n), dtype=torch.complex128, device=self.dev)
                for r in req.rhs:
                    d = torch.from_numpy(np.ascontiguousarray(r)[None]).to(self.dev, non_blocking=True)
                    p.apply(d, out=out)
                    h = out[0].cpu().numpy()   # synchronises this stream only
                    if keep:
                        outs.append(h)
                    else:
                        sums.append(complex(h.sum()))
                    points += req.n
                p.destroy()
            err = None
        except Exception as e:   # reported per request; the server keeps going
            err = f"{type(e).__name__}: {e}"
        finally:
            if not keep:
                req.release()
        return Result(req.rid, outs, req.arrival, admitted, time.perf_counter() - t0, err, points,
                      None if keep else sums)

    def run(self, requests: List[Request], realtime=True, keep_outputs=True, prefetch=8) -> List[Result]:
        """Serve `requests`. With realtime=True a request is not visible before its
        arrival time (seconds after the call starts); admission is FIFO. Lazily
        specified requests are materialised by a producer thread up to
        `prefetch` requests ahead of admission."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        results: List[Optional[Result]] = [None] * len(reqs)
        t0 = time.perf_counter()
        streams = [torch.cuda.Stream(device=self.dev) for _ in range(self.slots)]
        free_streams = list(range(self.slots))
        ready = threading.Semaphore(0)
        window = threading.Semaphore(max(1, prefetch))
        stop = threading.Event()

        def producer():
            for r in reqs:
                if not window.acquire(timeout=None) or stop.is_set():
                    return
                r.materialize()
                ready.release()

        prod = threading.Thread(target=producer, daemon=True)
        prod.start()

        def worker(i, req, sidx, need, admitted):
            try:
                results[i] = self._run_one(req, streams[sidx], t0, admitted, keep_outputs)
            finally:
                with self.cv:
                    self.in_use -= need
                    self.active -= 1
                    free_streams.append(sidx)
                    self.cv.notify_all()

        futs = []
        waiting = []
        k = 0
        try:
            # one long-lived host thread per slot (their plan-construction scratch is reused)
            with cfut.ThreadPoolExecutor(max_workers=self.slots) as pool:
                while k < len(reqs) or waiting:
                    now = time.perf_counter() - t0
                    while k < len(reqs) and (not realtime or reqs[k].arrival <= now):
                        if not ready.acquire(blocking=False):
                            break                    # its data is still being generated
                        waiting.append((k, reqs[k]))
                        k += 1
                    with self.cv:
                        progressed = False
                        while waiting and free_streams:
                            i, req = waiting[0]
                            need = min(estimate_bytes(req), self.budget)
                            if self.in_use + need > self.budget and self.active > 0:
                                break                   # the head of the queue waits for memory
                            waiting.pop(0)
                            window.release()
                            self.in_use += need
                            self.active += 1
                            sidx = free_streams.pop(0)
                            futs.append(pool.submit(worker, i, req, sidx, need, time.perf_counter() - t0))
                            progressed = True
                        if not progressed:
                            nxt = reqs[k].arrival - now if (realtime and k < len(reqs)) else 0.005
                            self.cv.wait(timeout=max(1e-4, min(0.005 if k < len(reqs) else 0.05, nxt)))
                for f in futs:
                    f.result()
        finally:
            stop.set()
            window.release()
        torch.cuda.synchronize(self.dev)
        return results


def summarize(results: List[Result], wall_s: float):
    lat = sorted(r.latency for r in results if r.error is None)
    pts = sum(r.points if r.points else len(r.outputs) * (r.outputs[0].shape[0] if r.outputs else 0)
              for r in results if r.error is None)

    def pct(p):
        if not lat:
            return None
        i = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[i]

    kinds = {}
    for r in results:
        if r.error:
            k = r.error[:80]
            kinds[k] = kinds.get(k, 0) + 1
    return {"requests": len(results), "errors": sum(1 for r in results if r.error), "error_kinds": kinds,
            "p50_s": pct(50), "p99_s": pct(99), "mean_s": statistics.mean(lat) if lat else None,
            "points_per_s": pts / wall_s if wall_s > 0 else None, "wall_s": wall_s}


def make_stream(nreq, seed=7, rate_hz=20.0, nmin=1_000, nmax=200_000, dims=(2,), max_matvec=20, lazy=False,
                precision=AUTO):
    """A Poisson stream of requests on the synthetic families: dim in `dims`,
    Laplace or Helmholtz (k ~ U[1, 50] in both dimensions), N log-uniform in
    [nmin, nmax], eps in {1e-3, 1e-6, 1e-9}, 1..max_matvec right-hand sides.
    lazy=True: the requests carry the parameters only (Request.materialize)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(nreq):
        t += rng.exponential(1.0 / rate_hz)
        dim = int(rng.choice(dims))
        helm = bool(rng.integers(0, 2))
        kappa = float(rng.uniform(1.0, 50.0)) if helm else 0.0
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        eps = float(rng.choice([1e-3, 1e-6, 1e-9]))
        nmv = int(rng.integers(1, max_matvec + 1))
        gseed = int(rng.integers(0, 2**31 - 1))
        t_half, height = 10.0 + 30.0 * rng.uniform(), float(rng.uniform(0.3, 1.0))
        spec = dict(n=n, nmv=nmv, gseed=gseed, t_half=t_half, height=height)
        r = Request(rid, dim, (1 if helm else 0) | SLP, kappa, eps, None, None, None, arrival=t,
                    sep=2 if dim == 3 else 1, precision=precision, spec=spec)
        if not lazy:
            r.materialize()
        out.append(r)
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="serve a Poisson stream of FMM apply requests")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--nmax", type=int, default=200_000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--dims", default="2", help="comma-separated dimensions, e.g. 2,3")
    args = ap.parse_args()
    dims = tuple(int(x) for x in args.dims.split(","))
    reqs = make_stream(args.requests, seed=args.seed, rate_hz=args.rate, nmax=args.nmax, dims=dims)
    srv = Server(slots=args.slots)
    t = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t
    print(json.dumps(dict(summarize(res, wall), rate_hz=args.rate, slots=args.slots)))


if __name__ == "__main__":
    main()
