"""Leaf-size autotuner.

The leaf size N_s (Sec. 6.1) trades near-field work (List 1 grows like N_s)
against expansion work (the number of boxes falls like 1/N_s). The best value
depends on the kernel, the precision mode (the mixed-precision near field is
much cheaper than the FP64 one, so it prefers larger leaves), the wavenumber
and the geometry. `tune_leaf_size` times the apply (the part repeated by an
iterative solver) of each candidate on the caller's geometry with CUDA events
and returns the fastest; results are memoised per
(dim, kernel, precision, log2 N, eps, kappa * root width) bucket.
"""
from __future__ import annotations

import math
import statistics

import numpy as np

from . import CfmmError, plan as make_plan

_CACHE = {}


def _bucket(dim, kernel, precision, n, eps, kappa, width, sep=1, top_level=0):
    return (dim, kernel & 0xF, precision, sep, top_level, int(round(math.log2(max(n, 1)))),
            int(round(math.log10(eps))), int(round(math.log2(1.0 + kappa * width))))


def tune_leaf_size(dim, kernel, kappa, eps, pts_re, pts_im, nrm_re=None, nrm_im=None,
                   precision=0, candidates=(32, 48, 64, 96, 128, 192), reps=3, stream=None,
                   use_cache=True, sep=1, top_level=0):
    """Returns (best_leaf_size, {leaf_size: median apply ms}). Inputs are CUDA tensors."""
    import torch
    n = int(pts_re.shape[0])
    width = float((pts_re.max(0).values - pts_re.min(0).values).max())
    key = _bucket(dim, kernel, precision, n, eps, kappa, width, sep, top_level)
    if use_cache and key in _CACHE:
        return _CACHE[key]
    dev = pts_re.device
    stream = stream or torch.cuda.current_stream(dev)
    dlp = nrm_re is not None
    ncomp = 2 if (dlp and (kernel & (1 << 4))) else 1
    dens = torch.ones((1, ncomp, n), dtype=torch.complex128, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for ls in candidates:
        try:
            p = make_plan(dim, kernel, kappa, eps, pts_re, pts_im, nrm_re, nrm_im, leaf_size=ls, sep=sep,
                          precision=precision, stream=stream, top_level=top_level)
        except CfmmError:
            continue          # a candidate the plan rejects (e.g. an order limit) is skipped
        out = p.apply(dens)
        ms = []
        for _ in range(reps):
            ev0.record(stream)
            p.apply(dens, out=out)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        times[ls] = statistics.median(ms)
        p.destroy()
    if not times:
        raise CfmmError(-7, "no leaf-size candidate gives a valid plan")
    best = min(times, key=times.get)
    _CACHE[key] = (best, times)
    return best, times
