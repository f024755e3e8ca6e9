"""Helpers for the GPU parity tests (CUDA path through the C ABI vs oracle)."""
import numpy as np


def to_dev(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def gpu_plan(cf, g, kernel, kappa, eps, dev, leaf, sep=1, dlp=False, top_level=0, precision=0):
    nre = to_dev(g.nrm_re, dev) if dlp else None
    nim = to_dev(g.nrm_im, dev) if dlp else None
    return cf.plan(g.dim, kernel | (cf.SLP | cf.DLP if dlp else cf.SLP), kappa, eps,
                   to_dev(g.re, dev), to_dev(g.im, dev), nre, nim, leaf_size=leaf, sep=sep,
                   top_level=top_level, precision=precision)


def compare_tree(T, tr_gpu, lists_gpu):
    """Bit-exact comparison of the oracle tree T with an exported GPU tree."""
    assert np.array_equal(tr_gpu["perm"], T.perm.astype(np.int64))
    assert np.array_equal(tr_gpu["keys"], T.keys)
    assert np.array_equal(tr_gpu["level"], T.box_level.astype(np.int32))
    assert np.array_equal(tr_gpu["prefix"], T.box_prefix.astype(np.uint64))
    assert np.array_equal(tr_gpu["start"], T.box_start.astype(np.int32))
    assert np.array_equal(tr_gpu["end"], T.box_end.astype(np.int32))
    assert np.array_equal(tr_gpu["leaf"], T.box_leaf)
    assert np.array_equal(tr_gpu["parent"], T.box_parent.astype(np.int32))
    for w in range(4):
        off, ent = lists_gpu[w]
        ref = T.lists[f"list{w + 1}"]
        assert off[-1] == sum(len(x) for x in ref), f"list{w + 1} length"
        for b in range(T.nboxes):
            got = list(ent[off[b]:off[b + 1]])
            assert got == ref[b], (w + 1, b, got, ref[b])


def _direct_chunk(args):
    from oracle.direct import direct
    dim, ker, kap, pts, trg, sigma, tau, nrm, green = args
    return direct(dim, ker, kap, pts, trg, sigma=sigma, tau=tau, nrm=nrm, green_scale=green)


def direct_sampled(dim, ker, kap, pts, idx, sigma=None, tau=None, nrm=None, green=False, workers=None):
    """The oracle's direct sum at the targets pts[idx] against all points, split
    over a process pool started with `spawn` (safe after CUDA is initialised)."""
    import concurrent.futures as fut
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    parts = np.array_split(np.asarray(idx), workers)
    jobs = [(dim, ker, kap, pts, pts[p], sigma, tau, nrm, green) for p in parts if len(p)]
    with fut.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_direct_chunk, jobs))
    return np.concatenate(res, axis=-1)
