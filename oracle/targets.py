"""Separate targets for the oracle FMMs (test infrastructure).

Sec. 2.3 Eq. evaluation_problem with targets x_i distinct from the sources
y_j. Reading (the same on both sides): the tree, complexified centres, lists
and orders are built on the sources and targets together (sources first, as
one point set of the paper's Sec. 6.1), the targets enter every expansion with
zero density (and zero normal), and the potential is read at the targets. A
source that coincides with a target is skipped for it, as in the direct sum
(oracle.direct), since the FMM skips pairs with x - y = 0.
"""
from __future__ import annotations

import numpy as np


def union_apply(apply_fn, src_re, src_im, trg_re, trg_im, sigma=None, tau=None, nrm_re=None, nrm_im=None):
    """apply_fn(re, im, sigma=, tau=, nrm_re=, nrm_im=) -> (u, T) is one of the
    oracle FMMs with its other arguments bound; sigma/tau are [m] or [nrhs, m].
    Returns (u at the targets, T)."""
    m = np.asarray(src_re).shape[0]
    n = np.asarray(trg_re).shape[0]
    re = np.concatenate([src_re, trg_re])
    im = np.concatenate([src_im, trg_im])

    def pad(v):
        if v is None:
            return None
        v = np.asarray(v, dtype=np.complex128)
        z = np.zeros(v.shape[:-1] + (n,), dtype=np.complex128)
        return np.concatenate([v, z], axis=-1)

    kw = dict(sigma=pad(sigma), tau=pad(tau))
    if nrm_re is not None:
        kw["nrm_re"] = np.concatenate([nrm_re, np.zeros_like(trg_re)])
        kw["nrm_im"] = np.concatenate([nrm_im, np.zeros_like(trg_re)])
    u, T = apply_fn(re, im, **kw)
    return u[..., m:], T
