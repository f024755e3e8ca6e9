"""Separate targets through the C ABI (cfmm_plan_targets): the potential of the
sources at targets with their own imaginary parts, against the oracle's
separate-target FMM (oracle/targets.py: tree on sources and targets together,
targets with zero density) to relative l2 1e-12, and against the oracle's
direct sum within eps; host and device inputs; mixed precision within 1e-6."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle import fmm2d, fmm3d, helm3d as H
from oracle.direct import direct, relerr_paper, relerr_l2
from oracle.targets import union_apply
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _geoms(dim):
    if dim == 2:
        s = curve2d(2000, seed=40, t_half=10.0, height=0.5)
        t = curve2d(700, seed=41, t_half=10.0, height=0.5, slope=0.45)
        t.re[:, 1] += 1.5
    else:
        s = surface3d(1200, seed=42, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
        t = surface3d(400, seed=43, half=4.0, amp=0.5, width=1.0, slope=0.25, rho0=1.0)
        t.re[:, 2] += 1.0
    return s, t


def _oracle(dim, ker, kap, eps, leaf, sep, s, t, dens):
    if dim == 2:
        f = lambda re, im, **kw: fmm2d.apply(re, im, ker, kap, eps, leaf, k=sep, **kw)
    elif ker == 0:
        f = lambda re, im, **kw: fmm3d.apply(re, im, eps, leaf, k=sep, **kw)
    else:
        f = lambda re, im, **kw: H.apply(re, im, kap, eps, leaf, k=sep, coaxial="exact", **kw)
    return union_apply(f, s.re, s.im, t.re, t.im, sigma=dens[0, 0], tau=dens[0, 1], nrm_re=s.nrm_re,
                       nrm_im=s.nrm_im)


@pytest.mark.parametrize("dim,ker,kap", [(2, 0, 0.0), (2, 1, 6.0), (3, 0, 0.0), (3, 1, 3.0)])
def test_separate_targets_vs_oracle(cuda, dim, ker, kap):
    import paper_2509_05458_gb300 as cf
    s, t = _geoms(dim)
    eps, leaf, sep = (1e-6, 24, 1) if dim == 2 else (1e-3, 24, 2)
    dens = densities(s.n, seed=44, nrhs=1, ncomp=2)
    flags = ker | cf.SLP | cf.DLP
    p = cf.plan_targets(dim, flags, kap, eps, to_dev(s.re, cuda), to_dev(s.im, cuda), to_dev(t.re, cuda),
                        to_dev(t.im, cuda), to_dev(s.nrm_re, cuda), to_dev(s.nrm_im, cuda), leaf_size=leaf, sep=sep)
    inf = p.info()
    assert inf["n_src"] == s.n and inf["n_trg"] == t.n and inf["n"] == s.n + t.n
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    assert u.shape == (t.n,)
    uo, T = _oracle(dim, ker, kap, eps, leaf, sep, s, t, dens)
    assert relerr_l2(u, uo) <= 1e-12
    u0 = direct(dim, ker, kap, s.re + 1j * s.im, t.re + 1j * t.im, sigma=dens[0, 0], tau=dens[0, 1],
                nrm=s.nrm_re + 1j * s.nrm_im)
    assert relerr_paper(u, u0, dens[0].reshape(-1)) <= eps
    # host arrays in and out give the same result
    ph = cf.plan_targets(dim, flags, kap, eps, s.re, s.im, t.re, t.im, s.nrm_re, s.nrm_im, leaf_size=leaf,
                         sep=sep)
    uh = ph.apply(np.ascontiguousarray(dens))[0]
    assert np.array_equal(uh, u)
    # mixed precision
    pm = cf.plan_targets(dim, flags, kap, eps, to_dev(s.re, cuda), to_dev(s.im, cuda), to_dev(t.re, cuda),
                         to_dev(t.im, cuda), to_dev(s.nrm_re, cuda), to_dev(s.nrm_im, cuda), leaf_size=leaf,
                         sep=sep, precision=cf.MIXED)
    um = pm.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    assert relerr_l2(um, uo) <= 1e-6
