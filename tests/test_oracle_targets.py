"""Pins of the oracle's separate-target reading (oracle/targets.py): the FMM on
sources and targets together, targets with zero density, matches the direct
sum with separate targets (the definition, Sec. 2.3) within eps, in 2D and 3D,
single and double layer, with targets whose imaginary parts follow their own
function of the real part."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle import fmm2d, fmm3d, helm3d as H
from oracle.direct import direct, relerr_paper
from oracle.targets import union_apply


def _targets_2d(n):
    # a parallel curve 1.5 above the sources with its own imaginary slope (the
    # cross pairs keep |Im dx| well below |Re dx|)
    g = curve2d(n, seed=31, t_half=10.0, height=0.5, slope=0.45)
    g.re[:, 1] += 1.5
    return g


@pytest.mark.parametrize("ker,kap", [(0, 0.0), (1, 6.0)])
def test_separate_targets_2d(ker, kap):
    s = curve2d(1200, seed=30, t_half=10.0, height=0.5)
    t = _targets_2d(500)
    eps = 1e-6
    dens = densities(s.n, seed=32, nrhs=1, ncomp=2)
    u, T = union_apply(lambda re, im, **kw: fmm2d.apply(re, im, ker, kap, eps, 24, **kw), s.re, s.im, t.re, t.im,
                       sigma=dens[0, 0], tau=dens[0, 1], nrm_re=s.nrm_re, nrm_im=s.nrm_im)
    u0 = direct(2, ker, kap, s.re + 1j * s.im, t.re + 1j * t.im, sigma=dens[0, 0], tau=dens[0, 1],
                nrm=s.nrm_re + 1j * s.nrm_im)
    assert u.shape == (t.n,)
    assert relerr_paper(u, u0, dens[0].reshape(-1)) <= eps


@pytest.mark.slow
@pytest.mark.parametrize("ker,kap", [(0, 0.0), (1, 3.0)])
def test_separate_targets_3d(ker, kap):
    s = surface3d(900, seed=33, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    t = surface3d(300, seed=34, half=4.0, amp=0.5, width=1.0, slope=0.2, rho0=1.0)
    t.re[:, 2] += 1.0
    eps = 1e-3
    dens = densities(s.n, seed=35, nrhs=1, ncomp=1)
    if ker == 0:
        f = lambda re, im, **kw: fmm3d.apply(re, im, eps, 24, k=2, **kw)
    else:
        f = lambda re, im, **kw: H.apply(re, im, kap, eps, 24, k=2, coaxial="exact", **kw)
    u, T = union_apply(f, s.re, s.im, t.re, t.im, sigma=dens[0, 0])
    u0 = direct(3, ker, kap, s.re + 1j * s.im, t.re + 1j * t.im, sigma=dens[0, 0])
    assert relerr_paper(u, u0, dens[0, 0]) <= eps
