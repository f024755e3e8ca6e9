"""Pins of the oracle's target gradients (Sec. 2.1: S' and D' are the normal
components of grad_x of the layer potentials):

* the pair gradients (oracle.direct.kernel_pair_grad) equal central finite
  differences of the direct sum in the target coordinates, for all four
  kernels, single and double layer, at complex points;
* the differentiated solid harmonics (oracle.fmm3d.regular_dir/irregular_dir)
  equal finite differences of the harmonics;
* the FMM gradients (differentiated P2P, M2P and L2P) match the direct
  gradient within eps.
"""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle import fmm2d, fmm3d, helm3d as H
from oracle.direct import direct, direct_grad


@pytest.mark.parametrize("dim,ker,kap", [(2, 0, 0.0), (2, 1, 5.0), (3, 0, 0.0), (3, 1, 4.0)])
def test_direct_gradient_is_finite_difference(dim, ker, kap):
    g = curve2d(60, seed=1, t_half=3.0) if dim == 2 else surface3d(60, seed=1, half=2.0, rho0=0.5)
    src, nrm = g.re + 1j * g.im, g.nrm_re + 1j * g.nrm_im
    trg = src[:5] + np.array([0.3, 0.7, 0.2][:dim]) * (1 + 0.1j)
    d = densities(60, seed=2, ncomp=2)[0]
    G = direct_grad(dim, ker, kap, src, trg, sigma=d[0], tau=d[1], nrm=nrm)
    h = 1e-5
    for a in range(dim):
        e = np.zeros(dim)
        e[a] = h
        fd = (direct(dim, ker, kap, src, trg + e, sigma=d[0], tau=d[1], nrm=nrm)
              - direct(dim, ker, kap, src, trg - e, sigma=d[0], tau=d[1], nrm=nrm)) / (2 * h)
        assert np.max(np.abs(fd - G[a])) <= 1e-7 * np.max(np.abs(G[a]))


def test_solid_harmonic_derivatives():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(6, 3)) + 0.1j * rng.normal(size=(6, 3))
    P, h = 8, 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        for f, fd in ((fmm3d.regular, fmm3d.regular_dir), (fmm3d.irregular, fmm3d.irregular_dir)):
            num = (f(P, x + e) - f(P, x - e)) / (2 * h)
            an = fd(P, x, np.eye(3)[a])
            assert np.max(np.abs(num - an)) <= 1e-6 * max(1.0, np.max(np.abs(an)))


@pytest.mark.parametrize("ker,kap,eps", [(0, 0.0, 1e-6), (1, 20.0, 1e-6), (1, 20.0, 1e-9)])
def test_fmm2d_gradient_matches_direct(ker, kap, eps):
    g = curve2d(2000, seed=3, t_half=10.0, height=0.5)
    d = densities(g.n, seed=4, ncomp=2)[0]
    u, gr, T = fmm2d.apply_grad(g.re, g.im, ker, kap, eps, 24, sigma=d[0], tau=d[1], nrm_re=g.nrm_re,
                                nrm_im=g.nrm_im)
    G0 = direct_grad(2, ker, kap, g.re + 1j * g.im, g.re + 1j * g.im, sigma=d[0], tau=d[1],
                     nrm=g.nrm_re + 1j * g.nrm_im)
    assert np.linalg.norm(gr - G0) <= eps * np.linalg.norm(G0)
    # the single layer alone (its gradient is less dominated by the closest pairs)
    u, gr, T = fmm2d.apply_grad(g.re, g.im, ker, kap, eps, 24, sigma=d[0])
    G0 = direct_grad(2, ker, kap, g.re + 1j * g.im, g.re + 1j * g.im, sigma=d[0])
    assert np.linalg.norm(gr - G0) <= eps * np.linalg.norm(G0)


@pytest.mark.slow
@pytest.mark.parametrize("ker,kap", [(0, 0.0), (1, 3.0)])
def test_fmm3d_gradient_matches_direct(ker, kap):
    g = surface3d(1200, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    d = densities(g.n, seed=4, ncomp=2)[0]
    eps = 1e-3
    if ker == 0:
        u, gr, T = fmm3d.apply_grad(g.re, g.im, eps, 24, k=2, sigma=d[0], tau=d[1], nrm_re=g.nrm_re,
                                    nrm_im=g.nrm_im)
    else:
        u, gr, T = H.apply_grad(g.re, g.im, kap, eps, 24, k=2, sigma=d[0], tau=d[1], nrm_re=g.nrm_re,
                                nrm_im=g.nrm_im, coaxial="exact")
    G0 = direct_grad(3, ker, kap, g.re + 1j * g.im, g.re + 1j * g.im, sigma=d[0], tau=d[1],
                     nrm=g.nrm_re + 1j * g.nrm_im)
    assert np.linalg.norm(gr - G0) <= eps * np.linalg.norm(G0)
