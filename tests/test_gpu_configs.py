"""The benchmark configurations at their stated sizes and accuracies, through
the C ABI against the oracle.

* 2D Helmholtz SLP+DLP, k = 20, N = 1e5 curve, leaf 64, FP64: tree,
  permutation and Lists 1-4 bit-exact and the FMM within relative l2 1e-12 of
  the oracle FMM over all targets (eps = 1e-6); at eps = 1e-9 within eps of the
  direct sum on sampled targets.
* 3D Laplace SLP+DLP at eps = 1e-6 against the oracle FMM (1e-12).
* 3D Laplace and Helmholtz (k = 10) single layer on the N = 1e6 plane with a
  bump, eps = 1e-6, FP64 and MIXED, within eps of the direct sum on 1,000
  sampled targets (relative l2 over the sample).
* CFMM_GREEN_SCALE through cfmm_apply for all four kernels: the constant-free
  result times -1/(2 pi), i/4, 1/(4 pi), 1/(4 pi), and within eps of the
  oracle's scaled direct sum.
"""
import numpy as np
import pytest

from cfmm_inputs import curve2d, curve2d_long, surface3d, plane3d, densities
from oracle import fmm2d, fmm3d, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2
from tests.gpu_util import gpu_plan, to_dev, compare_tree, direct_sampled

pytestmark = pytest.mark.gpu


def _export(p):
    t = p.export_tree()
    lists = [p.export_list(w) for w in (1, 2, 3, 4)]
    return t, lists


def test_helm2d_workload_full_size_vs_oracle_fmm(cuda):
    """N = 1e5: the oracle FMM over every target, and the tree bit for bit."""
    import paper_2509_05458_gb300 as cf
    g = curve2d_long()
    eps = 1e-6
    p = gpu_plan(cf, g, cf.HELMHOLTZ, 20.0, eps, cuda, 64, dlp=True)
    dens = densities(g.n, seed=0, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    T = tr.build_tree(g.re, g.im, 64, k=1, kappa=20.0, eps=eps, helmholtz=True)
    t, lists = _export(p)
    compare_tree(T, t, lists)
    assert p.info()["l0"] == T.l0
    uo, _ = fmm2d.apply(g.re, g.im, 1, 20.0, eps, 64, sigma=dens[0, 0], tau=dens[0, 1], nrm_re=g.nrm_re,
                        nrm_im=g.nrm_im, T=T)
    assert relerr_l2(u, uo) <= 1e-12


def test_helm2d_workload_eps_1e9_sampled(cuda):
    import paper_2509_05458_gb300 as cf
    g = curve2d_long()
    eps = 1e-9
    p = gpu_plan(cf, g, cf.HELMHOLTZ, 20.0, eps, cuda, 64, dlp=True)
    dens = densities(g.n, seed=0, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    idx = np.random.default_rng(4).choice(g.n, 400, replace=False)
    pts = g.re + 1j * g.im
    u0 = direct_sampled(2, 1, 20.0, pts, idx, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_l2(u[idx], u0) <= eps


def test_laplace3d_slp_dlp_eps_1e6_vs_oracle_fmm(cuda):
    import paper_2509_05458_gb300 as cf
    g = surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    eps = 1e-6
    p = gpu_plan(cf, g, cf.LAPLACE, 0.0, eps, cuda, 32, sep=2, dlp=True)
    dens = densities(g.n, seed=12, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    uo, T = fmm3d.apply(g.re, g.im, eps, 32, k=2, sigma=dens[0, 0], tau=dens[0, 1], nrm_re=g.nrm_re,
                        nrm_im=g.nrm_im)
    assert list(p.orders()) == fmm3d.expansion_orders(T, eps)
    assert relerr_l2(u, uo) <= 1e-12
    pts = g.re + 1j * g.im
    u0 = direct(3, 0, 0.0, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_paper(u, u0, dens[0].reshape(-1)) <= eps


_SURF = {}


def _surface_reference(ker, kap):
    """The 1e6-point surface, its densities and the oracle's direct sum at 1,000
    sampled targets (computed once per kernel)."""
    if ker not in _SURF:
        g = plane3d(1_000_000)
        dens = densities(g.n, seed=1, nrhs=1, ncomp=1)
        idx = np.random.default_rng(5).choice(g.n, 1000, replace=False)
        u0 = direct_sampled(3, ker, kap, g.re + 1j * g.im, idx, sigma=dens[0, 0])
        _SURF[ker] = (g, dens, idx, u0)
    return _SURF[ker]


@pytest.mark.parametrize("ker,kap", [(1, 10.0), (0, 0.0)])
@pytest.mark.parametrize("precision,leaf", [(0, 128), (1, 256)])
def test_surface3d_full_size_sampled(cuda, ker, kap, precision, leaf):
    """N = 1e6, eps = 1e-6, separation 2, the benchmark's leaf sizes."""
    import paper_2509_05458_gb300 as cf
    g, dens, idx, u0 = _surface_reference(ker, kap)
    eps = 1e-6
    p = gpu_plan(cf, g, ker, kap, eps, cuda, leaf, sep=2, precision=precision)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    p.destroy()
    assert relerr_l2(u[idx], u0) <= eps


@pytest.mark.parametrize("dim,ker,kap", [(2, 0, 0.0), (2, 1, 8.0), (3, 0, 0.0), (3, 1, 4.0)])
def test_green_scale_through_apply(cuda, dim, ker, kap):
    import paper_2509_05458_gb300 as cf
    from oracle.direct import GREEN_SCALE
    g = curve2d(2000, seed=13, t_half=8.0, height=0.5) if dim == 2 else \
        surface3d(1500, seed=13, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    eps = 1e-6
    dens = densities(g.n, seed=14, nrhs=1, ncomp=2)
    d = to_dev(dens, cuda)
    p0 = gpu_plan(cf, g, ker, kap, eps, cuda, 32, sep=2 if dim == 3 else 1, dlp=True)
    p1 = gpu_plan(cf, g, ker | cf.GREEN_SCALE, kap, eps, cuda, 32, sep=2 if dim == 3 else 1, dlp=True)
    u0 = p0.apply(d).cpu().numpy()[0]
    u1 = p1.apply(d).cpu().numpy()[0]
    c = GREEN_SCALE[(dim, ker)]
    assert relerr_l2(u1, c * u0) <= 1e-15
    pts = g.re + 1j * g.im
    ref = direct(dim, ker, kap, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im,
                 green_scale=True)
    assert relerr_paper(u1, ref, abs(c) * dens[0].reshape(-1)) <= eps
