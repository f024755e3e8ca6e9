"""Target gradients through the C ABI (cfmm_apply_grad; Sec. 2.1 S' and D' as
normal components): against the oracle's differentiated FMM (same tree and
orders) to relative l2 1e-12, and within eps of the oracle's direct gradient,
for all four kernels, single and double layer; at separate targets; on a
mixed-precision plan."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle import fmm2d, fmm3d, helm3d as H
from oracle.direct import direct_grad, relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu

CASES = [(2, 0, 0.0, 1e-6, 1), (2, 1, 20.0, 1e-6, 1), (3, 0, 0.0, 1e-3, 2), (3, 1, 3.0, 1e-3, 2)]


def _geom(dim):
    return curve2d(2000, seed=3, t_half=10.0, height=0.5) if dim == 2 else \
        surface3d(1200, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)


def _oracle_grad(dim, ker, kap, eps, leaf, sep, re, im, sigma, tau, nre, nim):
    kw = dict(sigma=sigma, tau=tau, nrm_re=nre, nrm_im=nim)
    if dim == 2:
        return fmm2d.apply_grad(re, im, ker, kap, eps, leaf, k=sep, **kw)
    if ker == 0:
        return fmm3d.apply_grad(re, im, eps, leaf, k=sep, **kw)
    return H.apply_grad(re, im, kap, eps, leaf, k=sep, coaxial="exact", **kw)


@pytest.mark.parametrize("dim,ker,kap,eps,sep", CASES)
def test_gradient_vs_oracle(cuda, dim, ker, kap, eps, sep):
    import paper_2509_05458_gb300 as cf
    g = _geom(dim)
    dens = densities(g.n, seed=4, nrhs=1, ncomp=2)
    p = gpu_plan(cf, g, ker, kap, eps, cuda, 24, sep=sep, dlp=True)
    u, gr = p.apply_grad(to_dev(dens, cuda))
    u, gr = u.cpu().numpy()[0], gr.cpu().numpy()[0]
    uo, go, T = _oracle_grad(dim, ker, kap, eps, 24, sep, g.re, g.im, dens[0, 0], dens[0, 1], g.nrm_re, g.nrm_im)
    assert relerr_l2(u, uo) <= 1e-12
    assert relerr_l2(gr.ravel(), go.ravel()) <= 1e-12
    pts, nrm = g.re + 1j * g.im, g.nrm_re + 1j * g.nrm_im
    G0 = direct_grad(dim, ker, kap, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=nrm)
    assert relerr_l2(gr.ravel(), G0.ravel()) <= eps
    # the plain apply gives the same potential bit for bit
    assert np.array_equal(p.apply(to_dev(dens, cuda)).cpu().numpy()[0], u)


@pytest.mark.parametrize("dim,ker,kap,eps,sep", [CASES[1], CASES[3]])
def test_gradient_at_separate_targets_and_mixed(cuda, dim, ker, kap, eps, sep):
    import paper_2509_05458_gb300 as cf
    s = _geom(dim)
    if dim == 2:
        t = curve2d(600, seed=41, t_half=10.0, height=0.5, slope=0.45)
        t.re[:, 1] += 1.5
    else:
        t = surface3d(400, seed=43, half=4.0, amp=0.5, width=1.0, slope=0.25, rho0=1.0)
        t.re[:, 2] += 1.0
    dens = densities(s.n, seed=5, nrhs=1, ncomp=1)
    d = to_dev(dens, cuda)
    p = cf.plan_targets(dim, ker | cf.SLP, kap, eps, to_dev(s.re, cuda), to_dev(s.im, cuda), to_dev(t.re, cuda),
                        to_dev(t.im, cuda), leaf_size=24, sep=sep)
    u, gr = p.apply_grad(d)
    gr = gr.cpu().numpy()[0]
    re, im = np.concatenate([s.re, t.re]), np.concatenate([s.im, t.im])
    sig = np.concatenate([dens[0, 0], np.zeros(t.n, complex)])
    uo, go, T = _oracle_grad(dim, ker, kap, eps, 24, sep, re, im, sig, None, None, None)
    assert relerr_l2(gr.ravel(), go[:, s.n:].ravel()) <= 1e-12
    G0 = direct_grad(dim, ker, kap, s.re + 1j * s.im, t.re + 1j * t.im, sigma=dens[0, 0])
    assert relerr_l2(gr.ravel(), G0.ravel()) <= eps
    # the normal derivative S' along the targets' own normals
    tn = t.nrm_re + 1j * t.nrm_im
    sp = np.sum(gr * tn.T, axis=0)
    sp0 = np.sum(G0 * tn.T, axis=0)
    assert relerr_l2(sp, sp0) <= 10 * eps
    # on a mixed-precision plan the gradient (FP64) sees the complex64 near
    # field only through the expansions
    pm = cf.plan_targets(dim, ker | cf.SLP, kap, eps, to_dev(s.re, cuda), to_dev(s.im, cuda), to_dev(t.re, cuda),
                         to_dev(t.im, cuda), leaf_size=24, sep=sep, precision=cf.MIXED)
    _, gm = pm.apply_grad(d)
    assert relerr_l2(gm.cpu().numpy()[0].ravel(), go[:, s.n:].ravel()) <= 1e-6
