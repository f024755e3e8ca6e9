"""GPU 3D Laplace FMM (Sec. 5.2 operators, Sec. 6.4 steps) against the oracle:
same tree and P, element-by-element relative l2 <= 1e-12 against the oracle
FMM; within eps of the direct sum; the plane-with-bump surface family at N = 1e5 on
sampled targets."""
import numpy as np
import pytest

from cfmm_inputs import surface3d, plane3d, densities
from oracle import fmm3d
from oracle.direct import direct, relerr_paper, relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_laplace3d_vs_oracle_fmm(cuda, eps):
    import paper_2509_05458_gb300 as cf
    g = surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    p = gpu_plan(cf, g, 0, 0.0, eps, cuda, 24, dlp=True)
    dens = densities(g.n, seed=3, nrhs=2, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    pts = g.re + 1j * g.im
    for r in range(2):
        uo, T = fmm3d.apply(g.re, g.im, eps, 24, sigma=dens[r, 0], tau=dens[r, 1], nrm_re=g.nrm_re,
                            nrm_im=g.nrm_im)
        assert list(p.orders()) == fmm3d.expansion_orders(T, eps)
        assert relerr_l2(u[r], uo) <= 1e-12
    u0 = direct(3, 0, 0.0, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_paper(u[0], u0, dens[0].reshape(-1)) <= eps


@pytest.mark.parametrize("precision", [0, 1])
def test_laplace3d_surface_1e5_sampled(cuda, precision):
    import paper_2509_05458_gb300 as cf
    g = plane3d(100_000)
    eps = 1e-3
    p = gpu_plan(cf, g, 0, 0.0, eps, cuda, 64, precision=precision)
    dens = densities(g.n, seed=4, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    idx = np.random.default_rng(3).choice(g.n, 200, replace=False)
    pts = g.re + 1j * g.im
    u0 = direct(3, 0, 0.0, pts, pts[idx], sigma=dens[0, 0])
    assert np.linalg.norm(u[idx] - u0) / np.linalg.norm(u0) <= eps


def test_laplace3d_single_layer_vs_oracle_fmm(cuda):
    """The single-layer column P2M (one lane per harmonic column, scaled into the
    solid-harmonic basis) at separation 2, against the oracle FMM."""
    import paper_2509_05458_gb300 as cf
    g = surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    eps = 1e-6
    p = gpu_plan(cf, g, 0, 0.0, eps, cuda, 48, sep=2)
    dens = densities(g.n, seed=6, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    uo, T = fmm3d.apply(g.re, g.im, eps, 48, k=2, sigma=dens[0, 0])
    assert list(p.orders()) == fmm3d.expansion_orders(T, eps)
    assert relerr_l2(u[0], uo) <= 1e-12
