"""Mixed precision (near field and L2P in complex64 arithmetic with
compensated sums, single-layer 3D P2M with complex64 products and FP64 sums,
translations FP64) against the FP64 oracle FMM on the same tree and orders:
relative l2 <= 1e-6 for all four kernels, single and double layer; with the
double layer the complex64 L2P runs as its own launch (one more kernel per
apply than the FP64 pass)."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle import fmm2d, fmm3d, helm3d as H
from oracle.direct import relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu


def _geom(dim):
    return curve2d(2500, seed=21, t_half=10.0, height=0.5) if dim == 2 else \
        surface3d(1500, seed=21, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)


def _oracle(dim, ker, kap, eps, leaf, sep, g, dens, dlp=True):
    tau = (lambda r: dens[r, 1]) if dlp else (lambda r: None)
    nrm = dict(nrm_re=g.nrm_re, nrm_im=g.nrm_im) if dlp else {}
    if dim == 2:
        return np.stack([fmm2d.apply(g.re, g.im, ker, kap, eps, leaf, k=sep, sigma=dens[r, 0], tau=tau(r),
                                     **nrm)[0] for r in range(dens.shape[0])])
    if ker == 0:
        return np.stack([fmm3d.apply(g.re, g.im, eps, leaf, k=sep, sigma=dens[r, 0], tau=tau(r), **nrm)[0]
                         for r in range(dens.shape[0])])
    kw = dict(sigma=dens[:, 0], tau=dens[:, 1], **nrm) if dlp else dict(sigma=dens[:, 0])
    return H.apply(g.re, g.im, kap, eps, leaf, k=sep, coaxial="exact", **kw)[0]


@pytest.mark.parametrize("dlp", [True, False])
@pytest.mark.parametrize("dim,ker,kap,sep", [(2, 0, 0.0, 1), (2, 1, 20.0, 1), (3, 0, 0.0, 2), (3, 1, 3.0, 2)])
def test_mixed_vs_fp64_oracle_fmm(cuda, dim, ker, kap, sep, dlp):
    import paper_2509_05458_gb300 as cf
    g = _geom(dim)
    eps, leaf = 1e-6, 32
    dens = densities(g.n, seed=22, nrhs=1, ncomp=2 if dlp else 1)
    d = to_dev(dens, cuda)
    pm = gpu_plan(cf, g, ker, kap, eps, cuda, leaf, sep=sep, dlp=dlp, precision=cf.MIXED)
    pf = gpu_plan(cf, g, ker, kap, eps, cuda, leaf, sep=sep, dlp=dlp, precision=cf.FP64)
    n0 = cf.launch_count()
    um = pm.apply(d).cpu().numpy()
    n1 = cf.launch_count()
    uf = pf.apply(d).cpu().numpy()
    n2 = cf.launch_count()
    if dlp:
        assert (n1 - n0) == (n2 - n1) + 1
    uo = _oracle(dim, ker, kap, eps, leaf, sep, g, dens, dlp)
    assert relerr_l2(uf[0], uo[0]) <= 1e-12
    assert relerr_l2(um[0], uo[0]) <= 1e-6
