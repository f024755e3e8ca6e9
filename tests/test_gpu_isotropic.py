"""A List-2 pair whose complexified shift d has d1^2 + d2^2 = 0 with
(d1, d2) != 0 (an isotropic complex direction, where the z-rotation of the
point-and-shoot translation has no angle): the GPU translates it in the frame
of a fixed real rotation. 3D Helmholtz against the oracle FMM (same fallback)
and 3D Laplace against the oracle FMM (direct O(P^4) translations, no
rotation), both to 1e-12, and both within eps of the direct sum."""
import pytest

from cfmm_inputs import isotropic_pair3d, densities
from oracle import fmm3d, helm3d as H, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ker,kap", [(1, 1.0), (0, 0.0)])
@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_isotropic_shift_pair(cuda, ker, kap, eps):
    import paper_2509_05458_gb300 as cf
    g = isotropic_pair3d()
    p = gpu_plan(cf, g, ker, kap, eps, cuda, 8, sep=2)
    dens = densities(g.n, seed=4, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    if ker == 1:
        T = tr.build_tree(g.re, g.im, 8, k=2, kappa=kap, eps=eps, helmholtz=True)
        n0 = H.DEGENERATE["count"]
        uo, _ = H.apply(g.re, g.im, kap, eps, 8, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
        assert H.DEGENERATE["count"] - n0 == 2
        uo = uo[0]
    else:
        uo, _ = fmm3d.apply(g.re, g.im, eps, 8, k=2, sigma=dens[0, 0])
    assert relerr_l2(u, uo) <= 1e-12
    pts = g.re + 1j * g.im
    u0 = direct(3, ker, kap, pts, pts, sigma=dens[0, 0])
    assert relerr_paper(u, u0, dens[0, 0]) <= eps
