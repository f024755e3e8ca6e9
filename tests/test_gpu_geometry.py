"""The geometry assumption (Assumptions 4.1/5.1: Im x Lipschitz in Re x with
L < 1, so Re r^2 > 0) checked at plan time, and the automatic separation
chosen from the Lipschitz estimate (Sec. 6.3 limits), against the oracle."""
import numpy as np
import pytest

import math

from cfmm_inputs import curve2d, surface3d
from oracle import tree as tr
from tests.gpu_util import gpu_plan, compare_tree

pytestmark = pytest.mark.gpu


def test_geometry_outside_assumptions_fails_with_egeom(cuda):
    import paper_2509_05458_gb300 as cf
    g = curve2d(2000, seed=2, slope=1.3)
    with pytest.raises(cf.CfmmError) as e:
        gpu_plan(cf, g, cf.HELMHOLTZ, 5.0, 1e-6, cuda, 32)
    assert e.value.status == cf.EGEOM


@pytest.mark.parametrize("dim,slope,kap", [(2, 0.5, 20.0), (3, 0.4, 6.0), (3, 0.73, 6.0)])
def test_lipschitz_estimate_and_auto_separation(cuda, dim, slope, kap):
    import paper_2509_05458_gb300 as cf
    g = curve2d(3000, seed=3, t_half=10.0, height=0.5, slope=slope) if dim == 2 else \
        surface3d(3000, seed=3, half=8.0, slope=slope, rho0=2.0)
    eps, leaf = 1e-6, 24
    p = gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=-1)
    inf = p.info()
    T0 = tr.build_tree(g.re, g.im, leaf)
    L = tr.lipschitz_estimate(g.re[T0.perm], g.im[T0.perm])
    assert abs(inf["lipschitz"] - L) <= 1e-5 * L
    k = tr.auto_separation(dim, L)
    assert inf["sep"] == k
    T = tr.build_tree(g.re, g.im, leaf, k=k, kappa=kap, eps=eps, helmholtz=True)
    compare_tree(T, p.export_tree(), [p.export_list(w) for w in (1, 2, 3, 4)])
