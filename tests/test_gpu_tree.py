"""GPU tree, permutation and Lists 1-4 are bit-exact against the oracle
(Sec. 6.1-6.2, readings in oracle/tree.py); complexified centres agree to
rounding (Eq. complexify_center_average)."""
import numpy as np
import pytest

from cfmm_inputs import curve2d_short, curve2d, surface3d
from oracle import tree as tr
from tests.gpu_util import gpu_plan, compare_tree

pytestmark = pytest.mark.gpu

CASES = [
    ("2d-lap-short-curve", lambda: curve2d_short(), 2, 0, 0.0, 32, 1),
    ("2d-lap-sep2", lambda: curve2d(3000, seed=2, t_half=10.0, height=0.6), 2, 0, 0.0, 16, 2),
    ("2d-helm-k20", lambda: curve2d(3000, seed=3, t_half=10.0, height=0.5), 2, 1, 20.0, 32, 1),
    ("2d-ragged", lambda: curve2d(1237, seed=9, t_half=3.0, height=1.5), 2, 0, 0.0, 7, 1),
    ("3d-lap", lambda: surface3d(4000, seed=1, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0), 3, 0, 0.0, 16, 1),
    ("3d-helm", lambda: surface3d(3000, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0), 3, 1, 6.0, 16, 1),
]


@pytest.mark.parametrize("name,geom,dim,ker,kap,leaf,sep", CASES, ids=[c[0] for c in CASES])
def test_tree_and_lists_bit_exact(cuda, name, geom, dim, ker, kap, leaf, sep):
    import paper_2509_05458_gb300 as cf
    g = geom()
    eps = 1e-6
    T = tr.build_tree(g.re, g.im, leaf, k=sep, kappa=kap, eps=eps, helmholtz=(ker == 1))
    p = gpu_plan(cf, g, ker, kap, eps, cuda, leaf, sep=sep)
    inf = p.info()
    assert inf["nboxes"] == T.nboxes and inf["nlevels"] == T.nlevels and inf["l0"] == T.l0
    np.testing.assert_array_equal(np.array(inf["root_lo"]), T.lo)
    assert inf["root_width"] == T.W
    tg = p.export_tree()
    compare_tree(T, tg, [p.export_list(w) for w in (1, 2, 3, 4)])
    np.testing.assert_allclose(tg["center_re"], T.center_re, rtol=0, atol=1e-14 * T.W)
    np.testing.assert_allclose(tg["center_im"], T.center_im, rtol=1e-13, atol=1e-13 * T.W)


def test_single_point_and_single_leaf(cuda):
    import paper_2509_05458_gb300 as cf
    g = curve2d(1, seed=0)
    p = gpu_plan(cf, g, 0, 0.0, 1e-6, cuda, 64)
    assert p.info()["nboxes"] == 1
    g = curve2d(50, seed=0)
    p = gpu_plan(cf, g, 0, 0.0, 1e-6, cuda, 64)
    inf = p.info()
    assert inf["nboxes"] == 1 and inf["list_len"][0] == 1
