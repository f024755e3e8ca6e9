"""GPU 3D Helmholtz FMM (Sec. 5.3 operators, Sec. 6.4 steps) against the oracle:
same tree and P, element by element relative l2 <= 1e-12 against the oracle
FMM with the exact coaxial translation (the CUDA path's translation; the
paper's projection differs from it by its aliasing error); within eps of the
direct sum; mixed precision against the FP64 oracle; a single leaf."""
import numpy as np
import pytest

from cfmm_inputs import surface3d, densities
from oracle import helm3d as H, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu

KAPPA = 3.0


def _geom():
    return surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)


@pytest.mark.parametrize("eps,sep", [(1e-3, 1), (1e-3, 2), (1e-6, 2)])
def test_helm3d_vs_oracle_fmm(cuda, eps, sep):
    import paper_2509_05458_gb300 as cf
    g = _geom()
    p = gpu_plan(cf, g, cf.HELMHOLTZ, KAPPA, eps, cuda, 24, sep=sep, dlp=True)
    dens = densities(g.n, seed=3, nrhs=2, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    T = tr.build_tree(g.re, g.im, 24, k=sep, kappa=KAPPA, eps=eps, helmholtz=True)
    assert p.info()["l0"] == T.l0
    assert list(p.orders()) == H.expansion_orders(T, KAPPA, eps)
    uo, _ = H.apply(g.re, g.im, KAPPA, eps, 24, k=sep, sigma=dens[:, 0], tau=dens[:, 1], nrm_re=g.nrm_re,
                    nrm_im=g.nrm_im, T=T, coaxial="exact")
    for r in range(2):
        assert relerr_l2(u[r], uo[r]) <= 1e-12
    pts = g.re + 1j * g.im
    u0 = direct(3, 1, KAPPA, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_paper(u[0], u0, dens[0].reshape(-1)) <= eps


@pytest.mark.parametrize("leaf", [24, 96])
def test_helm3d_single_layer_vs_oracle_fmm(cuda, leaf):
    """The single-layer-only P2M/P2L path (one lane per harmonic column)."""
    import paper_2509_05458_gb300 as cf
    g = _geom()
    eps = 1e-3
    p = gpu_plan(cf, g, cf.HELMHOLTZ, KAPPA, eps, cuda, leaf, sep=2, dlp=False)
    dens = densities(g.n, seed=5, nrhs=2, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=KAPPA, eps=eps, helmholtz=True)
    uo, _ = H.apply(g.re, g.im, KAPPA, eps, leaf, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
    for r in range(2):
        assert relerr_l2(u[r], uo[r]) <= 1e-12


def test_helm3d_mixed_precision(cuda):
    import paper_2509_05458_gb300 as cf
    g = _geom()
    eps = 1e-6
    p = gpu_plan(cf, g, cf.HELMHOLTZ, KAPPA, eps, cuda, 24, sep=2, dlp=True, precision=1)
    dens = densities(g.n, seed=4, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    pts = g.re + 1j * g.im
    u0 = direct(3, 1, KAPPA, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_l2(u, u0) <= 1e-6


def test_helm3d_single_leaf(cuda):
    import paper_2509_05458_gb300 as cf
    g = surface3d(50, seed=6, half=2.0)
    p = gpu_plan(cf, g, cf.HELMHOLTZ, KAPPA, 1e-6, cuda, 64)
    dens = densities(g.n, seed=7, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    pts = g.re + 1j * g.im
    u0 = direct(3, 1, KAPPA, pts, pts, sigma=dens[0, 0])
    assert relerr_l2(u, u0) <= 1e-13


def test_helm3d_repeat_bitwise(cuda):
    import paper_2509_05458_gb300 as cf
    g = _geom()
    p = gpu_plan(cf, g, cf.HELMHOLTZ, KAPPA, 1e-3, cuda, 24, sep=2)
    d = to_dev(densities(g.n, seed=8, nrhs=1, ncomp=1), cuda)
    a = p.apply(d).cpu().numpy()
    b = p.apply(d).cpu().numpy()
    assert np.array_equal(a, b)


def test_helm3d_top_level_deeper_than_initial_tree(cuda):
    """A shallow initial tree (leaf 700 on 1500 points) none of whose levels
    meets the top-level bound: both sides extrapolate the spread below the
    deepest level and refine to the level it picks."""
    import paper_2509_05458_gb300 as cf
    g = surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.8, rho0=1.0)
    kap, eps, leaf = 15.0, 1e-3, 700
    p = gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=2)
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True)
    assert p.info()["l0"] == T.l0 == 2
    assert list(p.orders()) == H.expansion_orders(T, kap, eps)
    dens = densities(g.n, seed=9, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    uo, _ = H.apply(g.re, g.im, kap, eps, leaf, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
    assert relerr_l2(u[0], uo[0]) <= 1e-12


# expansion order limit of the CUDA 3D translation kernels (a property of the
# library, not of the method)
GPU_MAX_ORDER_3D = 63


def test_helm3d_order_above_limit_unsupported(cuda):
    """Where the top-level rule picks a level whose order exceeds the library's
    3D limit, the plan fails with CFMM_EUNSUPPORTED (the oracle has no limit)."""
    import paper_2509_05458_gb300 as cf
    g = _geom()
    kap, eps, leaf = 25.0, 1e-6, 64
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True)
    assert H.expansion_orders(T, kap, eps)[T.l0] > GPU_MAX_ORDER_3D
    with pytest.raises(cf.CfmmError) as e:
        gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=2)
    assert e.value.status == cf.EUNSUPPORTED


@pytest.mark.parametrize("kap,eps,leaf", [(20.0, 1e-3, 700), (25.0, 1e-6, 64)])
def test_helm3d_explicit_top_level(cuda, kap, eps, leaf):
    """The same explicit top level on both sides where the rule's own level
    needs an order above the library's limit: a top level below a shallow
    initial tree (leaf 700), and a top-level order above 57 (kappa = 25, P = 59),
    where the translation kernel keeps its accumulator in global scratch as
    well as its coaxial work arrays."""
    import paper_2509_05458_gb300 as cf
    g = _geom()
    top = 2
    p = gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=2, top_level=top)
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True, top_level=top)
    orders = H.expansion_orders(T, kap, eps)
    assert p.info()["l0"] == T.l0 == top
    assert orders[T.l0] <= GPU_MAX_ORDER_3D
    assert min(T.box_level[b] for b in range(T.nboxes) if T.box_leaf[b]) >= top
    assert list(p.orders()) == orders
    dens = densities(g.n, seed=10, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    uo, _ = H.apply(g.re, g.im, kap, eps, leaf, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
    assert relerr_l2(u[0], uo[0]) <= 1e-12
    if kap == 25.0:
        assert orders[T.l0] > 57
        pts = g.re + 1j * g.im
        u0 = direct(3, 1, kap, pts, pts, sigma=dens[0, 0])
        assert relerr_paper(u[0], u0, dens[0].reshape(-1)) <= eps


def test_helm3d_top_fit(cuda):
    """CFMM_TOP_FIT: where the rule's top level needs an order above the
    library's limit, the plan takes the first deeper level whose order fits;
    the oracle, given that level explicitly, agrees to 1e-12."""
    import paper_2509_05458_gb300 as cf
    g = _geom()
    kap, eps, leaf = 25.0, 1e-6, 64
    T0 = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True)
    o0 = H.expansion_orders(T0, kap, eps)
    assert o0[T0.l0] > GPU_MAX_ORDER_3D
    top = T0.l0
    while o0[top] > GPU_MAX_ORDER_3D:
        top += 1
    p = gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=2, top_level=cf.TOP_FIT)
    assert p.info()["l0"] == top
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True, top_level=top)
    assert list(p.orders()) == H.expansion_orders(T, kap, eps)
    dens = densities(g.n, seed=11, nrhs=1, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    uo, _ = H.apply(g.re, g.im, kap, eps, leaf, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
    assert relerr_l2(u[0], uo[0]) <= 1e-12


def test_helm3d_operators_built_ahead_multi_rhs(cuda):
    """Several right-hand sides at a top-level order above 40 (P = 50 at the
    explicit top level 2, kappa = 20): the M2L operators are built once for all
    right-hand sides; each right-hand side matches the oracle to 1e-12."""
    import paper_2509_05458_gb300 as cf
    g = _geom()
    kap, eps, leaf, top = 20.0, 1e-6, 64, 2
    p = gpu_plan(cf, g, cf.HELMHOLTZ, kap, eps, cuda, leaf, sep=2, top_level=top)
    T = tr.build_tree(g.re, g.im, leaf, k=2, kappa=kap, eps=eps, helmholtz=True, top_level=top)
    orders = H.expansion_orders(T, kap, eps)
    assert 40 < orders[T.l0] <= 56
    assert list(p.orders()) == orders
    dens = densities(g.n, seed=12, nrhs=3, ncomp=1)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    uo, _ = H.apply(g.re, g.im, kap, eps, leaf, k=2, sigma=dens[:, 0], T=T, coaxial="exact")
    for r in range(3):
        assert relerr_l2(u[r], uo[r]) <= 1e-12
