"""GPU 2D FMM (Sec. 6.4 with the operators of Sec. 4) against the oracle:
same tree, same P per level, element-by-element relative l2 <= 1e-12 against
the oracle FMM, and the direct sum within eps (Eq. relerr)."""
import numpy as np
import pytest

from cfmm_inputs import curve2d_short, curve2d_long, curve2d, densities
from oracle import fmm2d, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2
from tests.gpu_util import gpu_plan, to_dev

pytestmark = pytest.mark.gpu


def _run(cuda, g, ker, kap, eps, leaf, dlp, nrhs=1, sep=1, seed=0):
    import paper_2509_05458_gb300 as cf
    p = gpu_plan(cf, g, ker, kap, eps, cuda, leaf, sep=sep, dlp=dlp)
    ncomp = 2 if dlp else 1
    dens = densities(g.n, seed=seed, nrhs=nrhs, ncomp=ncomp)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()
    return p, dens, u


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_laplace_short_curve_vs_oracle_fmm(cuda, eps):
    g = curve2d_short()
    p, dens, u = _run(cuda, g, 0, 0.0, eps, 32, False)
    uo, T = fmm2d.apply(g.re, g.im, 0, 0.0, eps, 32, sigma=dens[0, 0])
    assert list(p.orders()) == fmm2d.expansion_orders(T, 0, 0.0, eps)
    assert relerr_l2(u[0], uo) <= 1e-12
    pts = g.re + 1j * g.im
    u0 = direct(2, 0, 0.0, pts, pts, sigma=dens[0, 0])
    assert relerr_paper(u[0], u0, dens[0, 0]) <= eps


@pytest.mark.parametrize("ker,kap", [(0, 0.0), (1, 20.0), (1, 1.5)])
def test_slp_dlp_vs_oracle_fmm(cuda, ker, kap):
    g = curve2d(2500, seed=3, t_half=10.0, height=0.5)
    eps = 1e-6
    p, dens, u = _run(cuda, g, ker, kap, eps, 24, True, nrhs=2)
    for r in range(2):
        uo, T = fmm2d.apply(g.re, g.im, ker, kap, eps, 24, sigma=dens[r, 0], tau=dens[r, 1],
                            nrm_re=g.nrm_re, nrm_im=g.nrm_im)
        assert p.info()["l0"] == T.l0
        assert relerr_l2(u[r], uo) <= 1e-12, r


def test_helmholtz_meets_eps_vs_direct(cuda):
    g = curve2d(3000, seed=5, t_half=10.0, height=0.8)
    pts = g.re + 1j * g.im
    nrm = g.nrm_re + 1j * g.nrm_im
    for eps in (1e-6, 1e-9):
        p, dens, u = _run(cuda, g, 1, 20.0, eps, 32, True, seed=1)
        u0 = direct(2, 1, 20.0, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=nrm)
        assert relerr_paper(u[0], u0, dens[0].reshape(-1)) <= eps


def test_single_leaf_equals_direct(cuda):
    g = curve2d(40, seed=1)
    p, dens, u = _run(cuda, g, 1, 3.0, 1e-6, 64, True)
    pts = g.re + 1j * g.im
    u0 = direct(2, 1, 3.0, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    np.testing.assert_allclose(u[0], u0, rtol=1e-12, atol=1e-12 * np.abs(u0).max())


def test_repeat_apply_bitwise_identical(cuda):
    g = curve2d(2000, seed=6, t_half=10.0)
    import paper_2509_05458_gb300 as cf
    p = gpu_plan(cf, g, 1, 20.0, 1e-6, cuda, 32, dlp=True)
    dens = to_dev(densities(g.n, seed=2, ncomp=2), cuda)
    a = p.apply(dens).cpu().numpy()
    b = p.apply(dens).cpu().numpy()
    assert np.array_equal(a, b)


def test_long_curve_full_size_sampled(cuda):
    """2D Helmholtz k=20, N=1e5, SLP+DLP, leaf 64, eps 1e-6: sampled targets vs direct."""
    g = curve2d_long()
    eps = 1e-6
    p, dens, u = _run(cuda, g, 1, 20.0, eps, 64, True)
    rng = np.random.default_rng(1)
    idx = rng.choice(g.n, 150, replace=False)
    pts = g.re + 1j * g.im
    nrm = g.nrm_re + 1j * g.nrm_im
    u0 = direct(2, 1, 20.0, pts, pts[idx], sigma=dens[0, 0], tau=dens[0, 1], nrm=nrm)
    err = np.linalg.norm(u[0, idx] - u0) / np.linalg.norm(u0)
    assert err <= eps, err


@pytest.mark.parametrize("ker,kap", [(0, 0.0), (1, 20.0)])
def test_mixed_precision_fmm(cuda, ker, kap):
    """MIXED: near field in complex64 arithmetic; relative l2 against the FP64
    oracle FMM (same tree, same P) <= 1e-6 and against the direct sum <= eps."""
    import paper_2509_05458_gb300 as cf
    g = curve2d(2500, seed=3, t_half=10.0, height=0.5)
    eps = 1e-6
    p = gpu_plan(cf, g, ker, kap, eps, cuda, 24, dlp=True, precision=cf.MIXED)
    dens = densities(g.n, seed=0, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    uo, T = fmm2d.apply(g.re, g.im, ker, kap, eps, 24, sigma=dens[0, 0], tau=dens[0, 1],
                        nrm_re=g.nrm_re, nrm_im=g.nrm_im)
    assert relerr_l2(u, uo) <= 1e-6
    pts = g.re + 1j * g.im
    u0 = direct(2, ker, kap, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_paper(u, u0, dens[0].reshape(-1)) <= eps


def test_long_curve_mixed_full_size_sampled(cuda):
    """The benchmark workload in MIXED precision meets eps = 1e-6 on sampled targets."""
    import paper_2509_05458_gb300 as cf
    g = curve2d_long()
    eps = 1e-6
    p = gpu_plan(cf, g, 1, 20.0, eps, cuda, 64, dlp=True, precision=cf.MIXED)
    dens = densities(g.n, seed=0, nrhs=1, ncomp=2)
    u = p.apply(to_dev(dens, cuda)).cpu().numpy()[0]
    idx = np.random.default_rng(2).choice(g.n, 150, replace=False)
    pts = g.re + 1j * g.im
    u0 = direct(2, 1, 20.0, pts, pts[idx], sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert np.linalg.norm(u[idx] - u0) / np.linalg.norm(u0) <= eps


def test_autotuned_leaf_size_runs(cuda):
    """The leaf-size autotuner times real applies and returns one of its candidates."""
    import torch
    from paper_2509_05458_gb300 import autotune, HELMHOLTZ, SLP, MIXED
    g = curve2d(20000, seed=9, t_half=20.0)
    t = lambda a: torch.from_numpy(a).to(cuda)
    best, times = autotune.tune_leaf_size(2, HELMHOLTZ | SLP, 10.0, 1e-6, t(g.re), t(g.im), precision=MIXED,
                                          candidates=(32, 64, 128), reps=2)
    assert best in (32, 64, 128) and set(times) == {32, 64, 128}
    assert all(v > 0 for v in times.values())
