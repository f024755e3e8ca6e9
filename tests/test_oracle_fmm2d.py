"""Pins of the oracle's 2D complex-coordinate FMM (Sec. 4, Sec. 6.4).

* whole FMM vs the direct sum within eps (Eq. relerr metric) on the 2D
  Laplace workload (N=4000) and on a 2D Helmholtz case, SLP + DLP;
* a single leaf (N <= N_s) reduces the FMM to the direct sum;
* a constant imaginary shift of all points gives the real-coordinate result;
* single-level operator chains against the direct sum, inside the proven
  Lipschitz range: P2M->M2P below the bound of Thm 4.2.2 (Eq. l2d_mp_err),
  P2M->M2L->L2P below the bound of Thm 4.2.x (Eq. M2L_lap2d_err), with
  geometric decay in P; M2M and L2L exactness; Helmholtz chains converge.
"""
import math

import numpy as np
import pytest

from cfmm_inputs import curve2d_short, curve2d, densities
from oracle import fmm2d, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2, LAPLACE, HELMHOLTZ


@pytest.fixture(scope="module")
def short_curve():
    g = curve2d_short()
    pts = g.re + 1j * g.im
    s = densities(g.n, seed=0)[0, 0]
    u0 = direct(2, LAPLACE, 0.0, pts, pts, sigma=s)
    return g, s, u0


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_laplace_short_curve_meets_eps(short_curve, eps):
    g, s, u0 = short_curve
    u, T = fmm2d.apply(g.re, g.im, LAPLACE, 0.0, eps, 32, sigma=s)
    assert relerr_paper(u, u0, s) <= eps
    assert T.nlevels >= 5


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 20.0), (HELMHOLTZ, 1.0)])
def test_slp_dlp_meets_eps(kernel, kap):
    g = curve2d(1500, seed=3, t_half=10.0, height=0.5)
    pts = g.re + 1j * g.im
    nrm = g.nrm_re + 1j * g.nrm_im
    s = densities(g.n, seed=0)[0, 0]
    t = densities(g.n, seed=1)[0, 0]
    u0 = direct(2, kernel, kap, pts, pts, sigma=s, tau=t, nrm=nrm)
    for eps in (1e-6, 1e-9):
        u, T = fmm2d.apply(g.re, g.im, kernel, kap, eps, 24, sigma=s, tau=t,
                           nrm_re=g.nrm_re, nrm_im=g.nrm_im)
        assert relerr_paper(u, u0, np.concatenate([s, t])) <= eps


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 5.0)])
def test_single_leaf_is_direct(kernel, kap):
    g = curve2d(40, seed=1)
    pts = g.re + 1j * g.im
    s = densities(g.n, seed=2)[0, 0]
    u, T = fmm2d.apply(g.re, g.im, kernel, kap, 1e-6, 64, sigma=s)
    assert T.nboxes == 1
    np.testing.assert_allclose(u, direct(2, kernel, kap, pts, pts, sigma=s), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 4.0)])
def test_constant_imaginary_shift_gives_real_result(kernel, kap):
    g = curve2d(1200, seed=4, t_half=8.0, slope=0.0)
    s = densities(g.n, seed=0)[0, 0]
    u_real, T0 = fmm2d.apply(g.re, np.zeros_like(g.im), kernel, kap, 1e-9, 20, sigma=s)
    u_shift, T1 = fmm2d.apply(g.re, np.zeros_like(g.im) + np.array([0.7, -1.3]), kernel, kap,
                              1e-9, 20, sigma=s)
    assert T0.nboxes == T1.nboxes
    assert relerr_l2(u_shift, u_real) < 1e-12


def _lipschitz_box(n, r, L, center, seed):
    """Points with |Re y - c| < r and Im y = psi(Re y) with Lipschitz constant L."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = r * np.sqrt(rng.uniform(0, 1, n)) * 0.999
    re = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1) + center
    A = np.array([[0.6, -0.8], [0.8, 0.6]]) * L          # rotation times L: Lipschitz L
    im = re @ A.T
    return re + 1j * im, A


def test_laplace_multipole_bound_and_decay():
    """Thm 4.2.2: |u - u_P| <= A/(c-1) c^-P, c = (1-L)R/((1+L)r)."""
    L, r, R = 0.2, 1.0, 3.0
    y, A = _lipschitz_box(300, r, L, np.zeros(2), 0)
    rng = np.random.default_rng(1)
    ang = rng.uniform(0, 2 * np.pi, 50)
    xr = np.stack([np.cos(ang), np.sin(ang)], 1) * R * 1.0001
    x = xr + 1j * (xr @ A.T)
    s = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    u0 = direct(2, LAPLACE, 0.0, y, x, sigma=s)
    X = fmm2d.Expansions2D(LAPLACE, 0.0, None)
    c = (1 - L) * R / ((1 + L) * r)
    Aabs = np.abs(s).sum()
    errs = []
    for P in (4, 8, 12, 16, 20):
        M = X.lap_p2m(P, y, s[None, :])
        u = X.lap_m2p(P, M, x)[0]
        err = np.max(np.abs(u - u0))
        assert err <= Aabs / (c - 1) * c ** (-P)
        errs.append(err)
    assert errs[-1] < 1e-3 * errs[0]


def test_laplace_m2l_bound():
    """Thm 4.2.x M2L: |u - u_P| <= A/(c-1) c^-P, c = (1-L)a/(1+L), |Re x0| > (1+a) r."""
    L, r, a = 0.15, 1.0, 3.0
    src_c = np.array([(1 + a) * r * 1.01, 0.0])
    y, A = _lipschitz_box(200, r, L, src_c, 2)
    x, _ = _lipschitz_box(60, r, L, np.zeros(2), 3)
    cs = src_c + 1j * (src_c @ A.T)
    s = np.random.default_rng(4).standard_normal(200) + 0j
    u0 = direct(2, LAPLACE, 0.0, y, x, sigma=s)
    X = fmm2d.Expansions2D(LAPLACE, 0.0, None)
    c = (1 - L) * a / (1 + L)
    for P in (6, 12, 18):
        M = X.lap_p2m(60, y - cs, s[None, :])          # exact multipole (P=60)
        Lc = X.lap_m2l(60, M, cs)
        Lt = Lc.copy()
        Lt[:, P + 1:61] = 0
        Lt[:, 61 + P:] = 0
        u = X.lap_l2p(60, Lt, x)[0]
        assert np.max(np.abs(u - u0)) <= np.abs(s).sum() / (c - 1) * c ** (-P)


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 2.0)])
def test_operator_chain_single_level(kernel, kap):
    """P2M -> M2M -> M2L -> L2L -> L2P equals the direct sum (charges + dipoles)."""
    L = 0.2
    y, A = _lipschitz_box(100, 0.4, L, np.array([3.0, 0.4]), 5)
    x, _ = _lipschitz_box(50, 0.4, L, np.array([-0.2, 0.1]), 6)
    cplx = lambda c: c + 1j * (c @ A.T)
    cs, cp = cplx(np.array([3.1, 0.3])), cplx(np.array([3.3, 0.6]))
    ct, cq = cplx(np.array([-0.25, 0.05])), cplx(np.array([0.0, 0.2]))
    rng = np.random.default_rng(8)
    s = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    t = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    nrm = rng.standard_normal((100, 2)) + 0.2j * rng.standard_normal((100, 2))
    nu, nut = nrm[:, 0] + 1j * nrm[:, 1], nrm[:, 0] - 1j * nrm[:, 1]
    u0 = direct(2, kernel, kap, y, x, sigma=s, tau=t, nrm=nrm)
    P = 40
    X = fmm2d.Expansions2D(kernel, kap, None)
    if kernel == LAPLACE:
        M = X.lap_p2m(P, y - cs, s[None], (nu, nut, t[None]))
        M = X.lap_m2m(P, P, M, cs - cp)
        Lc = X.lap_m2l(P, M, cp - cq)
        Lc = X.lap_l2l(P, P, Lc, cq - ct)
        u = X.lap_l2p(P, Lc, x - ct)[0]
        # P2L on the same pair
        Lp = X.lap_p2l(P, y - ct, s[None], (nu, nut, t[None]))
        u2 = X.lap_l2p(P, Lp, x - ct)[0]
    else:
        M = X.hel_p2m(P, cs, y, s[None], (nu, nut, t[None]))
        M = X.hel_shift("J", P, P, M, cp - cs)
        Lc = X.hel_shift("H", P, P, M, cq - cp)
        Lc = X.hel_shift("J", P, P, Lc, ct - cq)
        u = X.hel_l2p(P, Lc, ct, x)[0]
        Lp = X.hel_p2l(P, ct, y, s[None], (nu, nut, t[None]))
        u2 = X.hel_l2p(P, Lp, ct, x)[0]
    assert relerr_l2(u, u0) < 1e-10
    assert relerr_l2(u2, u0) < 1e-10
