"""Pins of the oracle's 3D complex-coordinate Laplace FMM (Sec. 5.2, Sec. 6.4).

* the solid-harmonic form of the addition theorem (Lemma 5.2.1 with Eq.
  sphaddition) at complex points: 1/|x-y| = sum (-1)^m U_n^{-m}(y) T_n^m(x);
* the regular and irregular translation theorems behind Eqs. L3dM2M,
  L3dM2L, L3dL2L, at complex points;
* the gradient relations used for the double layer (finite differences);
* the multipole truncation bound of Thm 5.2.2 (Eq. lap3d_err_mp) inside the
  proven Lipschitz range, with geometric decay;
* operator chains and the whole FMM against the direct sum (Eq. relerr).
"""
import math

import numpy as np
import pytest

from cfmm_inputs import surface3d, densities
from oracle import fmm3d, tree as tr
from oracle.direct import direct, relerr_paper, relerr_l2

X = fmm3d.Laplace3D
idx = fmm3d.idx
R = fmm3d.regular
T = fmm3d.irregular

x0 = np.array([2.0 + 0.3j, -1.0 + 0.2j, 1.5 - 0.1j])
y0 = np.array([0.2 + 0.05j, 0.3 - 0.02j, -0.1 + 0.03j])


def test_addition_theorem_complex_points():
    P = 28
    Ry, Tx = R(P, y0), T(P, x0)
    s = sum((-1) ** m * Ry[idx(n, -m)] * Tx[idx(n, m)] for n in range(P + 1) for m in range(-n, n + 1))
    d = x0 - y0
    assert abs(s - 1 / np.sqrt(np.sum(d * d))) < 1e-13


def test_translation_theorems():
    a = np.array([0.3 + 0.1j, -0.2, 0.4j])
    b = np.array([0.1, 0.25 - 0.1j, -0.3])
    Ra, Rb, Rab = R(10, a), R(10, b), R(10, a + b)
    for n in range(8):
        for m in range(-n, n + 1):
            s = sum(Ra[idx(k, l)] * Rb[idx(n - k, m - l)] for k in range(n + 1) for l in range(-k, k + 1)
                    if abs(m - l) <= n - k)
            assert abs(s - Rab[idx(n, m)]) < 1e-15
    Tx, Ry, Txy = T(40, x0), R(40, y0), T(4, x0 - y0)
    for n in range(4):
        for m in range(-n, n + 1):
            s = sum((-1) ** l * Ry[idx(k, -l)] * Tx[idx(n + k, m + l)] for k in range(0, 34)
                    for l in range(-k, k + 1) if abs(m + l) <= n + k)
            assert abs(s - Txy[idx(n, m)]) < 1e-12


def test_gradient_relations_finite_difference():
    v = np.array([0.3 + 0.1j, -0.7, 0.5 - 0.2j])
    h = 1e-6
    nup, num = v[0] + 1j * v[1], v[0] - 1j * v[1]
    g = lambda tab, n, m: tab[idx(n, m)] if 0 <= n and abs(m) <= n else 0
    R0, T0 = R(9, y0), T(9, x0)
    Rp, Rm = R(8, y0 + h * v), R(8, y0 - h * v)
    Tp, Tm = T(7, x0 + h * v), T(7, x0 - h * v)
    for n in range(0, 8):
        for m in range(-n, n + 1):
            fd = (Rp[idx(n, m)] - Rm[idx(n, m)]) / (2 * h)
            an = -0.5 * nup * g(R0, n - 1, m - 1) + 0.5 * num * g(R0, n - 1, m + 1) + v[2] * g(R0, n - 1, m)
            assert abs(fd - an) < 1e-8 * max(1, abs(fd))
            if n <= 7:
                fd = (Tp[idx(n, m)] - Tm[idx(n, m)]) / (2 * h)
                an = -0.5 * nup * g(T0, n + 1, m - 1) + 0.5 * num * g(T0, n + 1, m + 1) - v[2] * g(T0, n + 1, m)
                assert abs(fd - an) < 1e-7 * max(1, abs(fd))


def _cloud(n, c, r, L, seed):
    rr = np.random.default_rng(seed)
    dirs = rr.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    re = dirs * (r * rr.uniform(0, 1, n) ** (1 / 3) * 0.999)[:, None] + c
    A = np.array([[0.6, -0.8, 0], [0.8, 0.6, 0], [0, 0, 1.0]]) * L
    return re + 1j * (re @ A.T), A


def test_multipole_bound_thm522():
    """|u - u_P| <= A/(sqrt(1-L^2) R (c~-1)) c~^-P, c~ = R/(C_L r), for L < z_c."""
    L, r, Rr = 0.05, 1.0, 4.0
    assert L < tr.z_c(Rr / r)
    y, A = _cloud(200, np.zeros(3), r, L, 1)
    rng = np.random.default_rng(2)
    dirs = rng.standard_normal((40, 3))
    xr = dirs / np.linalg.norm(dirs, axis=1)[:, None] * Rr * 1.0001
    x = xr + 1j * (xr @ A.T)
    s = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    u0 = direct(3, 0, 0.0, y, x, sigma=s)
    CL = math.sqrt(L * L + 10 * L + 1) / (1 - L)
    ct = Rr / (CL * r)
    errs = []
    for P in (3, 6, 9, 12):
        u = X.m2p(P, X.p2m(P, y, s[None]), x)[0]
        err = np.max(np.abs(u - u0))
        assert err <= np.abs(s).sum() / (math.sqrt(1 - L * L) * Rr * (ct - 1)) * ct ** (-P)
        errs.append(err)
    assert errs[-1] < 1e-3 * errs[0]


def test_operator_chain_with_dipoles():
    y, A = _cloud(60, np.array([3.0, 0.5, 0.2]), 0.35, 0.2, 1)
    x, _ = _cloud(40, np.array([-0.1, 0.1, 0.0]), 0.35, 0.2, 2)
    cpl = lambda c: c + 1j * (c @ A.T)
    cs, cp = cpl(np.array([3.05, 0.45, 0.2])), cpl(np.array([3.3, 0.7, 0.3]))
    ct, cq = cpl(np.array([-0.05, 0.05, 0.0])), cpl(np.array([0.2, 0.25, -0.1]))
    rng = np.random.default_rng(0)
    s = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    t = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    nrm = rng.standard_normal((60, 3)) + 0.2j * rng.standard_normal((60, 3))
    u0 = direct(3, 0, 0.0, y, x, sigma=s, tau=t, nrm=nrm)
    P = 18
    M = X.p2m(P, y - cs, s[None], (nrm, t[None]))
    assert relerr_l2(X.m2p(P, M, x - cs)[0], u0) < 1e-12
    M2 = X.m2m(P, P, M, cs - cp)
    L = X.m2l(P, M2, cq - cp)
    L2 = X.l2l(P, P, L, ct - cq)
    assert relerr_l2(X.l2p(P, L2, x - ct)[0], u0) < 1e-8
    Lp = X.p2l(P, y - ct, s[None], (nrm, t[None]))
    assert relerr_l2(X.l2p(P, Lp, x - ct)[0], u0) < 1e-12


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_fmm3d_meets_eps(eps):
    g = surface3d(1200, seed=1, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    pts = g.re + 1j * g.im
    s = densities(g.n, seed=0)[0, 0]
    t = densities(g.n, seed=1)[0, 0]
    u0 = direct(3, 0, 0.0, pts, pts, sigma=s, tau=t, nrm=g.nrm_re + 1j * g.nrm_im)
    u, T = fmm3d.apply(g.re, g.im, eps, 24, sigma=s, tau=t, nrm_re=g.nrm_re, nrm_im=g.nrm_im)
    assert T.nboxes > 20
    assert relerr_paper(u, u0, np.concatenate([s, t])) <= eps
