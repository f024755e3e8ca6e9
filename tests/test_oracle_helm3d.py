"""Pins of the oracle's 3D complex-coordinate Helmholtz FMM (Sec. 5.3, Sec. 6.4).

Each pin checks the oracle against something other than itself:
* the harmonics Z_n^m against the Laplace solid harmonics (independently
  pinned) and the addition theorem of Eq. sphaddition against numpy's
  Legendre series at complex points;
* spherical Bessel/Hankel functions of complex argument against mpmath;
* gradient relations by finite differences;
* Gegenbauer's addition theorem for e^{ikr}/r at complex points;
* P2M/M2P and P2L/L2P against the direct sum, with geometric decay in P;
* the projection rotation of Eq. mp_y_rot: invariance of the expansion under
  a complex rotation, and identity for Q = I;
* the coaxial z-translation: the projection of Eq. helm3d_M2L_z_axis and the
  exact Gaunt-coefficient translation against each other and against direct
  evaluation of the translated wave functions;
* point-and-shoot M2M, M2L, L2L against the direct sum;
* the whole FMM against the direct sum within eps (Eq. relerr), and a single
  leaf reducing to the direct sum.
"""
import math

import numpy as np
import pytest

from cfmm_inputs import surface3d, densities
from oracle import fmm3d, helm3d as H
from oracle.direct import direct, relerr_paper, relerr_l2

idx = H.idx
x0 = np.array([2.0 + 0.3j, -1.0 + 0.2j, 1.5 - 0.1j])
y0 = np.array([0.2 + 0.05j, 0.3 - 0.02j, -0.1 + 0.03j])
KAPPA = 3.0


def test_harmonics_match_solid_harmonics():
    P = 12
    Z = H.ylm(P, x0)
    U = fmm3d.regular(P, x0)
    for n in range(P + 1):
        for m in range(-n, n + 1):
            e = 1.0 if m >= 0 else (-1.0) ** m
            ref = e * math.sqrt(math.factorial(n - abs(m)) * math.factorial(n + abs(m))) * U[idx(n, m)]
            assert abs(Z[idx(n, m)] - ref) <= 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("P", [10, 40])
def test_spherical_addition_theorem(P):
    Zx, Zy = H.ylm(P, x0), H.ylm(P, y0)
    rx, ry = np.sqrt(x0 @ x0), np.sqrt(y0 @ y0)
    cg = (x0 @ y0) / (rx * ry)
    for n in range(P + 1):
        s = sum(Zx[idx(n, m)] * Zy[idx(n, -m)] for m in range(-n, n + 1)) / (rx * ry) ** n
        c = np.zeros(n + 1)
        c[n] = 1
        ref = np.polynomial.legendre.legval(cg, c)
        assert abs(s - ref) <= 1e-12 * max(1.0, abs(ref))


def test_spherical_bessel_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for z in (0.7 + 0.2j, 3.0 - 0.5j, 12.0 + 2.0j):
        j = H.sph_j(30, np.array(z))
        h = H.sph_h(30, np.array(z))
        for n in (0, 1, 5, 17, 30):
            zz = mp.mpc(z.real, z.imag)
            jr = mp.sqrt(mp.pi / (2 * zz)) * mp.besselj(n + 0.5, zz)
            hr = jr + 1j * mp.sqrt(mp.pi / (2 * zz)) * mp.bessely(n + 0.5, zz)
            assert abs(complex(j[n]) - complex(jr)) <= 1e-12 * abs(complex(jr))
            assert abs(complex(h[n]) - complex(hr)) <= 1e-12 * abs(complex(hr))


def test_gradients_finite_difference():
    P = 10
    v = np.array([0.3 + 0.1j, -0.7, 0.5 - 0.2j])
    h = 1e-6
    fd = (H.ylm(P, x0 + h * v) - H.ylm(P, x0 - h * v)) / (2 * h)
    an = H.ylm_dir(P, x0, v)
    assert np.max(np.abs(fd - an) / np.maximum(1.0, np.abs(an))) < 1e-8
    for kind in ("j", "h"):
        fd = (H.wave(kind, P, KAPPA, x0 + h * v) - H.wave(kind, P, KAPPA, x0 - h * v)) / (2 * h)
        an = H.wave_dir(kind, P, KAPPA, x0, v)
        assert np.max(np.abs(fd - an) / np.maximum(1.0, np.abs(an))) < 1e-7


def test_gegenbauer_addition_complex_points():
    P = 30
    R, S = H.wave("j", P, KAPPA, y0), H.wave("h", P, KAPPA, x0)
    s = sum(1j * KAPPA * (2 * n + 1) * R[idx(n, -m)] * S[idx(n, m)]
            for n in range(P + 1) for m in range(-n, n + 1))
    d = x0 - y0
    r = np.sqrt(d @ d)
    assert abs(s - np.exp(1j * KAPPA * r) / r) < 1e-13


class _W:
    def width(self, level):
        return 1.0


def _cluster(rng, centre, n, half=0.5, slope=0.2):
    re = rng.uniform(-half, half, (n, 3)) + centre
    return re + 1j * slope * re


def test_point_expansions_vs_direct():
    rng = np.random.default_rng(0)
    ops = H.Helmholtz3D(KAPPA, _W())
    src = _cluster(rng, np.zeros(3), 20)
    far = np.array([3.0, 0.0, 0.0])
    trg = _cluster(rng, far, 10)
    sig = rng.normal(size=(1, 20)) + 1j * rng.normal(size=(1, 20))
    tau = rng.normal(size=(1, 20)) + 1j * rng.normal(size=(1, 20))
    nrm = rng.normal(size=(20, 3)) + 0.1j * rng.normal(size=(20, 3))
    u0 = direct(3, 1, KAPPA, src, trg, sigma=sig[0], tau=tau[0], nrm=nrm)
    errs_m, errs_l = [], []
    for P in (8, 14, 20):
        M = ops.p2m(P, src - 0.0, sig, (nrm, tau))
        errs_m.append(relerr_l2(ops.m2p(P, M, trg)[0], u0))
        L = ops.p2l(P, src - far, sig, (nrm, tau))
        errs_l.append(relerr_l2(ops.l2p(P, L, trg - far)[0], u0))
    for e in (errs_m, errs_l):
        assert e[0] > e[1] > e[2]
        assert e[2] < 1e-6 and e[2] < 1e-3 * e[0]


def test_projection_rotation():
    rng = np.random.default_rng(1)
    P = 10
    c = rng.normal(size=(1, (P + 1) ** 2)) + 1j * rng.normal(size=(1, (P + 1) ** 2))
    al = 0.4 + 0.15j
    ca, sa = np.cos(al), np.sin(al)
    Q = np.array([[[ca, 0, -sa], [0, 1, 0], [sa, 0, ca]]])
    ct = H.rotate_proj(c, P, Q)
    for _ in range(3):
        x = rng.normal(size=3) + 0.2j * rng.normal(size=3)
        lhs = c[0] @ H.ylm(P, x)
        rhs = ct[0] @ H.ylm(P, Q[0] @ x)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    same = H.rotate_proj(c, P, np.eye(3)[None].astype(complex))
    assert np.max(np.abs(same - c)) < 1e-13


def test_coaxial_exact_vs_direct_waves():
    """S_{n'}^m(x + t e3) = sum_n T^m_{n n'} R_n^m(x) and R -> R, checked by
    evaluating both sides."""
    t = 1.2 + 0.1j
    x = np.array([0.2 + 0.02j, -0.3, 0.25 - 0.01j])
    Pi, Po = 4, 44
    for kin, kout in (("h", "j"), ("j", "j")):
        for n2 in range(Pi + 1):
            for m in (-min(n2, 2), 0, min(n2, 1)):
                c = np.zeros((1, (Pi + 1) ** 2), complex)
                c[0, idx(n2, m)] = 1.0
                L = H.zshift_exact(c, Pi, Po, np.array([t]), KAPPA, kin, kout)[0]
                lhs = H.wave(kin, Pi, KAPPA, x + np.array([0, 0, t]))[idx(n2, m)]
                rhs = L @ H.wave(kout, Po, KAPPA, x)
                assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_coaxial_projection_vs_exact():
    rng = np.random.default_rng(2)
    P = 20
    c = rng.normal(size=(1, (P + 1) ** 2)) + 1j * rng.normal(size=(1, (P + 1) ** 2))
    c *= np.array([1 / abs(H.sph_h(n, np.array(KAPPA * 0.866))[n]) for n in range(P + 1)
                   for m in range(-n, n + 1)])
    t = np.array([2.0 + 0.2j])
    a = H.zshift(c, P, P, t, 0.866, KAPPA, "h", "j")[0]
    b = H.zshift_exact(c, P, P, t, KAPPA, "h", "j")[0]
    xs = rng.normal(size=(20, 3))
    xs = xs / np.linalg.norm(xs, axis=1)[:, None] * 0.7
    W = H.wave("j", P, KAPPA, xs)
    assert np.max(np.abs(a @ W - b @ W)) <= 1e-12 * np.max(np.abs(b @ W))


@pytest.mark.parametrize("coaxial", ["projection", "exact"])
def test_translations_vs_direct(coaxial):
    rng = np.random.default_rng(3)
    P = 18
    ops = H.Helmholtz3D(KAPPA, _W(), coaxial)
    sig = rng.normal(size=(1, 30)) + 1j * rng.normal(size=(1, 30))
    # M2L: source box at the origin, target box two widths away
    src = _cluster(rng, np.zeros(3), 30)
    tc = np.array([2.0, 1.0, 0.0])
    trg = _cluster(rng, tc, 10)
    cs = 1j * np.mean(src.imag, 0)
    ct = tc + 1j * np.mean(trg.imag, 0)
    M = ops.p2m(P, src - cs, sig)
    L = ops.m2l(P, M, ct - cs, 0)
    u0 = direct(3, 1, KAPPA, src, trg, sigma=sig[0])
    assert relerr_l2(ops.l2p(P, L, trg - ct)[0], u0) < 1e-8
    # M2M: child box of width 1/2 into its parent of width 1
    src2 = _cluster(rng, np.array([0.25, 0.25, 0.25]), 30, half=0.25)
    cc = np.array([0.25, 0.25, 0.25]) + 1j * np.mean(src2.imag, 0)
    cp = 0.5j * np.mean(src2.imag, 0)
    Mp = ops.m2m(P, P, ops.p2m(P, src2 - cc, sig), cc - cp, 0)
    trg3 = _cluster(rng, np.array([2.5, 0, 0]), 10)
    u0 = direct(3, 1, KAPPA, src2, trg3, sigma=sig[0])
    assert relerr_l2(ops.m2p(P, Mp, trg3 - cp)[0], u0) < 1e-8
    # L2L: parent local from far sources, shifted into a child
    ops_c = H.Helmholtz3D(KAPPA, type("W", (), {"width": lambda self, l: 0.5})(), coaxial)
    srcf = _cluster(rng, np.array([3.0, 0.5, -0.5]), 30)
    cp = np.zeros(3) + 0j
    cc = np.array([0.25, 0.25, 0.25]) + 0.05j
    trgc = _cluster(rng, np.array([0.25, 0.25, 0.25]), 10, half=0.25, slope=0.0) + 0.05j
    Lp = ops.p2l(P, srcf - cp, sig)
    Lc = ops_c.l2l(P, P, Lp, cc - cp, 0)
    u0 = direct(3, 1, KAPPA, srcf, trgc, sigma=sig[0])
    assert relerr_l2(ops.l2p(P, Lc, trgc - cc)[0], u0) < 1e-8


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_fmm_vs_direct(eps):
    g = surface3d(900, seed=2, half=3.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0)
    dens = densities(g.n, seed=3, nrhs=1, ncomp=2)
    pts = g.re + 1j * g.im
    u, T = H.apply(g.re, g.im, KAPPA, eps, 24, k=2, sigma=dens[0, 0], tau=dens[0, 1],
                   nrm_re=g.nrm_re, nrm_im=g.nrm_im, coaxial="exact")
    assert T.nlevels >= 3
    u0 = direct(3, 1, KAPPA, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=g.nrm_re + 1j * g.nrm_im)
    assert relerr_paper(u, u0, dens[0].reshape(-1)) <= eps


def test_single_leaf_is_direct():
    g = surface3d(40, seed=4, half=2.0)
    dens = densities(g.n, seed=5, nrhs=1, ncomp=1)
    pts = g.re + 1j * g.im
    u, T = H.apply(g.re, g.im, KAPPA, 1e-6, 64, sigma=dens[0, 0])
    assert T.nboxes == 1
    u0 = direct(3, 1, KAPPA, pts, pts, sigma=dens[0, 0])
    assert relerr_l2(u, u0) < 1e-14


def test_top_level_deeper_than_initial_tree():
    """When no level of the initial tree meets the top-level bound (a shallow
    tree: leaf 700 on 1500 points), the spread is extrapolated below the
    deepest level by halving it per level, the top level is the first level
    where that meets the bound, and the forced refinement reaches it."""
    import math
    from oracle import tree as tr
    g = surface3d(1500, seed=2, half=4.0, amp=0.5, width=1.0, slope=0.8, rho0=1.0)
    kap, eps = 15.0, 1e-3
    T0 = tr.build_tree(g.re, g.im, 700, k=2)
    assert T0.nlevels == 2
    # the deepest initial level misses the bound, one level below meets it
    tau = tr.C_TOP[3] * math.log(eps / tr.EPS_MACH)
    g1 = float(tr.imag_spread(T0, g.im[T0.perm])[T0.box_level == 1].max())
    assert kap * math.sqrt(3) * g1 > tau >= kap * math.sqrt(3) * g1 / 2
    T = tr.build_tree(g.re, g.im, 700, k=2, kappa=kap, eps=eps, helmholtz=True)
    assert T.l0 == 2 and T.nlevels == 3
    assert min(T.box_level[b] for b in range(T.nboxes) if T.box_leaf[b]) >= T.l0


def test_laplace_multipole_from_schmidt_harmonics():
    """The identity the CUDA path's single-layer 3D Laplace P2M uses: with
    Z_n^m = e_m s_n^m U_n^m (s = sqrt((n-|m|)!(n+|m|)!), e_m = (-1)^m for
    m < 0, else 1), the solid-harmonic multipole (-1)^m sum sigma U_n^{-m}(y)
    equals (e_m / s_n^m) sum sigma Z_n^{-m}(y)."""
    rng = np.random.default_rng(11)
    P = 14
    y = rng.normal(size=(25, 3)) * 0.4 + 0.05j * rng.normal(size=(25, 3))
    sig = rng.normal(size=(1, 25)) + 1j * rng.normal(size=(1, 25))
    M = fmm3d.Laplace3D.p2m(P, y, sig)[0]
    Z = H.ylm(P, y)
    for n in range(P + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            s = math.sqrt(math.factorial(n - am) * math.factorial(n + am))
            e = (-1.0) ** m if m < 0 else 1.0
            ref = e / s * (sig[0] @ Z[idx(n, -m)])
            assert abs(M[idx(n, m)] - ref) <= 1e-12 * max(1.0, abs(ref))


def _shifts(rng, n):
    # imaginary parts small enough that |e| = |(d1 + i d2)/s| stays near 1: the
    # direct rotation scales coefficient m by e^m, so |e| far from 1 makes it
    # (not the fixed frame) lose digits
    re = rng.normal(size=(n, 3))
    return re * (1.0 + 0.1j * rng.normal(size=(n, 3)))


@pytest.mark.parametrize("kinds", [("h", "h"), ("h", "j"), ("j", "j")])
def test_fixed_frame_equals_standard_rotation(monkeypatch, kinds):
    """The fixed-frame translation (turn by Q_k, translate Q_k d, turn back) is
    the same operator as the direct rotation to the z-axis: forced on generic
    shifts (both frames k = 0, 1), it reproduces the standard path to 1e-12."""
    rng = np.random.default_rng(7)
    P = 12
    d = _shifts(rng, 8) * 2.0
    d[:4, 1] *= 0.2       # mostly frame 1
    d[4:, 0] *= 0.2       # mostly frame 0
    c = rng.normal(size=(8, (P + 1) ** 2)) + 1j * rng.normal(size=(8, (P + 1) ** 2))
    monkeypatch.setattr(H, "DEGEN_TOL", -1.0)
    ref = H.translate(c, P, P, d, 0.5, KAPPA, kinds[0], kinds[1], coaxial="exact")
    monkeypatch.setattr(H, "DEGEN_TOL", np.inf)
    fr = H._fixed_frame(d)
    assert set(fr) == {0, 1}
    out = H.translate(c, P, P, d, 0.5, KAPPA, kinds[0], kinds[1], coaxial="exact")
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_isotropic_shift_translations(monkeypatch):
    """Shifts with d1^2 + d2^2 = 0 and (d1, d2) != 0 (isotropic complex
    directions, where e = (d1 + i d2)/s is undefined): M2M and M2L through the
    fixed frame reproduce the direct sum; the plain rotation (beta = 0, as for
    a shift on the z-axis) does not."""
    rng = np.random.default_rng(8)
    P = 18
    ops = H.Helmholtz3D(KAPPA, _W(), "exact")
    sig = rng.normal(size=(1, 30)) + 1j * rng.normal(size=(1, 30))
    src = _cluster(rng, np.zeros(3), 30, half=0.25, slope=0.0)
    M = ops.p2m(P, src, sig)
    # M2M to c_new = d: d1^2 + d2^2 = 0.09 - 0.09 = 0
    d = np.array([0.3, 0.3j, 0.6])
    trg = _cluster(rng, np.array([4.0, 1.0, -1.0]), 10, slope=0.0)
    u0 = direct(3, 1, KAPPA, src, trg, sigma=sig[0])
    n0 = H.DEGENERATE["count"]
    Mn = ops.m2m(P, P, M, -d, 0)      # a = c_child - c_parent
    assert H.DEGENERATE["count"] == n0 + 1
    assert relerr_l2(ops.m2p(P, Mn, trg - d)[0], u0) < 1e-8
    # M2L to a target box around t: t1^2 + t2^2 = 2.25 - 2.25 = 0
    t = np.array([1.5, 1.5j, 3.0])
    trg2 = _cluster(rng, np.zeros(3), 10, half=0.25, slope=0.0) + t
    u2 = direct(3, 1, KAPPA, src, trg2, sigma=sig[0])
    L = ops.m2l(P, M, t, 0)
    assert relerr_l2(ops.l2p(P, L, trg2 - t)[0], u2) < 1e-8
    monkeypatch.setattr(H, "DEGEN_TOL", -1.0)
    Lb = ops.m2l(P, M, t, 0)
    assert relerr_l2(ops.l2p(P, Lb, trg2 - t)[0], u2) > 1e-3


def test_isotropic_pair_in_fmm(monkeypatch):
    """An FMM whose tree holds a List-2 pair with an isotropic complex shift
    (cfmm_inputs.isotropic_pair3d): the fixed frame is taken for that pair
    (both directions) and the result meets the direct sum; without it the
    M2L of that pair is wrong."""
    from cfmm_inputs import isotropic_pair3d
    g = isotropic_pair3d()
    pts = g.re + 1j * g.im
    dens = densities(g.n, seed=4, nrhs=1, ncomp=1)[0, 0]
    u0 = direct(3, 1, 1.0, pts, pts, sigma=dens)
    n0 = H.DEGENERATE["count"]
    u, _ = H.apply(g.re, g.im, 1.0, 1e-10, 8, k=2, sigma=dens, coaxial="exact")
    assert H.DEGENERATE["count"] - n0 == 2
    assert relerr_paper(u, u0, dens) <= 1e-10
    monkeypatch.setattr(H, "DEGEN_TOL", -1.0)
    ub, _ = H.apply(g.re, g.im, 1.0, 1e-10, 8, k=2, sigma=dens, coaxial="exact")
    assert relerr_paper(ub, u0, dens) > 1e-4
