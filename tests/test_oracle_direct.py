"""Pins of the oracle's direct sums (Sec. 2.1 layer potentials; Eqs.
lap_2d_pot, helm_2d_pot, lap_3d_pot and the 3D Helmholtz sum of Sec. 5.3)
against facts the mathematics fixes, not against a retyped formula:

* real points reduce to the textbook real kernels (mpmath / hypot);
* a constant imaginary shift of every point leaves every r_xy unchanged;
* complex-symmetric reciprocity <tau, S sigma> = <sigma, S tau>;
* the double layer is the directional derivative of the single layer
  along the (complex) normal at the source (finite differences);
* Gauss' theorem and Green's representation on complexified closed
  curves and surfaces (the value of a closed contour integral is
  invariant under analytic deformation of the contour).
"""
import numpy as np
import pytest

from oracle.direct import direct, kernel_pair, LAPLACE, HELMHOLTZ

mp = pytest.importorskip("mpmath")
RNG = np.random.default_rng(7)
KERNELS = [(2, LAPLACE, 0.0), (2, HELMHOLTZ, 3.0), (3, LAPLACE, 0.0), (3, HELMHOLTZ, 2.5)]


def _cloud(n, dim, scale_im=0.2, seed=0):
    r = np.random.default_rng(seed)
    re = r.uniform(-1, 1, size=(n, dim))
    im = scale_im * np.tanh(re)          # Lipschitz imaginary part
    return re + 1j * im


@pytest.mark.parametrize("dim,kernel,kap", KERNELS)
def test_real_points_reduce_to_textbook(dim, kernel, kap):
    x = RNG.uniform(-1, 1, size=(6, dim))
    y = RNG.uniform(-1, 1, size=(9, dim))
    s = RNG.standard_normal(9) + 1j * RNG.standard_normal(9)
    u = direct(dim, kernel, kap, y.astype(complex), x.astype(complex), sigma=s)
    for i in range(6):
        ref = mp.mpc(0)
        for j in range(9):
            r = mp.sqrt(sum(mp.mpf(float(x[i, d] - y[j, d])) ** 2 for d in range(dim)))
            if dim == 2 and kernel == LAPLACE:
                k = mp.log(r)
            elif dim == 2:
                k = mp.hankel1(0, kap * r)
            elif kernel == LAPLACE:
                k = 1 / r
            else:
                k = mp.exp(1j * kap * r) / r
            ref += k * mp.mpc(s[j].real, s[j].imag)
        assert abs(u[i] - complex(ref)) < 1e-12 * max(1, abs(complex(ref)))


@pytest.mark.parametrize("dim,kernel,kap", KERNELS)
def test_constant_imaginary_shift_invariance(dim, kernel, kap):
    pts = RNG.uniform(-1, 1, size=(40, dim)).astype(complex)
    nrm = RNG.standard_normal((40, dim)) + 0j
    s = RNG.standard_normal(40) + 1j * RNG.standard_normal(40)
    t = RNG.standard_normal(40) + 1j * RNG.standard_normal(40)
    shift = 1j * RNG.uniform(-3, 3, size=dim)
    u0 = direct(dim, kernel, kap, pts, pts, sigma=s, tau=t, nrm=nrm)
    u1 = direct(dim, kernel, kap, pts + shift, pts + shift, sigma=s, tau=t, nrm=nrm)
    np.testing.assert_allclose(u1, u0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,kernel,kap", KERNELS)
def test_reciprocity_complex_symmetric(dim, kernel, kap):
    pts = _cloud(60, dim)
    s = RNG.standard_normal(60) + 1j * RNG.standard_normal(60)
    t = RNG.standard_normal(60) + 1j * RNG.standard_normal(60)
    Ss = direct(dim, kernel, kap, pts, pts, sigma=s)
    St = direct(dim, kernel, kap, pts, pts, sigma=t)
    assert abs(np.sum(t * Ss) - np.sum(s * St)) < 1e-11 * np.linalg.norm(Ss) * np.linalg.norm(t)


@pytest.mark.parametrize("dim,kernel,kap", KERNELS)
def test_dlp_is_normal_derivative_of_slp(dim, kernel, kap):
    x = _cloud(5, dim, seed=1) + 2.5
    y = _cloud(7, dim, seed=2)
    nrm = RNG.standard_normal((7, dim)) + 1j * 0.3 * RNG.standard_normal((7, dim))
    h = 1e-5
    d = x[:, None, :] - y[None, :, :]
    _, dlp = kernel_pair(dim, kernel, kap, d, np.broadcast_to(nrm[None], d.shape))
    # d/dy along n: K(x, y + h n) - K(x, y - h n) over 2h (K analytic in y)
    kp, _ = kernel_pair(dim, kernel, kap, x[:, None, :] - (y + h * nrm)[None])
    km, _ = kernel_pair(dim, kernel, kap, x[:, None, :] - (y - h * nrm)[None])
    fd = (kp - km) / (2 * h)
    np.testing.assert_allclose(dlp, fd, rtol=1e-7, atol=1e-9)


def _complex_circle(n, delta):
    """Circle with parameter t -> t + i delta sin t: points stay on x1^2+x2^2=1 in C^2."""
    s = 2 * np.pi * np.arange(n) / n
    t = s + 1j * delta * np.sin(s)
    dt = 1 + 1j * delta * np.cos(s)
    g = np.stack([np.cos(t), np.sin(t)], axis=1)
    gp = np.stack([-np.sin(t), np.cos(t)], axis=1) * dt[:, None]
    w = 2 * np.pi / n
    nrm = np.stack([gp[:, 1], -gp[:, 0]], axis=1) * w      # outward normal x weight
    return g, nrm, gp * w


def _complex_curve(n, delta):
    """A closed curve that is not a circle: ellipse-like, complexified in x1 by a
    smooth periodic imaginary part i*delta*sin(2t)."""
    t = 2 * np.pi * np.arange(n) / n
    g = np.stack([1.3 * np.cos(t) + 1j * delta * np.sin(2 * t), 0.9 * np.sin(t)], axis=1)
    gp = np.stack([-1.3 * np.sin(t) + 2j * delta * np.cos(2 * t), 0.9 * np.cos(t)], axis=1)
    w = 2 * np.pi / n
    nrm = np.stack([gp[:, 1], -gp[:, 0]], axis=1) * w
    return g, nrm


@pytest.mark.parametrize("curve", ["circle", "ellipse"])
def test_gauss_2d_laplace_complex_curve(curve):
    """sum n.grad_y log r w = 2 pi (target inside), 0 (outside): Gauss' lemma for
    the constant-free kernel log r = -2 pi G, continued to a complex contour."""
    if curve == "circle":
        g, nrm, _ = _complex_circle(400, 0.15)
    else:
        g, nrm = _complex_curve(400, 0.1)
    tin = np.array([[0.2, 0.1], [-0.3, 0.25]], dtype=complex)
    tout = np.array([[2.2, 0.3], [0.1, 1.8]], dtype=complex)
    one = np.ones(len(g), dtype=complex)
    uin = direct(2, LAPLACE, 0.0, g, tin, tau=one, nrm=nrm)
    uout = direct(2, LAPLACE, 0.0, g, tout, tau=one, nrm=nrm)
    np.testing.assert_allclose(uin, 2 * np.pi, atol=1e-10)
    np.testing.assert_allclose(uout, 0.0, atol=1e-10)


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 2.0)])
def test_green_representation_2d(kernel, kap):
    """S[du/dn] - D[u] = c u(x) inside, 0 outside, for a solution u:
    c = -2 pi (K = log r = -2pi G) and c = -4i (K = H0 = -4i G)."""
    g, nrm = _complex_curve(500, 0.1)
    if kernel == LAPLACE:
        f = lambda p: np.exp(p[..., 0]) * np.cos(p[..., 1])
        grad = lambda p: np.stack([np.exp(p[..., 0]) * np.cos(p[..., 1]),
                                   -np.exp(p[..., 0]) * np.sin(p[..., 1])], -1)
        c = -2 * np.pi
    else:
        dirv = np.array([0.6, 0.8])
        f = lambda p: np.exp(1j * kap * (p @ dirv))
        grad = lambda p: 1j * kap * dirv[None, :] * f(p)[:, None]
        c = -4j
    dudn = np.sum(nrm * grad(g), axis=1)         # weight already in nrm
    u = f(g)
    tin = np.array([[0.2, 0.1], [-0.4, -0.2]], dtype=complex)
    wgt = np.ones(len(g))
    S = direct(2, kernel, kap, g, tin, sigma=dudn)
    D = direct(2, kernel, kap, g, tin, tau=u, nrm=nrm)
    np.testing.assert_allclose(S - D, c * f(tin), atol=1e-9)


def _complex_sphere(nt, nphi, delta):
    """Unit sphere with azimuth phi -> phi + i delta sin phi (stays on x.x = 1)."""
    xg, wg = np.polynomial.legendre.leggauss(nt)
    s = 2 * np.pi * np.arange(nphi) / nphi
    ph = s + 1j * delta * np.sin(s)
    dph = 1 + 1j * delta * np.cos(s)
    ct = xg[:, None]
    st = np.sqrt(1 - ct ** 2)
    p = np.stack(np.broadcast_arrays(st * np.cos(ph), st * np.sin(ph), ct + 0 * ph), -1).reshape(-1, 3)
    # area element d(cos theta) dphi, outward normal = position (|x|=1), times dphi'(s)
    w = (wg[:, None] * (2 * np.pi / nphi) * dph[None, :]).reshape(-1)
    return p, p * w[:, None]


@pytest.mark.parametrize("kernel,kap", [(LAPLACE, 0.0), (HELMHOLTZ, 1.5)])
def test_green_representation_3d(kernel, kap):
    """S[du/dn] - D[u] = 4 pi u(x) inside the complexified sphere
    (K = 1/rho = 4 pi G, and the same constant for e^{ik rho}/rho)."""
    p, nrm = _complex_sphere(24, 48, 0.1)
    if kernel == LAPLACE:
        f = lambda q: q[..., 0] * q[..., 1] + q[..., 2] ** 2 - 0.5 * q[..., 0] ** 2 - 0.5 * q[..., 1] ** 2
        grad = lambda q: np.stack([q[..., 1] - q[..., 0], q[..., 0] - q[..., 1], 2 * q[..., 2]], -1)
    else:
        dv = np.array([0.48, 0.6, 0.64])
        f = lambda q: np.exp(1j * kap * (q @ dv))
        grad = lambda q: 1j * kap * dv[None, :] * f(q)[:, None]
    dudn = np.sum(nrm * grad(p), axis=1)
    u = f(p)
    tin = np.array([[0.1, -0.2, 0.15], [0.0, 0.3, -0.2]], dtype=complex)
    S = direct(3, kernel, kap, p, tin, sigma=dudn)
    D = direct(3, kernel, kap, p, tin, tau=u, nrm=nrm)
    np.testing.assert_allclose(S - D, 4 * np.pi * f(tin), atol=1e-7)


def test_self_pair_skipped():
    pts = _cloud(10, 2)
    s = np.ones(10, complex)
    u = direct(2, LAPLACE, 0.0, pts, pts, sigma=s)
    assert np.all(np.isfinite(u))
