"""Pins of the special functions the oracle calls (scipy, complex arguments)
against mpmath at 30 digits: H_n^(1), J_n (Sec. 3.2, Thm 3.2.1) and the
spherical j_n, h_n^(1) (Sec. 3.2) on Re z > 0, plus the Graf addition
theorem (Thm 3.2.1, Eq. addition_for_H) evaluated pointwise at complex
arguments, and the Legendre bound (Eq. lege_bound)."""
import numpy as np
import pytest
import scipy.special as sps

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30

ZS = [0.3 + 0.05j, 1.7 + 0.9j, 4.0 + 2.0j, 9.5 + 3.0j, 25.0 + 12.0j, 2.0 - 0.4j]


@pytest.mark.parametrize("z", ZS)
@pytest.mark.parametrize("n", [0, 1, 2, 7, 25])
def test_hankel_bessel_complex(z, n):
    ref_h = complex(mp.hankel1(n, mp.mpc(z.real, z.imag)))
    ref_j = complex(mp.besselj(n, mp.mpc(z.real, z.imag)))
    assert abs(sps.hankel1(n, z) - ref_h) <= 1e-13 * max(1.0, abs(ref_h))
    assert abs(sps.jv(n, z) - ref_j) <= 1e-13 * max(1.0, abs(ref_j))


@pytest.mark.parametrize("z", ZS)
@pytest.mark.parametrize("n", [0, 1, 5, 20])
def test_spherical_complex(z, n):
    zz = mp.mpc(z.real, z.imag)
    jref = complex(mp.sqrt(mp.pi / (2 * zz)) * mp.besselj(n + mp.mpf(1) / 2, zz))
    href = complex(mp.sqrt(mp.pi / (2 * zz)) * mp.hankel1(n + mp.mpf(1) / 2, zz))
    # h_n is taken from the half-integer-order Hankel function: forming
    # j_n + i y_n cancels catastrophically when Im z is large.
    j = sps.spherical_jn(n, z)
    h = np.sqrt(np.pi / (2 * z)) * sps.hankel1(n + 0.5, z)
    assert abs(j - jref) <= 1e-12 * max(1.0, abs(jref))
    assert abs(h - href) <= 1e-12 * max(1.0, abs(href))


def test_graf_addition_complex():
    """H_0(kappa r_xy) = sum_n H_n(kappa r_x) e^{in phi_x} J_n(kappa r_y) e^{-in phi_y}
    for complex points with |r_y e^{+-i alpha}| < |r_x| (Thm 3.2.1, Lemma 4.1.1)."""
    kap = 3.0
    x = np.array([2.0 + 0.5j, 1.0 + 0.2j])
    y = np.array([0.3 + 0.1j, -0.2 + 0.05j])

    def pol(d):
        z, e = d[0] + 1j * d[1], d[0] - 1j * d[1]
        r = np.sqrt(z * e)
        return r, z / r, e / r

    rx, ex, _ = pol(x)
    ry, _, ey = pol(y)
    d = x - y
    rxy = np.sqrt(np.sum(d * d))
    n = np.arange(-60, 61)
    ang_x = np.where(n >= 0, ex ** np.abs(n), (1 / ex) ** np.abs(n))
    ang_y = np.where(n >= 0, ey ** np.abs(n), (1 / ey) ** np.abs(n))
    s = np.sum(sps.hankel1(n, kap * rx) * ang_x * sps.jv(n, kap * ry) * ang_y)
    ref = complex(mp.hankel1(0, mp.mpc(kap * rxy.real, kap * rxy.imag)))
    assert abs(s - ref) < 1e-12


def test_legendre_bound_complex_angle():
    """|P_n(cos a)| <= max |e^{+-ina}| for complex a (Eq. lege_bound)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        a = rng.uniform(0, np.pi) + 1j * rng.uniform(-1, 1)
        for n in range(0, 30):
            p = complex(mp.legendre(n, mp.cos(mp.mpc(a.real, a.imag))))
            bound = max(abs(np.exp(1j * n * a)), abs(np.exp(-1j * n * a)))
            assert abs(p) <= bound * (1 + 1e-12)
