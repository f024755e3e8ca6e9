"""Plain CPU 3D complex-coordinate Helmholtz FMM (single and double layer).

Test infrastructure (oracle): only the tests, the smoke check and the CPU
baseline of the benchmark use it. Follows Sec. 5.3 of the paper (Thms 5.3.1
and 5.3.2 for the expansions, "Translation operators" for M2M/M2L/L2L) and
the eight steps of Sec. 6.4 through the shared driver ``oracle.fmm3d.fmm3d``.

Notation. x is a complex 3-vector, x+ = x1 + i x2, x- = x1 - i x2,
rho^2 = x.x (bilinear, Def. 3.2), rho the principal root. Angles are never
formed. The spherical harmonics of Sec. 3.2 (Schmidt semi-normalised,
Y_n^m = sqrt((n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i m phi}, up to the sign
eps_m) enter through the homogeneous polynomials Z_n^m(x) = rho^n Y_n^m,
computed by their normalised three-term recurrences in x+, x-, x3 and rho^2:
  Z_0^0 = 1,  Z_m^m = -x+ sqrt((2m-1)/(2m)) Z_{m-1}^{m-1},
  Z_{m+1}^m = sqrt(2m+1) x3 Z_m^m,
  Z_n^m = (2n-1) x3 Z_{n-1}^m / sqrt((n-m)(n+m))
          - rho^2 Z_{n-2}^m sqrt((n-m-1)(n+m-1)/((n-m)(n+m))),
and Z_n^{-m} = Z_n^m with x+ and x- exchanged. With these,
sum_m Y_n^m(x) Y_n^{-m}(y) = P_n(x.y / (rho_x rho_y)) (Eq. sphaddition,
pinned in tests/test_oracle_helm3d.py). Gradients (pinned by finite
differences), with d+ = d/dx+, d- = d/dx-, n.grad = nu+ d+ + nu- d- + n3 d3:
  d3 Z_n^m = sqrt((n-m)(n+m)) Z_{n-1}^m,
  d+ Z_n^m = -s+ sqrt((n+m)(n+m-1)) Z_{n-1}^{m-1} / 2,  s+ = 1 (m >= 1), -1 (m <= 0),
  d- Z_n^m =  s- sqrt((n-m)(n-m-1)) Z_{n-1}^{m+1} / 2,  s- = 1 (m >= 0), -1 (m < 0).

Wave functions R_n^m(x) = j_n(kappa rho) Y_n^m (entire) and
S_n^m(x) = h_n(kappa rho) Y_n^m, with h_n = h_n^(1). Gegenbauer's addition
theorem (Eqs. addition_sph_hankel with sphaddition) for the constant-free
kernel e^{i kappa r}/r = i kappa h_0(kappa r) reads
  e^{i kappa |x - y|}/|x - y| = i kappa sum_{n,m} (2n+1) R_n^{-m}(y) S_n^m(x)
for y inside and x outside (in the sense of Thms 5.3.1/5.3.2). Hence
  P2M  M_n^m = i kappa (2n+1) sum_j s_j R_n^{-m}(y_j - c)   M2P u = sum M_n^m S_n^m(x - c)
  P2L  L_n^m = i kappa (2n+1) sum_j s_j S_n^{-m}(y_j - c)   L2P u = sum L_n^m R_n^m(x - c)
(the paper's M_n^m and L_n^m without the i kappa of the constant-free
kernel; its (-1)^n in the local coefficients is Y_n^m(-x) = (-1)^n Y_n^m(x)).
Double layer: the source-side wave function is differentiated along the
normal, grad(f_n(kappa rho) rho^-n Z) = f_n rho^-n grad Z
- kappa f_{n+1}(kappa rho) rho^-(n+1) Z x for f = j, h.

Translations ("point and shoot", Sec. 5.3 translation operators with the
rotations of Sec. 5.2): for a shift d = c_new - c_old,
  1. rotate about z: s = sqrt(d1^2 + d2^2), e^{i beta} = (d1 + i d2)/s, the
     frame x' = R_z(-beta) x carries d to (s, 0, d3); coefficients are
     multiplied by e^{i m beta}. If s^2 = 0 (a shift along z) then beta = 0;
  2. rotate about y by alpha, cos alpha = d3/t, sin alpha = s/t,
     t = sqrt(d.d): d goes to (0, 0, t). The rotated coefficients are
     computed by projection (Eq. mp_y_rot): the order-n part F_n and its
     theta-derivative G_n are sampled at the 2P+1 equator points
     phi_j = 2 pi j/(2P+1) of the new frame and Fourier-projected; since
     Y_n^m(pi/2, phi) = a_n^m e^{i m phi} and d_theta Y_n^m = b_n^m e^{i m phi}
     with exactly one of a, b non-zero, c~ = (a F^ + b G^)/(a^2 + b^2);
  3. shift along z by projection (Eq. helm3d_M2L_z_axis): the old expansion
     and its radial derivative are sampled at rho_s u_j around the new
     centre, u_j = (sqrt(1 - x_j^2), 0, x_j), x_j the N_quad = floor(2.5 P)
     Gauss-Legendre nodes, separately for each m, and projected onto
     w_n(kappa rho_s) Y_n^m(u_j) (w = j for local, h for multipole
     results) with the weight pair (conj w_n, kappa conj w_n'), which equals
     the paper's (j_n, kappa j_n') for real j_n and never divides by zero;
  4. undo step 2 (projection) and step 1 (diagonal).
Sampling radius rho_s (the paper leaves it open): the radius sqrt(3)/2 w of the box the
result is centred on (target box for M2L and L2L, parent box for M2M).
"""
from __future__ import annotations

import functools
import math

import numpy as np
import scipy.special as sps

from . import tree as tr
from .direct import HELMHOLTZ


def idx(n, m):
    return n * n + n + m


def _pm(x):
    x = np.asarray(x, complex)
    return x[..., 0] + 1j * x[..., 1], x[..., 0] - 1j * x[..., 1], x[..., 2]


def ylm(P, x):
    """Z_n^m(x) = rho^n Y_n^m for n <= P, stacked by idx(n, m); x complex [..., 3]."""
    xp, xm, z = _pm(x)
    r2 = xp * xm + z * z
    out = np.zeros(((P + 1) ** 2,) + z.shape, complex)
    for sgn, xs in ((1, xp), (-1, xm)):
        diag = np.ones_like(z)
        for m in range(P + 1):
            if m > 0:
                diag = -xs * math.sqrt((2 * m - 1) / (2 * m)) * diag
            if sgn < 0 and m == 0:
                continue
            mm = sgn * m
            out[idx(m, mm)] = diag
            if m + 1 > P:
                continue
            p2, p1 = diag, math.sqrt(2 * m + 1) * z * diag
            out[idx(m + 1, mm)] = p1
            for n in range(m + 2, P + 1):
                a = (2 * n - 1) / math.sqrt((n - m) * (n + m))
                b = math.sqrt((n - m - 1) * (n + m - 1) / ((n - m) * (n + m)))
                cur = a * z * p1 - b * r2 * p2
                out[idx(n, mm)] = cur
                p2, p1 = p1, cur
    return out


def ylm_dir(P, x, v, Z=None):
    """v . grad Z_n^m(x) for n <= P (v complex [..., 3], broadcast with x)."""
    if Z is None:
        Z = ylm(P, x)
    v = np.asarray(v, complex)
    vp, vm, v3 = v[..., 0] + 1j * v[..., 1], v[..., 0] - 1j * v[..., 1], v[..., 2]
    out = np.zeros_like(Z)
    for n in range(1, P + 1):
        for m in range(-n, n + 1):
            acc = 0.0
            if abs(m) <= n - 1:
                acc = acc + v3 * math.sqrt((n - m) * (n + m)) * Z[idx(n - 1, m)]
            if abs(m - 1) <= n - 1:
                sp = 1.0 if m >= 1 else -1.0
                acc = acc - vp * (0.5 * sp * math.sqrt((n + m) * (n + m - 1))) * Z[idx(n - 1, m - 1)]
            if abs(m + 1) <= n - 1:
                sm = 1.0 if m >= 0 else -1.0
                acc = acc + vm * (0.5 * sm * math.sqrt((n - m) * (n - m - 1))) * Z[idx(n - 1, m + 1)]
            out[idx(n, m)] = acc
    return out


def sph_j(N, z):
    """j_n(z), n = 0..N, complex z [...] -> [N+1, ...] (scipy, AMOS)."""
    z = np.asarray(z, complex)
    n = np.arange(N + 1).reshape((-1,) + (1,) * z.ndim)
    return sps.spherical_jn(n, z[None])


def sph_h(N, z):
    """h_n^(1)(z) = sqrt(pi/(2z)) H^(1)_{n+1/2}(z), n = 0..N -> [N+1, ...]."""
    z = np.asarray(z, complex)
    n = np.arange(N + 1).reshape((-1,) + (1,) * z.ndim)
    return np.sqrt(np.pi / (2 * z))[None] * sps.hankel1(n + 0.5, z[None])


def _radial(kind, N, kappa, rho):
    """f_n(kappa rho) / rho^n for n = 0..N+1 (f = j or h); rho = 0 takes the
    limit kappa^n/(2n+1)!! of the regular kind."""
    rho = np.asarray(rho, complex)
    zero = rho == 0
    r = np.where(zero, 1.0, rho)
    f = sph_j(N + 1, kappa * r) if kind == "j" else sph_h(N + 1, kappa * r)
    n = np.arange(N + 2).reshape((-1,) + (1,) * rho.ndim)
    out = f / r[None] ** n
    if np.any(zero):
        if kind != "j":
            raise ValueError("outgoing wave at its centre")
        lim = np.array([kappa ** k / sps.factorial2(2 * k + 1) for k in range(N + 2)])
        out = np.where(zero[None], lim.reshape((-1,) + (1,) * rho.ndim), out)
    return out


def wave(kind, P, kappa, x):
    """R_n^m(x) (kind 'j') or S_n^m(x) (kind 'h'), n <= P -> [(P+1)^2, ...]."""
    x = np.asarray(x, complex)
    rho = np.sqrt(np.sum(x * x, axis=-1))
    F = _radial(kind, P, kappa, rho)
    Z = ylm(P, x)
    out = np.empty_like(Z)
    for n in range(P + 1):
        out[n * n:(n + 1) ** 2] = F[n][None] * Z[n * n:(n + 1) ** 2]
    return out


def wave_dir(kind, P, kappa, x, v):
    """v . grad of R_n^m or S_n^m at x (v broadcast with x)."""
    x = np.asarray(x, complex)
    v = np.broadcast_to(np.asarray(v, complex), x.shape)
    rho = np.sqrt(np.sum(x * x, axis=-1))
    F = _radial(kind, P, kappa, rho)
    Z = ylm(P, x)
    dZ = ylm_dir(P, x, v, Z)
    xv = np.sum(x * v, axis=-1)
    out = np.empty_like(Z)
    for n in range(P + 1):
        # grad(f_n rho^-n Z) = f_n rho^-n grad Z - kappa f_{n+1} rho^-(n+1) Z x
        sl = slice(n * n, (n + 1) ** 2)
        out[sl] = F[n][None] * dZ[sl] - kappa * (F[n + 1] * xv)[None] * Z[sl]
    return out


@functools.lru_cache(maxsize=None)
def gauss_legendre(nq):
    x, w = np.polynomial.legendre.leggauss(nq)
    return x, w


@functools.lru_cache(maxsize=None)
def equator_ab(P):
    """a_n^m = Y_n^m(e_x) and b_n^m = d_theta Y_n^m at theta = pi/2, phi = 0."""
    e = np.array([1.0 + 0j, 0.0, 0.0])
    Z = ylm(P, e)
    b = np.zeros((P + 1) ** 2)
    for n in range(1, P + 1):
        for m in range(-n + 1, n):
            b[idx(n, m)] = -math.sqrt((n - m) * (n + m)) * Z[idx(n - 1, m)].real
    return Z.real.copy(), b


def rotate_proj(c, P, Q):
    """Coefficients in the frames x' = Q_b x (Q_b complex orthogonal) by projection.

    c: [B, ..., (P+1)^2], Q: [B, 3, 3]; for each b,
    sum_m c_n^m Y_n^m(x) = sum_m c~_n^m Y_n^m(Q_b x).
    """
    c = np.asarray(c, complex)
    Q = np.asarray(Q, complex)
    nphi = 2 * P + 1
    phi = 2 * np.pi * np.arange(nphi) / nphi
    e = np.stack([np.cos(phi), np.sin(phi), np.zeros(nphi)], axis=-1)
    pts = np.einsum("ji,bik->bjk", e, Q)          # Q_b^T e_j, [B, nphi, 3]
    v = -Q[:, 2, :]                                # Q_b^T e_theta at theta = pi/2
    Z = ylm(P, pts)                                # [(P+1)^2, B, nphi]
    dZ = ylm_dir(P, pts, v[:, None, :], Z)
    a, b = equator_ab(P)
    out = np.zeros_like(c)
    for n in range(P + 1):
        sl = slice(n * n, (n + 1) ** 2)
        F = np.einsum("b...k,kbj->b...j", c[..., sl], Z[sl])
        G = np.einsum("b...k,kbj->b...j", c[..., sl], dZ[sl])
        ms = np.arange(-n, n + 1)
        E = np.exp(-1j * np.outer(phi, ms)) / nphi     # [nphi, 2n+1]
        Fh, Gh = F @ E, G @ E
        an, bn = a[sl], b[sl]
        out[..., sl] = (an * Fh + bn * Gh) / (an * an + bn * bn)
    return out


def zshift(c, P_in, P_out, t, rho_s, kappa, kind_in, kind_out):
    """Re-expand about (0, 0, t_b) by projection on a Gauss-Legendre meridian.

    c: [B, ..., (P_in+1)^2] coefficients of wave functions kind_in ('h' or
    'j') centred at the origin; t: [B]. Returns [B, ..., (P_out+1)^2] of
    kind_out centred at (0, 0, t_b), sampled on the sphere of radius rho_s
    about the new centre.
    """
    c = np.asarray(c, complex)
    t = np.asarray(t, complex).reshape(-1)
    Pm = max(P_in, P_out)
    nq = max(int(math.floor(2.5 * Pm)), Pm + 1)
    xq, wq = gauss_legendre(nq)
    u = np.stack([np.sqrt(1.0 - xq * xq), np.zeros(nq), xq], axis=-1)
    y = (u * rho_s)[None].astype(complex) + np.einsum("b,k->bk", t, [0.0, 0.0, 1.0])[:, None, :]
    ub = np.broadcast_to(u, y.shape)
    W = wave(kind_in, P_in, kappa, y)              # [(P_in+1)^2, B, nq]
    dW = wave_dir(kind_in, P_in, kappa, y, ub)
    Zo = ylm(P_out, u.astype(complex)).real         # Y_n^m(u_j) on the real meridian
    z = kappa * rho_s
    nn = np.arange(P_out + 1)
    if kind_out == "j":
        fo = sps.spherical_jn(nn, z)
        fo1 = sps.spherical_jn(nn, z, derivative=True)
    else:
        hh = sph_h(P_out + 1, np.array(z))
        fo = hh[:P_out + 1]
        fo1 = nn / z * hh[:P_out + 1] - hh[1:P_out + 2]
    out = np.zeros(c.shape[:-1] + ((P_out + 1) ** 2,), complex)
    for m in range(-Pm, Pm + 1):
        ni = list(range(abs(m), P_in + 1))
        no = list(range(abs(m), P_out + 1))
        if not ni or not no:
            continue
        ii = [idx(n, m) for n in ni]
        ko = [idx(n, m) for n in no]
        f = np.einsum("b...k,kbj->b...j", c[..., ii], W[ii])     # [B, ..., nq]
        g = np.einsum("b...k,kbj->b...j", c[..., ii], dW[ii])
        A = (wq[None, :] * Zo[ko]).T                               # [nq, len(no)]
        wn = fo[no]
        wd = kappa * fo1[no]
        den = (2.0 / (2 * np.array(no) + 1)) * (np.abs(wn) ** 2 + np.abs(wd) ** 2)
        out[..., ko] = (np.conj(wn) * (f @ A) + np.conj(wd) * (g @ A)) / den
    return out


@functools.lru_cache(maxsize=None)
def gaunt_coax(P_in, P_out):
    """C^m[n - m, n' - m, l] for m = 0..min(P_in, P_out) (dense, zero where unused):
    T^m_{n n'}(t) = sum_l C^m[n, n', l] f_l(kappa t), with
    C = (2n+1)(2l+1)(-1)^((n+l-n')/2) G(n, l, n'; m),
    G = (1/2) int_{-1}^{1} Ybar_n^m(x) P_l(x) Ybar_{n'}^m(x) dx
    (Ybar_n^m(cos theta) = Y_n^m at phi = 0), from the plane-wave expansion
    e^{i kappa k.x} = sum (2n+1) i^n R_n^m(x) Y_n^{-m}(k) integrated against
    Y_{n'}^m(k): R_{n'}^m(x + t e3) = sum_n T^m_{n n'} R_n^m(x) with f = j;
    the same coefficients with f = h give S_{n'}^m(x + t e3) = sum_n T R_n^m(x)
    (|x| < |t|), and with f = j they also give S -> S (|x| > |t|).
    """
    L = P_in + P_out
    nq = L + 2
    xq, wq = np.polynomial.legendre.leggauss(nq)
    u = np.stack([np.sqrt(1.0 - xq * xq), np.zeros(nq), xq], axis=-1).astype(complex)
    Yb = ylm(max(P_in, P_out, L), u).real
    out = []
    for m in range(min(P_in, P_out) + 1):
        C = np.zeros((P_out + 1 - m, P_in + 1 - m, L + 1))
        for n in range(m, P_out + 1):
            for n2 in range(m, P_in + 1):
                for l in range(abs(n - n2), n + n2 + 1, 2):
                    G = 0.5 * np.sum(wq * Yb[idx(n, m)] * Yb[idx(l, 0)] * Yb[idx(n2, m)])
                    C[n - m, n2 - m, l] = (2 * n + 1) * (2 * l + 1) * (-1) ** ((n + l - n2) // 2) * G
        out.append(C)
    return out


def zshift_exact(c, P_in, P_out, t, kappa, kind_in, kind_out):
    """The exact coaxial re-expansion that ``zshift`` approximates by projection.

    c: [B, ..., (P_in+1)^2]; t: [B]. Uses T^m = T^{-m} (reflection x2 -> -x2).
    """
    c = np.asarray(c, complex)
    t = np.asarray(t, complex).reshape(-1)
    if kind_in == "j" and kind_out == "h":
        raise ValueError("a local expansion has no multipole re-expansion")
    fk = "h" if (kind_in == "h" and kind_out == "j") else "j"
    L = P_in + P_out
    f = sph_h(L, kappa * t) if fk == "h" else sph_j(L, kappa * t)      # [L+1, B]
    C = gaunt_coax(P_in, P_out)
    out = np.zeros(c.shape[:-1] + ((P_out + 1) ** 2,), complex)
    for m in range(min(P_in, P_out) + 1):
        T = np.einsum("abl,lq->qab", C[m], f)                         # [B, n, n']
        for sg in ((1, -1) if m > 0 else (1,)):
            mm = sg * m
            ii = [idx(n, mm) for n in range(m, P_in + 1)]
            oo = [idx(n, mm) for n in range(m, P_out + 1)]
            out[..., oo] = np.einsum("bac,b...c->b...a", T, c[..., ii])
    return out


def _mscale(P, e, sign):
    """Diagonal z-rotation factors e^{i sign m beta} stacked by idx(n, m); e: [B]."""
    ms = np.array([m for n in range(P + 1) for m in range(-n, n + 1)])
    return np.asarray(e, complex)[:, None] ** (sign * ms)[None, :]


DEGENERATE = {"count": 0}
# a shift with |d1^2 + d2^2| <= DEGEN_TOL * sum |d_i|^2 and (d1, d2) != 0 (an
# isotropic complex direction in the xy-plane) is translated in a frame turned
# by a fixed real rotation (see ``translate``)
DEGEN_TOL = 1e-8


def _fixed_frame(d):
    """Frame index k per shift: -1 = none; 0, 1 = the real rotation Q_k with
    Q_0 d = (-d3, d2, d1), Q_1 d = (-d3, -d1, d2) (the rotation of ``translate``
    with e = i^k and alpha = pi/2), chosen for a larger |(Q d)_1^2 + (Q d)_2^2|."""
    s2 = d[:, 0] ** 2 + d[:, 1] ** 2
    nrm2 = np.sum(np.abs(d) ** 2, axis=-1)
    xy = (d[:, 0] != 0) | (d[:, 1] != 0)
    bad = xy & (np.abs(s2) <= DEGEN_TOL * nrm2)
    k = np.where(np.abs(d[:, 2] ** 2 + d[:, 1] ** 2) >= np.abs(d[:, 2] ** 2 + d[:, 0] ** 2), 0, 1)
    return np.where(bad, k, -1)


def _rot_frame(c, P, e, ca, sa, sign):
    """Coefficients in the frame of the rotation x' = R_y(alpha) R_z(-beta) x
    (e = e^{i beta}, ca = cos alpha, sa = sin alpha; sign = +1) or back
    (sign = -1): E(e) then the y-rotation by projection, or the reverse."""
    Ry = np.zeros((e.shape[0], 3, 3), complex)
    Ry[:, 0, 0], Ry[:, 0, 2], Ry[:, 1, 1] = ca, -sa, 1.0
    Ry[:, 2, 0], Ry[:, 2, 2] = sa, ca
    ext = (slice(None),) + (None,) * (c.ndim - 2) + (slice(None),)
    if sign > 0:
        return rotate_proj(c * _mscale(P, e, 1)[ext], P, Ry)
    return rotate_proj(c, P, np.transpose(Ry, (0, 2, 1))) * _mscale(P, e, -1)[ext]


def translate(c, P_in, P_out, d, rho_s, kappa, kind_in, kind_out, coaxial="projection"):
    """Point-and-shoot re-expansion of c_b about c_old + d_b (steps 1-4 above).

    c: [B, ..., (P_in+1)^2], d: complex [B, 3]. coaxial = "projection" (step 3
    as the paper does it) or "exact" (``zshift_exact``).

    Rotation to the z-axis: e = (d1 + i d2)/s, s^2 = d1^2 + d2^2, and
    cos alpha = d3/t, sin alpha = s/t. With s = 0 and d1 = d2 = 0 the shift is
    already on the z-axis (beta = 0). When s^2 is zero or nearly zero while
    (d1, d2) is not (an isotropic complex direction: e and 1/e blow up), the
    expansion is first turned by the fixed real rotation Q_k of ``_fixed_frame``
    and the shift Q_k d is translated in that frame, then the result is turned
    back; in exact arithmetic this is the same operator.
    """
    c = np.asarray(c, complex)
    d = np.asarray(d, complex).reshape(-1, 3)
    fr = _fixed_frame(d)
    DEGENERATE["count"] += int(np.sum(fr >= 0))
    if np.any(fr >= 0):
        # shift in the fixed frame; the expansion turned into it
        dq = d.copy()
        q0, q1 = fr == 0, fr == 1
        dq[q0] = np.stack([-d[q0, 2], d[q0, 1], d[q0, 0]], axis=-1)
        dq[q1] = np.stack([-d[q1, 2], -d[q1, 0], d[q1, 1]], axis=-1)
        sel = fr >= 0
        ek = np.where(fr == 1, 1j, 1.0 + 0j)[sel]
        one, zero = np.ones(ek.shape[0]), np.zeros(ek.shape[0])
        cq = c.copy()
        cq[sel] = _rot_frame(c[sel], P_in, ek, zero, one, 1)
        out = _translate_frame(cq, P_in, P_out, dq, rho_s, kappa, kind_in, kind_out, coaxial)
        out[sel] = _rot_frame(out[sel], P_out, ek, zero, one, -1)
        return out
    return _translate_frame(c, P_in, P_out, d, rho_s, kappa, kind_in, kind_out, coaxial)


def _translate_frame(c, P_in, P_out, d, rho_s, kappa, kind_in, kind_out, coaxial):
    s2 = d[:, 0] ** 2 + d[:, 1] ** 2
    tt = np.sqrt(np.sum(d * d, axis=-1))
    flat = s2 == 0
    s = np.where(flat, 0.0, np.sqrt(s2))
    e = np.where(flat, 1.0 + 0j, (d[:, 0] + 1j * d[:, 1]) / np.where(flat, 1.0, s))
    c2 = _rot_frame(c, P_in, e, d[:, 2] / tt, s / tt, 1)
    if coaxial == "exact":
        c3 = zshift_exact(c2, P_in, P_out, tt, kappa, kind_in, kind_out)
    else:
        c3 = zshift(c2, P_in, P_out, tt, rho_s, kappa, kind_in, kind_out)
    return _rot_frame(c3, P_out, e, d[:, 2] / tt, s / tt, -1)


class Helmholtz3D:
    """3D Helmholtz operators with the call signatures of ``fmm3d.Laplace3D``."""

    kernel = HELMHOLTZ

    def __init__(self, kappa, T, coaxial="projection"):
        self.kappa = float(kappa)
        self.T = T
        self.coaxial = coaxial

    def _src(self, kind, P, d, s, dip):
        nr = s.shape[0] if s is not None else dip[1].shape[0]
        out = np.zeros((nr, (P + 1) ** 2), complex)
        W = wave(kind, P, self.kappa, d)             # [(P+1)^2, np]
        dW = None
        if dip is not None:
            dW = wave_dir(kind, P, self.kappa, d, dip[0])
        for n in range(P + 1):
            pref = 1j * self.kappa * (2 * n + 1)
            for m in range(-n, n + 1):
                if s is not None:
                    out[:, idx(n, m)] += pref * (s @ W[idx(n, -m)])
                if dW is not None:
                    out[:, idx(n, m)] += pref * (dip[1] @ dW[idx(n, -m)])
        return out

    def p2m(self, P, d, s, dip=None):
        return self._src("j", P, d, s, dip)

    def p2l(self, P, d, s, dip=None):
        return self._src("h", P, d, s, dip)

    def m2p(self, P, M, d):
        return M @ wave("h", P, self.kappa, d)

    def l2p(self, P, L, d):
        return L @ wave("j", P, self.kappa, d)

    def m2p_grad(self, P, M, d):
        """target gradient of M2P: [nrhs, 3, ntarg] (wave_dir along the axes)."""
        return np.stack([M @ wave_dir("h", P, self.kappa, d, np.eye(3)[a]) for a in range(3)], axis=1)

    def l2p_grad(self, P, L, d):
        """target gradient of L2P: [nrhs, 3, ntarg]."""
        return np.stack([L @ wave_dir("j", P, self.kappa, d, np.eye(3)[a]) for a in range(3)], axis=1)

    def _radius(self, level):
        return math.sqrt(3.0) * 0.5 * self.T.width(level)

    batched = True

    def m2m(self, Pc, Pp, M, a, level=None):
        """a = c_child - c_parent: the parent expansion is centred at -a from the child's.
        M: [nrhs, K] for one child, or [B, nrhs, K] with a: [B, 3]."""
        return self._tr(M, Pc, Pp, -np.asarray(a), level, "h", "h")

    def m2l(self, P, M, X0, level=None):
        """X0 = c_target - c_source."""
        return self._tr(M, P, P, X0, level, "h", "j")

    def l2l(self, Pp, Pc, L, a, level=None):
        """a = c_child - c_parent."""
        return self._tr(L, Pp, Pc, a, level, "j", "j")

    def _tr(self, c, Pi, Po, d, level, ki, ko):
        c = np.asarray(c, complex)
        d = np.asarray(d, complex)
        if d.ndim == 1:
            return translate(c[None], Pi, Po, d[None], self._radius(level), self.kappa, ki, ko,
                             self.coaxial)[0]
        Pm = max(Pi, Po)
        chunk = max(1, min(64, int(2e7 // ((Pm + 1) ** 2 * (3 * Pm + 2)))))
        out = []
        for s in range(0, d.shape[0], chunk):
            out.append(translate(c[s:s + chunk], Pi, Po, d[s:s + chunk], self._radius(level),
                                 self.kappa, ki, ko, self.coaxial))
        return np.concatenate(out, axis=0)


def expansion_orders(T, kappa, eps):
    """P per level (Sec. 6.3, Eq. nterms_criteria_3d, prefactors dropped, with the
    Helmholtz eps headroom of tree.P_HEADROOM_HELM)."""
    e = eps * tr.P_HEADROOM_HELM
    return [tr.nterms_helmholtz(3, T.k, e, kappa, T.width(l), tr.helm3d_pair)
            for l in range(T.nlevels)]


def apply(geom_re, geom_im, kappa, eps, N_s, k=1, sigma=None, tau=None, nrm_re=None,
          nrm_im=None, P_levels=None, T=None, top_level=0, coaxial="projection"):
    """User-order 3D Helmholtz FMM; sigma/tau complex [nrhs, n] or [n]. Returns (u, T).

    coaxial: "projection" (the paper's z-translation) or "exact" (the
    translation it approximates; the CUDA path computes this one)."""
    from . import fmm3d
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, kappa=kappa, eps=eps, helmholtz=True,
                          top_level=top_level)
    if P_levels is None:
        P_levels = expansion_orders(T, kappa, eps)
    return fmm3d.apply(geom_re, geom_im, eps, N_s, k=k, sigma=sigma, tau=tau, nrm_re=nrm_re,
                       nrm_im=nrm_im, P_levels=P_levels, T=T, ops=Helmholtz3D(kappa, T, coaxial))


def apply_grad(geom_re, geom_im, kappa, eps, N_s, k=1, sigma=None, tau=None, nrm_re=None,
               nrm_im=None, P_levels=None, T=None, top_level=0, coaxial="projection"):
    """As ``apply``, also returning the target gradient: (u, g, T)."""
    from . import fmm3d
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, kappa=kappa, eps=eps, helmholtz=True,
                          top_level=top_level)
    if P_levels is None:
        P_levels = expansion_orders(T, kappa, eps)
    return fmm3d.apply_grad(geom_re, geom_im, eps, N_s, k=k, sigma=sigma, tau=tau, nrm_re=nrm_re,
                            nrm_im=nrm_im, P_levels=P_levels, T=T, ops=Helmholtz3D(kappa, T, coaxial))
