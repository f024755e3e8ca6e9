"""Plain CPU 2D complex-coordinate FMM (Laplace and Helmholtz, SLP + DLP).

Test infrastructure (oracle). The eight steps of Sec. 6.4 in the paper's
order, over the tree and lists of ``oracle.tree``.

Notation. For a complex displacement d = (d1, d2) in C^2 put
zeta = d1 + i d2 and eta = d1 - i d2, so r^2 = zeta*eta, e^{i phi} = zeta/r
and e^{-i phi} = eta/r (Def. 3.1). Then r^n e^{i n phi} = zeta^n and
r^n e^{-i n phi} = eta^n, and angles are never formed.

2D Laplace (Sec. 4.2, Eqs. lap2d_mp_coef, lap2d_loc_coef, M2M_lap2d,
M2L_lap2d, L2L_lap2d) in these variables:
  multipole  u = M0 log r + sum_n Mp_n eta^-n + sum_n Mm_n zeta^-n,
             Mp_n = -(1/2n) sum eta_j^n s_j,  Mm_n = -(1/2n) sum zeta_j^n s_j;
  local      u = L0 + sum_n Lp_n zeta^n + sum_n Lm_n eta^n,
             Lp_n = -(1/2n) sum zeta_j^-n s_j, Lm_n = -(1/2n) sum eta_j^-n s_j;
  M2M/M2L/L2L are the binomial re-expansions of Lemma 4.2.4, applied in zeta
  and eta separately. The M0 term of M2L carries a factor 1/k, derived from
  log(1 - z) = -sum z^k/k (the printed Eq. M2L_lap2d omits it).

2D Helmholtz (Sec. 4.3): with G_n(d) = J_n(kappa r) e^{i n phi} and
S_n(d) = H_n^(1)(kappa r) e^{i n phi}, Graf's theorem (Thm 3.2.1) gives
G_n(u+v) = sum_m G_{n-m}(u) G_m(v) and S_n(u+v) = sum_m S_{n-m}(u) G_m(v)
(|v| small). Hence, for expansions about c re-centred at c':
  P2M  M_n = sum_j G_{-n}(c - y_j) s_j          (paper: J_n(k r_y) e^{-in phi_y})
  M2P  u(x) = sum_n M_n S_n(x - c)
  M2M  M'_m = sum_n G_{n-m}(c' - c) M_n
  M2L  L_j  = sum_n S_{n-j}(c' - c) M_n
  L2L  L'_m = sum_n G_{n-m}(c' - c) L_n
  P2L  L_j  = sum_i S_{-j}(c' - y_i) s_i
  L2P  u(x) = sum_n L_n G_n(x - c')
These are Eqs. M2M_helm2d, M2L_helm2d, L2L_helm2d derived from the addition
theorems rather than transcribed (the printed index conventions mix n and m).

Double layer: every source-side formula is differentiated along the
caller's normal, n . grad_y = nu d/dzeta_y + nut d/deta_y with nu = n1 + i n2,
nut = n1 - i n2, using d/dzeta G_n = (kappa/2) G_{n-1} and
d/deta G_n = -(kappa/2) G_{n+1} (same for S).
"""
from __future__ import annotations

import numpy as np
import scipy.special as sps

from . import tree as tr
from .direct import kernel_pair, kernel_pair_grad, LAPLACE, HELMHOLTZ


def _zeta_eta(d):
    return d[..., 0] + 1j * d[..., 1], d[..., 0] - 1j * d[..., 1]


def _r(zeta, eta):
    return np.sqrt(zeta * eta)


def cyl_seq(kind, nmin, nmax, kappa, d):
    """G_n(d) (kind='J') or S_n(d) (kind='H') for n = nmin..nmax.

    d: complex [m, 2]. Returns [m, nmax-nmin+1]. Uses scipy's Bessel/Hankel
    functions of complex argument and (zeta/r)^n, (eta/r)^n for the angle.
    """
    zeta, eta = _zeta_eta(np.atleast_2d(d))
    r = _r(zeta, eta)
    n = np.arange(nmin, nmax + 1)
    zero = (r == 0)
    rs = np.where(zero, 1.0, r)
    z = kappa * rs
    if kind == "J":
        f = sps.jv(n[None, :], z[:, None])
    else:
        f = sps.hankel1(n[None, :], z[:, None])
    ez = (zeta / rs)[:, None]
    ee = (eta / rs)[:, None]
    ang = np.where(n[None, :] >= 0, ez ** np.abs(n)[None, :], ee ** np.abs(n)[None, :])
    out = f * ang
    if kind == "J" and np.any(zero):
        out[zero, :] = (n == 0).astype(float)[None, :]
    return out


class Expansions2D:
    """Per-level expansion orders and the operator set for one 2D kernel."""

    def __init__(self, kernel, kappa, P_levels):
        self.kernel = kernel
        self.kappa = kappa
        self.P = P_levels

    # ---- Laplace pieces ------------------------------------------------
    def lap_p2m(self, P, d, s, dip=None):
        """d = y - c [m,2]; s [nrhs,m]; dip = (nu, nut, tau) or None. -> [nrhs, 2P+1]."""
        zeta, eta = _zeta_eta(d)
        out = np.zeros((s.shape[0] if s is not None else dip[2].shape[0], 2 * P + 1), complex)
        n = np.arange(1, P + 1)
        if s is not None:
            out[:, 0] += s.sum(axis=1)
            out[:, 1:P + 1] += -(1.0 / (2 * n))[None, :] * (s @ (eta[:, None] ** n[None, :]))
            out[:, P + 1:] += -(1.0 / (2 * n))[None, :] * (s @ (zeta[:, None] ** n[None, :]))
        if dip is not None:
            nu, nut, tau = dip
            out[:, 1:P + 1] += -0.5 * ((tau * nut[None, :]) @ (eta[:, None] ** (n - 1)[None, :]))
            out[:, P + 1:] += -0.5 * ((tau * nu[None, :]) @ (zeta[:, None] ** (n - 1)[None, :]))
        return out

    def lap_m2p(self, P, M, d):
        zeta, eta = _zeta_eta(d)
        n = np.arange(1, P + 1)
        u = M[:, :1] * (0.5 * np.log(zeta * eta))[None, :]
        u = u + M[:, 1:P + 1] @ (eta[:, None] ** (-n)[None, :]).T
        u = u + M[:, P + 1:] @ (zeta[:, None] ** (-n)[None, :]).T
        return u

    def lap_p2l(self, P, d, s, dip=None):
        """d = y - c (source relative to the local centre)."""
        zeta, eta = _zeta_eta(d)
        nr = s.shape[0] if s is not None else dip[2].shape[0]
        out = np.zeros((nr, 2 * P + 1), complex)
        n = np.arange(1, P + 1)
        if s is not None:
            out[:, 0] += s @ (0.5 * np.log(zeta * eta))
            out[:, 1:P + 1] += -(1.0 / (2 * n))[None, :] * (s @ (zeta[:, None] ** (-n)[None, :]))
            out[:, P + 1:] += -(1.0 / (2 * n))[None, :] * (s @ (eta[:, None] ** (-n)[None, :]))
        if dip is not None:
            nu, nut, tau = dip
            out[:, 0] += tau @ (0.5 * (nu / zeta + nut / eta))
            out[:, 1:P + 1] += 0.5 * ((tau * nu[None, :]) @ (zeta[:, None] ** (-n - 1)[None, :]))
            out[:, P + 1:] += 0.5 * ((tau * nut[None, :]) @ (eta[:, None] ** (-n - 1)[None, :]))
        return out

    def lap_l2p(self, P, L, d):
        zeta, eta = _zeta_eta(d)
        n = np.arange(1, P + 1)
        u = L[:, :1] + L[:, 1:P + 1] @ (zeta[:, None] ** n[None, :]).T
        u = u + L[:, P + 1:] @ (eta[:, None] ** n[None, :]).T
        return u

    @staticmethod
    def _binom(a, b):
        return sps.comb(a, b, exact=False)

    def lap_m2m(self, Pc, Pp, M, a):
        """a = c_child - c_parent (original centre relative to the new one)."""
        z0, e0 = a[0] + 1j * a[1], a[0] - 1j * a[1]
        out = np.zeros((M.shape[0], 2 * Pp + 1), complex)
        out[:, 0] = M[:, 0]
        for k in range(1, Pp + 1):
            out[:, k] += -(1.0 / (2 * k)) * e0 ** k * M[:, 0]
            out[:, Pp + k] += -(1.0 / (2 * k)) * z0 ** k * M[:, 0]
            for n in range(1, min(k, Pc) + 1):
                c = self._binom(k - 1, k - n)
                out[:, k] += c * e0 ** (k - n) * M[:, n]
                out[:, Pp + k] += c * z0 ** (k - n) * M[:, Pc + n]
        return out

    def lap_m2l(self, P, M, a):
        """a = c_source - c_target."""
        z0, e0 = a[0] + 1j * a[1], a[0] - 1j * a[1]
        out = np.zeros_like(M)
        out[:, 0] = M[:, 0] * 0.5 * np.log(z0 * e0)
        for n in range(1, P + 1):
            out[:, 0] += (-1) ** n * e0 ** (-n) * M[:, n] + (-1) ** n * z0 ** (-n) * M[:, P + n]
        for k in range(1, P + 1):
            out[:, k] += -(1.0 / (2 * k)) * z0 ** (-k) * M[:, 0]
            out[:, P + k] += -(1.0 / (2 * k)) * e0 ** (-k) * M[:, 0]
            for n in range(1, P + 1):
                c = (-1) ** n * self._binom(n + k - 1, k)
                out[:, k] += c * z0 ** (-(n + k)) * M[:, P + n]
                out[:, P + k] += c * e0 ** (-(n + k)) * M[:, n]
        return out

    def lap_l2l(self, Pp, Pc, L, a):
        """a = c_parent - c_child."""
        z0, e0 = a[0] + 1j * a[1], a[0] - 1j * a[1]
        out = np.zeros((L.shape[0], 2 * Pc + 1), complex)
        out[:, 0] = L[:, 0]
        for n in range(1, Pp + 1):
            out[:, 0] += (-z0) ** n * L[:, n] + (-e0) ** n * L[:, Pp + n]
        for k in range(1, Pc + 1):
            for n in range(k, Pp + 1):
                c = self._binom(n, k)
                out[:, k] += c * (-z0) ** (n - k) * L[:, n]
                out[:, Pc + k] += c * (-e0) ** (n - k) * L[:, Pp + n]
        return out

    # ---- Helmholtz pieces ------------------------------------------------
    def hel_p2m(self, P, c, y, s, dip=None):
        """M_n = sum G_{-n}(c - y) s (+ dipole), n=-P..P."""
        d = c[None, :] - y
        kap = self.kappa
        G = cyl_seq("J", -P - 1, P + 1, kap, d)        # G_m, m=-P-1..P+1 (index m+P+1)
        idx = P + 1 - np.arange(-P, P + 1)             # G_{-n}
        nr = s.shape[0] if s is not None else dip[2].shape[0]
        out = np.zeros((nr, 2 * P + 1), complex)
        if s is not None:
            out += s @ G[:, idx]
        if dip is not None:
            nu, nut, tau = dip
            # n.grad_y G_{-n}(c-y) = -(kappa/2)(nu G_{-n-1} - nut G_{-n+1})(c-y)
            term = -(kap / 2.0) * (nu[:, None] * G[:, idx - 1] - nut[:, None] * G[:, idx + 1])
            out += tau @ term
        return out

    def hel_m2p(self, P, M, c, x):
        S = cyl_seq("H", -P, P, self.kappa, x - c[None, :])
        return M @ S.T

    def hel_p2l(self, P, c, y, s, dip=None):
        d = c[None, :] - y
        kap = self.kappa
        S = cyl_seq("H", -P - 1, P + 1, kap, d)
        idx = P + 1 - np.arange(-P, P + 1)             # S_{-j}
        nr = s.shape[0] if s is not None else dip[2].shape[0]
        out = np.zeros((nr, 2 * P + 1), complex)
        if s is not None:
            out += s @ S[:, idx]
        if dip is not None:
            nu, nut, tau = dip
            term = -(kap / 2.0) * (nu[:, None] * S[:, idx - 1] - nut[:, None] * S[:, idx + 1])
            out += tau @ term
        return out

    def hel_l2p(self, P, L, c, x):
        G = cyl_seq("J", -P, P, self.kappa, x - c[None, :])
        return L @ G.T

    # ---- target gradients (d/dx1 = d/dzeta + d/deta, d/dx2 = i (d/dzeta - d/deta)) ----

    @staticmethod
    def _grad(dz, de):
        """[nrhs, ntarg] d/dzeta, d/deta -> [nrhs, 2, ntarg] gradient."""
        return np.stack([dz + de, 1j * (dz - de)], axis=1)

    def lap_m2p_grad(self, P, M, d):
        """grad of M0 log r + sum Mp_n eta^-n + sum Mm_n zeta^-n (log r = log(zeta eta)/2)."""
        zeta, eta = _zeta_eta(d)
        n = np.arange(1, P + 1)
        dz = M[:, :1] * (0.5 / zeta)[None, :] - M[:, P + 1:] @ (n[:, None] * zeta[None, :] ** (-n - 1)[:, None])
        de = M[:, :1] * (0.5 / eta)[None, :] - M[:, 1:P + 1] @ (n[:, None] * eta[None, :] ** (-n - 1)[:, None])
        return self._grad(dz, de)

    def lap_l2p_grad(self, P, L, d):
        """grad of L0 + sum Lp_n zeta^n + sum Lm_n eta^n."""
        zeta, eta = _zeta_eta(d)
        n = np.arange(1, P + 1)
        dz = L[:, 1:P + 1] @ (n[:, None] * zeta[None, :] ** (n - 1)[:, None])
        de = L[:, P + 1:] @ (n[:, None] * eta[None, :] ** (n - 1)[:, None])
        return self._grad(dz, de)

    def hel_m2p_grad(self, P, M, c, x):
        """d/dzeta S_n = (kappa/2) S_{n-1}, d/deta S_n = -(kappa/2) S_{n+1}."""
        S = cyl_seq("H", -P - 1, P + 1, self.kappa, x - c[None, :])
        idx = np.arange(-P, P + 1) + P + 1
        dz = (0.5 * self.kappa) * (M @ S[:, idx - 1].T)
        de = (-0.5 * self.kappa) * (M @ S[:, idx + 1].T)
        return self._grad(dz, de)

    def hel_l2p_grad(self, P, L, c, x):
        """d/dzeta G_n = (kappa/2) G_{n-1}, d/deta G_n = -(kappa/2) G_{n+1}."""
        G = cyl_seq("J", -P - 1, P + 1, self.kappa, x - c[None, :])
        idx = np.arange(-P, P + 1) + P + 1
        dz = (0.5 * self.kappa) * (L @ G[:, idx - 1].T)
        de = (-0.5 * self.kappa) * (L @ G[:, idx + 1].T)
        return self._grad(dz, de)

    def hel_shift(self, kind, Pin, Pout, E, a):
        """E'_m = sum_n T_{n-m}(a) E_n, |m|<=Pout, |n|<=Pin; T = G or S."""
        T = cyl_seq(kind, -(Pin + Pout), Pin + Pout, self.kappa, a[None, :])[0]
        n = np.arange(-Pin, Pin + 1)
        m = np.arange(-Pout, Pout + 1)
        mat = T[(n[None, :] - m[:, None]) + (Pin + Pout)]   # [m, n]
        return E @ mat.T


def expansion_orders(T, kernel, kappa, eps):
    """P per level: the Sec. 6.3 criteria with the prefactors dropped and the
    eps headroom factors of tree.P_HEADROOM / P_HEADROOM_HELM."""
    nl = T.nlevels
    if kernel == LAPLACE:
        return [tr.nterms_laplace(2, T.k, eps * tr.P_HEADROOM)] * nl
    e = eps * tr.P_HEADROOM_HELM
    return [tr.nterms_helmholtz(2, T.k, e, kappa, T.width(l), tr.helm2d_pair) for l in range(nl)]


def fmm2d(T, kernel, kappa, eps, pts, sigma=None, tau=None, nrm=None, P_levels=None, grad=False):
    """Apply the 2D complex-coordinate FMM on tree T.

    pts: complex [n, 2] in tree (sorted) order; sigma/tau: complex [nrhs, n]
    sorted; nrm: complex [n, 2] sorted. Returns u: complex [nrhs, n] sorted;
    with grad=True, (u, g) with the target gradient g [nrhs, 2, n] from the
    differentiated evaluation steps (P2P, M2P, L2P; the expansions are the
    same).
    """
    n = pts.shape[0]
    if P_levels is None:
        P_levels = expansion_orders(T, kernel, kappa, eps)
    X = Expansions2D(kernel, kappa, P_levels)
    nr = (sigma if sigma is not None else tau).shape[0]
    u = np.zeros((nr, n), complex)
    g = np.zeros((nr, 2, n), complex) if grad else None
    nb = T.nboxes
    lv = T.box_level
    cen = T.center_re + 1j * T.center_im          # complexified centres, Eq. complexify_center_average
    st, en = T.box_start, T.box_end
    lap = kernel == LAPLACE
    l0 = T.l0
    dipole = tau is not None
    nu = nut = None
    if dipole:
        nu = nrm[:, 0] + 1j * nrm[:, 1]
        nut = nrm[:, 0] - 1j * nrm[:, 1]

    def src(b):
        s, e = st[b], en[b]
        sg = None if sigma is None else sigma[:, s:e]
        dp = None if not dipole else (nu[s:e], nut[s:e], tau[:, s:e])
        return s, e, sg, dp

    M = {}
    Lc = {}
    expand = nb > 1
    # (1) P2M at childless boxes
    for b in range(nb):
        if not expand or lv[b] < l0 or not T.box_leaf[b]:
            continue
        P = P_levels[lv[b]]
        s, e, sg, dp = src(b)
        if lap:
            M[b] = X.lap_p2m(P, pts[s:e] - cen[b][None, :], sg, dp)
        else:
            M[b] = X.hel_p2m(P, cen[b], pts[s:e], sg, dp)
    # (2) M2M, finest level first
    for l in range(T.nlevels - 1, l0 - 1, -1):
        for b in range(T.level_offset[l], T.level_offset[l + 1]):
            if not expand or T.box_leaf[b]:
                continue
            Pp = P_levels[l]
            acc = np.zeros((nr, 2 * Pp + 1), complex)
            for c in range(T.level_offset[l + 1], T.level_offset[l + 2]):
                if T.box_parent[c] != b:
                    continue
                Pc = P_levels[l + 1]
                if lap:
                    acc += X.lap_m2m(Pc, Pp, M[c], cen[c] - cen[b])
                else:
                    acc += X.hel_shift("J", Pc, Pp, M[c], cen[b] - cen[c])
            M[b] = acc
    # (3) P2P over List 1
    for b in range(nb):
        if not T.box_leaf[b]:
            continue
        ts, te = st[b], en[b]
        for a in T.lists["list1"][b] if expand else [b]:
            s, e, sg, dp = src(a)
            d = pts[ts:te, None, :] - pts[None, s:e, :]
            zero = np.all(d == 0, axis=-1)
            dd = np.where(zero[..., None], 1.0, d)
            slp, dlp = kernel_pair(2, kernel, kappa, dd,
                                   None if not dipole else np.broadcast_to(nrm[None, s:e, :], dd.shape))
            if sg is not None:
                u[:, ts:te] += sg @ np.where(zero, 0, slp).T
            if dipole:
                u[:, ts:te] += tau[:, s:e] @ np.where(zero, 0, dlp).T
            if grad:
                gs, gd = kernel_pair_grad(2, kernel, kappa, dd,
                                          None if not dipole else np.broadcast_to(nrm[None, s:e, :], dd.shape))
                if sg is not None:
                    g[:, :, ts:te] += np.einsum("tmk,rm->rkt", np.where(zero[..., None], 0, gs), sg)
                if dipole:
                    g[:, :, ts:te] += np.einsum("tmk,rm->rkt", np.where(zero[..., None], 0, gd), tau[:, s:e])
    if not expand:
        return (u, g) if grad else u
    # (4) M2L over List 2
    for b in range(nb):
        if lv[b] < l0:
            continue
        P = P_levels[lv[b]]
        acc = np.zeros((nr, 2 * P + 1), complex)
        for a in T.lists["list2"][b]:
            if lap:
                acc += X.lap_m2l(P, M[a], cen[a] - cen[b])
            else:
                acc += X.hel_shift("H", P, P, M[a], cen[b] - cen[a])
        Lc[b] = acc
    # (5) M2P over List 3
    for b in range(nb):
        if not T.box_leaf[b] or lv[b] < l0:
            continue
        ts, te = st[b], en[b]
        for a in T.lists["list3"][b]:
            Pa = P_levels[lv[a]]
            if lap:
                u[:, ts:te] += X.lap_m2p(Pa, M[a], pts[ts:te] - cen[a][None, :])
                if grad:
                    g[:, :, ts:te] += X.lap_m2p_grad(Pa, M[a], pts[ts:te] - cen[a][None, :])
            else:
                u[:, ts:te] += X.hel_m2p(Pa, M[a], cen[a], pts[ts:te])
                if grad:
                    g[:, :, ts:te] += X.hel_m2p_grad(Pa, M[a], cen[a], pts[ts:te])
    # (6) P2L over List 4
    for b in range(nb):
        if lv[b] < l0:
            continue
        P = P_levels[lv[b]]
        for a in T.lists["list4"][b]:
            s, e, sg, dp = src(a)
            if lap:
                Lc[b] += X.lap_p2l(P, pts[s:e] - cen[b][None, :], sg, dp)
            else:
                Lc[b] += X.hel_p2l(P, cen[b], pts[s:e], sg, dp)
    # (7) L2L, coarsest level first
    for l in range(l0 + 1, T.nlevels):
        for b in range(T.level_offset[l], T.level_offset[l + 1]):
            p = T.box_parent[b]
            Pp, Pc = P_levels[l - 1], P_levels[l]
            if lap:
                Lc[b] += X.lap_l2l(Pp, Pc, Lc[p], cen[p] - cen[b])
            else:
                Lc[b] += X.hel_shift("J", Pp, Pc, Lc[p], cen[b] - cen[p])
    # (8) L2P at childless boxes
    for b in range(nb):
        if not T.box_leaf[b] or lv[b] < l0:
            continue
        ts, te = st[b], en[b]
        P = P_levels[lv[b]]
        if lap:
            u[:, ts:te] += X.lap_l2p(P, Lc[b], pts[ts:te] - cen[b][None, :])
            if grad:
                g[:, :, ts:te] += X.lap_l2p_grad(P, Lc[b], pts[ts:te] - cen[b][None, :])
        else:
            u[:, ts:te] += X.hel_l2p(P, Lc[b], cen[b], pts[ts:te])
            if grad:
                g[:, :, ts:te] += X.hel_l2p_grad(P, Lc[b], cen[b], pts[ts:te])
    return (u, g) if grad else u


def apply(geom_re, geom_im, kernel, kappa, eps, N_s, k=1, sigma=None, tau=None,
          nrm_re=None, nrm_im=None, P_levels=None, T=None):
    """User-order convenience wrapper: build the tree, run the FMM, un-permute.

    sigma/tau: complex [nrhs, n] or [n] in input order. Returns (u, T).
    """
    pts = np.asarray(geom_re) + 1j * np.asarray(geom_im)
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, kappa=kappa, eps=eps,
                          helmholtz=(kernel == HELMHOLTZ))
    perm = T.perm
    single = False
    def prep(v):
        nonlocal single
        if v is None:
            return None
        v = np.asarray(v, complex)
        if v.ndim == 1:
            single = True
            v = v[None, :]
        return v[:, perm]
    sg, tu = prep(sigma), prep(tau)
    nrm = None
    if tau is not None:
        nrm = (np.asarray(nrm_re) + 1j * np.asarray(nrm_im))[perm]
    u_s = fmm2d(T, kernel, kappa, eps, pts[perm], sg, tu, nrm, P_levels)
    u = np.empty_like(u_s)
    u[:, perm] = u_s
    return (u[0] if single else u), T


def apply_grad(geom_re, geom_im, kernel, kappa, eps, N_s, k=1, sigma=None, tau=None,
               nrm_re=None, nrm_im=None, P_levels=None, T=None):
    """As ``apply``, also returning the target gradient: (u, g, T) with g
    [nrhs, 2, n] (or [2, n]) in input order."""
    pts = np.asarray(geom_re) + 1j * np.asarray(geom_im)
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, kappa=kappa, eps=eps,
                          helmholtz=(kernel == HELMHOLTZ))
    perm = T.perm
    single = (sigma if sigma is not None else tau).ndim == 1
    prep = lambda v: None if v is None else np.atleast_2d(np.asarray(v, complex))[:, perm]
    nrm = None
    if tau is not None:
        nrm = (np.asarray(nrm_re) + 1j * np.asarray(nrm_im))[perm]
    u_s, g_s = fmm2d(T, kernel, kappa, eps, pts[perm], prep(sigma), prep(tau), nrm, P_levels, grad=True)
    u = np.empty_like(u_s)
    u[:, perm] = u_s
    g = np.empty_like(g_s)
    g[:, :, perm] = g_s
    return (u[0], g[0], T) if single else (u, g, T)
