"""Plain CPU 3D complex-coordinate Laplace FMM (SLP + DLP).

Test infrastructure (oracle). The eight steps of Sec. 6.4 over the tree and
lists of ``oracle.tree``, with the 3D Laplace expansions of Sec. 5.2
(Thm 5.2.2 multipole, Thm 5.2.3 local, Eqs. L3dM2M, L3dM2L, L3dL2L).

Notation. For a complex 3-vector x put x+ = x1 + i x2, x- = x1 - i x2,
z = x3 and rho^2 = x+ x- + z^2 (= x.x; no conjugation, Def. 3.2). The
spherical harmonics of Sec. 3.2 enter through the solid harmonics
  regular   U_n^m(x) = rho^n P_n^m(cos theta) e^{i m phi} / (n+m)!
  irregular T_n^m(x) = (n-m)! P_n^m(cos theta) e^{i m phi} / rho^{n+1}
which are polynomial (resp. rational in x and 1/rho) and are computed by
their three-term recurrences in x+, x-, z and rho^2 (entire continuation; no
angle is formed, which avoids the sin(theta) = sqrt(1 - cos^2) branch of
Def. 3.2). For m < 0, U_n^m = (-1)^|m| times the m > 0 value with x+ and x-
exchanged (likewise T). The addition theorem of Lemma 5.2.1 with Eq.
sphaddition then reads
  1/|x - y| = sum_{n,m} (-1)^m U_n^{-m}(y) T_n^m(x),
and the translation theorems behind Eqs. L3dM2M/L3dM2L/L3dL2L are
  U_n^m(a + b) = sum_{k,l} U_k^l(a) U_{n-k}^{m-l}(b),
  T_n^m(x - y) = sum_{k,l} (-1)^l U_k^{-l}(y) T_{n+k}^{m+l}(x).
These were checked numerically at complex points (tests/test_oracle_fmm3d.py)
rather than transcribed: the printed index conventions of Lemma 5.2.4 are
garbled. Expansions:
  P2M  M_n^m = sum_j s_j (-1)^m U_n^{-m}(y_j - c)         M2P  u = sum M_n^m T_n^m(x - c)
  M2M  M_n^m(c) = sum_{k,l} (-1)^l U_k^l(c' - c) M_{n-k}^{m+l}(c')
  M2L  L_k^l = (-1)^{k+l} sum_{n,m} M_n^m T_{n+k}^{m-l}(c_t - c_s)
  L2L  L'_k^l = sum_{n,m} L_n^m U_{n-k}^{m-l}(c' - c)
  P2L  L_k^l = sum_j s_j (-1)^l T_k^{-l}(y_j - c)         L2P  u = sum L_k^l U_k^l(x - c)
Double layer: n . grad_y with n.grad = nu+ d/dx+ + nu- d/dx- + n3 d/dz
(nu+- = n1 +- i n2) and d+ U_n^m = -U_{n-1}^{m-1}/2, d- U_n^m = U_{n-1}^{m+1}/2,
dz U_n^m = U_{n-1}^m; d+ T_n^m = -T_{n+1}^{m-1}/2, d- T_n^m = T_{n+1}^{m+1}/2,
dz T_n^m = -T_{n+1}^m (finite-difference pinned).
"""
from __future__ import annotations

import functools

import numpy as np

from . import tree as tr
from .direct import kernel_pair, kernel_pair_grad, LAPLACE


def idx(n, m):
    return n * n + n + m


def _columns(P, xs, z, r2, first, diag, sub, rec):
    out = np.zeros(((P + 1) ** 2,) + np.shape(z), complex)
    col = None
    for m in range(P + 1):
        col = first if m == 0 else diag(m, xs, col)
        out[idx(m, m)] = col
        if m + 1 <= P:
            prev2, prev1 = col, sub(m, z, col)
            out[idx(m + 1, m)] = prev1
            for n in range(m + 2, P + 1):
                cur = rec(n, m, z, r2, prev1, prev2)
                out[idx(n, m)] = cur
                prev2, prev1 = prev1, cur
    return out


def regular(P, x):
    """U_n^m(x) for n <= P, stacked by idx(n, m); x: complex [..., 3]."""
    x = np.asarray(x, complex)
    xp, xm, z = x[..., 0] + 1j * x[..., 1], x[..., 0] - 1j * x[..., 1], x[..., 2]
    r2 = xp * xm + z * z
    one = np.ones_like(z)
    diag = lambda m, xs, c: -xs / (2 * m) * c
    sub = lambda m, z, c: z * c
    rec = lambda n, m, z, r2, p1, p2: ((2 * n - 1) * z * p1 - r2 * p2) / ((n - m) * (n + m))
    pos = _columns(P, xp, z, r2, one, diag, sub, rec)
    neg = _columns(P, xm, z, r2, one, diag, sub, rec)
    out = pos.copy()
    for n in range(P + 1):
        for m in range(1, n + 1):
            out[idx(n, -m)] = (-1) ** m * neg[idx(n, m)]
    return out


def irregular(P, x):
    """T_n^m(x) for n <= P, stacked by idx(n, m); x: complex [..., 3]."""
    x = np.asarray(x, complex)
    xp, xm, z = x[..., 0] + 1j * x[..., 1], x[..., 0] - 1j * x[..., 1], x[..., 2]
    r2 = xp * xm + z * z
    rho = np.sqrt(r2)
    diag = lambda m, xs, c: -(2 * m - 1) * xs / r2 * c
    sub = lambda m, z, c: (2 * m + 1) * z / r2 * c
    rec = lambda n, m, z, r2, p1, p2: ((2 * n - 1) * z * p1 - ((n - 1) ** 2 - m * m) * p2) / r2
    pos = _columns(P, xp, z, r2, 1.0 / rho, diag, sub, rec)
    neg = _columns(P, xm, z, r2, 1.0 / rho, diag, sub, rec)
    out = pos.copy()
    for n in range(P + 1):
        for m in range(1, n + 1):
            out[idx(n, -m)] = (-1) ** m * neg[idx(n, m)]
    return out


def _get(tab, n, m):
    if n < 0 or abs(m) > n:
        return 0.0
    return tab[idx(n, m)]


def regular_dir(P, x, v):
    """v . grad U_n^m(x), n <= P (d+ U_n^m = -U_{n-1}^{m-1}/2, d- U_n^m = U_{n-1}^{m+1}/2,
    dz U_n^m = U_{n-1}^m with v . grad = v+ d+ + v- d- + v3 dz, v+- = v1 +- i v2)."""
    U = regular(P, x)
    v = np.asarray(v, complex)
    vp, vm, v3 = v[..., 0] + 1j * v[..., 1], v[..., 0] - 1j * v[..., 1], v[..., 2]
    out = np.zeros_like(U)
    for n in range(1, P + 1):
        for m in range(-n, n + 1):
            out[idx(n, m)] = (vp * (-0.5) * _get(U, n - 1, m - 1) + vm * 0.5 * _get(U, n - 1, m + 1)
                              + v3 * _get(U, n - 1, m))
    return out


def irregular_dir(P, x, v):
    """v . grad T_n^m(x), n <= P (d+ T_n^m = -T_{n+1}^{m-1}/2, d- T_n^m = T_{n+1}^{m+1}/2,
    dz T_n^m = -T_{n+1}^m)."""
    T = irregular(P + 1, x)
    v = np.asarray(v, complex)
    vp, vm, v3 = v[..., 0] + 1j * v[..., 1], v[..., 0] - 1j * v[..., 1], v[..., 2]
    out = np.zeros(((P + 1) ** 2,) + T.shape[1:], complex)
    for n in range(P + 1):
        for m in range(-n, n + 1):
            out[idx(n, m)] = (vp * (-0.5) * _get(T, n + 1, m - 1) + vm * 0.5 * _get(T, n + 1, m + 1)
                              - v3 * _get(T, n + 1, m))
    return out


_UNIT = np.eye(3)


class Laplace3D:
    """Operators of the 3D Laplace expansions (coefficients stacked by idx(n, m))."""

    @staticmethod
    def p2m(P, d, s, dip=None):
        """d = y - c [np, 3]; s [nrhs, np]; dip = (nrm [np, 3], tau [nrhs, np])."""
        U = regular(P + 1, d)                       # [(P+2)^2, np]
        nr = s.shape[0] if s is not None else dip[1].shape[0]
        out = np.zeros((nr, (P + 1) ** 2), complex)
        for n in range(P + 1):
            for m in range(-n, n + 1):
                sgn = (-1) ** m
                if s is not None:
                    out[:, idx(n, m)] += sgn * (s @ U[idx(n, -m)])
                if dip is not None:
                    nrm, tau = dip
                    nup, num = nrm[:, 0] + 1j * nrm[:, 1], nrm[:, 0] - 1j * nrm[:, 1]
                    g = (nup * (-0.5) * _get(U, n - 1, -m - 1) + num * 0.5 * _get(U, n - 1, -m + 1)
                         + nrm[:, 2] * _get(U, n - 1, -m))
                    out[:, idx(n, m)] += sgn * (tau @ g)
        return out

    @staticmethod
    def m2p(P, M, d):
        T = irregular(P, d)
        return M @ T

    @staticmethod
    def p2l(P, d, s, dip=None):
        """d = y - c (source relative to the local centre)."""
        T = irregular(P + 1, d)
        nr = s.shape[0] if s is not None else dip[1].shape[0]
        out = np.zeros((nr, (P + 1) ** 2), complex)
        for k in range(P + 1):
            for l in range(-k, k + 1):
                sgn = (-1) ** l
                if s is not None:
                    out[:, idx(k, l)] += sgn * (s @ T[idx(k, -l)])
                if dip is not None:
                    nrm, tau = dip
                    nup, num = nrm[:, 0] + 1j * nrm[:, 1], nrm[:, 0] - 1j * nrm[:, 1]
                    g = (nup * (-0.5) * _get(T, k + 1, -l - 1) + num * 0.5 * _get(T, k + 1, -l + 1)
                         - nrm[:, 2] * _get(T, k + 1, -l))
                    out[:, idx(k, l)] += sgn * (tau @ g)
        return out

    @staticmethod
    def l2p(P, L, d):
        U = regular(P, d)
        return L @ U

    @staticmethod
    def m2p_grad(P, M, d):
        """target gradient of M2P: [nrhs, 3, ntarg]."""
        return np.stack([M @ irregular_dir(P, d, _UNIT[a]) for a in range(3)], axis=1)

    @staticmethod
    def l2p_grad(P, L, d):
        """target gradient of L2P: [nrhs, 3, ntarg]."""
        return np.stack([L @ regular_dir(P, d, _UNIT[a]) for a in range(3)], axis=1)

    kernel = LAPLACE
    kappa = 0.0

    @staticmethod
    def m2m(Pc, Pp, M, a, level=None):
        """a = c_child - c_parent: M_n^m(c) = sum_{k,l} (-1)^l U_k^l(a) M_{n-k}^{m+l}."""
        U = regular(Pp, a[None, :])[:, 0]
        I, S, K = _m2m_index(Pc, Pp)
        mat = np.where(K, S * U[I], 0.0)
        return M @ mat.T

    @staticmethod
    def m2l(P, M, X0, level=None):
        """X0 = c_t - c_s: L_k^l = (-1)^{k+l} sum_{n,m} M_n^m T_{n+k}^{m-l}(X0)."""
        T = irregular(2 * P, X0[None, :])[:, 0]
        I, S = _m2l_index(P)
        return M @ (S * T[I]).T

    @staticmethod
    def l2l(Pp, Pc, L, a, level=None):
        """a = c_child - c_parent: L'_k^l = sum_{n,m} L_n^m U_{n-k}^{m-l}(a)."""
        U = regular(Pp, a[None, :])[:, 0]
        I, K = _l2l_index(Pp, Pc)
        mat = np.where(K, U[I], 0.0)
        return L @ mat.T


def _nm(P):
    return [(n, m) for n in range(P + 1) for m in range(-n, n + 1)]


@functools.lru_cache(maxsize=None)
def _m2m_index(Pc, Pp):
    rows, cols = _nm(Pp), _nm(Pc)
    I = np.zeros((len(rows), len(cols)), int)
    S = np.zeros((len(rows), len(cols)))
    K = np.zeros((len(rows), len(cols)), bool)
    for r, (n, m) in enumerate(rows):
        for c, (n2, m2) in enumerate(cols):
            k, l = n - n2, m2 - m
            if 0 <= k and abs(l) <= k:
                I[r, c], S[r, c], K[r, c] = idx(k, l), (-1) ** l, True
    return I, S, K


@functools.lru_cache(maxsize=None)
def _m2l_index(P):
    nm = _nm(P)
    I = np.zeros((len(nm), len(nm)), int)
    S = np.zeros((len(nm), len(nm)))
    for r, (k, l) in enumerate(nm):
        for c, (n, m) in enumerate(nm):
            I[r, c], S[r, c] = idx(n + k, m - l), (-1) ** (k + l)
    return I, S


@functools.lru_cache(maxsize=None)
def _l2l_index(Pp, Pc):
    rows, cols = _nm(Pc), _nm(Pp)
    I = np.zeros((len(rows), len(cols)), int)
    K = np.zeros((len(rows), len(cols)), bool)
    for r, (k, l) in enumerate(rows):
        for c, (n, m) in enumerate(cols):
            if n >= k and abs(m - l) <= n - k:
                I[r, c], K[r, c] = idx(n - k, m - l), True
    return I, K


def expansion_orders(T, eps):
    return [tr.nterms_laplace(3, T.k, eps * tr.P_HEADROOM)] * T.nlevels


def fmm3d(T, eps, pts, sigma=None, tau=None, nrm=None, P_levels=None, ops=None, grad=False):
    """3D FMM on tree T; pts/sigma/tau/nrm in tree (sorted) order. grad=True
    returns (u, g) with the target gradient g [nrhs, 3, n] from the
    differentiated P2P, M2P and L2P steps.

    ops: the expansion operators (``Laplace3D`` by default, or an instance of
    ``oracle.helm3d.Helmholtz3D``); translations receive the level of the box
    their result is centred on.
    """
    n = pts.shape[0]
    if P_levels is None:
        P_levels = expansion_orders(T, eps)
    X = Laplace3D if ops is None else ops
    nr = (sigma if sigma is not None else tau).shape[0]
    u = np.zeros((nr, n), complex)
    g = np.zeros((nr, 3, n), complex) if grad else None
    nb = T.nboxes
    lv = T.box_level
    cen = T.center_re + 1j * T.center_im
    st, en = T.box_start, T.box_end
    l0 = T.l0
    dipole = tau is not None

    def src(b):
        s, e = st[b], en[b]
        sg = None if sigma is None else sigma[:, s:e]
        dp = None if not dipole else (nrm[s:e], tau[:, s:e])
        return s, e, sg, dp

    expand = nb > 1
    M, Lc = {}, {}
    for b in range(nb):
        if expand and lv[b] >= l0 and T.box_leaf[b]:
            s, e, sg, dp = src(b)
            M[b] = X.p2m(P_levels[lv[b]], pts[s:e] - cen[b][None, :], sg, dp)
    batched = getattr(X, "batched", False)
    for l in range(T.nlevels - 1, l0 - 1, -1):
        Pp = P_levels[l]
        for b in range(T.level_offset[l], T.level_offset[l + 1]):
            if expand and not T.box_leaf[b]:
                M[b] = np.zeros((nr, (Pp + 1) ** 2), complex)
        if not expand or l + 1 >= T.nlevels:
            continue
        kids = [c for c in range(T.level_offset[l + 1], T.level_offset[l + 2])]
        if batched and kids:
            par = [T.box_parent[c] for c in kids]
            out = X.m2m(P_levels[l + 1], Pp, np.stack([M[c] for c in kids]),
                        np.stack([cen[c] - cen[p] for c, p in zip(kids, par)]), l)
            for i, p in enumerate(par):
                M[p] += out[i]
        else:
            for c in kids:
                p = T.box_parent[c]
                M[p] += X.m2m(P_levels[l + 1], Pp, M[c], cen[c] - cen[p], l)
    for b in range(nb):
        if not T.box_leaf[b]:
            continue
        ts, te = st[b], en[b]
        for a in (T.lists["list1"][b] if expand else [b]):
            s, e, sg, dp = src(a)
            d = pts[ts:te, None, :] - pts[None, s:e, :]
            zero = np.all(d == 0, axis=-1)
            dd = np.where(zero[..., None], 1.0, d)
            slp, dlp = kernel_pair(3, X.kernel, X.kappa, dd, None if not dipole else
                                   np.broadcast_to(nrm[None, s:e, :], dd.shape))
            if sg is not None:
                u[:, ts:te] += sg @ np.where(zero, 0, slp).T
            if dipole:
                u[:, ts:te] += tau[:, s:e] @ np.where(zero, 0, dlp).T
            if grad:
                gs, gd = kernel_pair_grad(3, X.kernel, X.kappa, dd, None if not dipole else
                                          np.broadcast_to(nrm[None, s:e, :], dd.shape))
                if sg is not None:
                    g[:, :, ts:te] += np.einsum("tmk,rm->rkt", np.where(zero[..., None], 0, gs), sg)
                if dipole:
                    g[:, :, ts:te] += np.einsum("tmk,rm->rkt", np.where(zero[..., None], 0, gd), tau[:, s:e])
    if not expand:
        return (u, g) if grad else u
    for b in range(nb):
        if lv[b] >= l0:
            Lc[b] = np.zeros((nr, (P_levels[lv[b]] + 1) ** 2), complex)
    for l in range(l0, T.nlevels):
        pairs = [(b, a) for b in range(T.level_offset[l], T.level_offset[l + 1])
                 for a in T.lists["list2"][b]]
        if batched and pairs:
            out = X.m2l(P_levels[l], np.stack([M[a] for b, a in pairs]),
                        np.stack([cen[b] - cen[a] for b, a in pairs]), l)
            for i, (b, a) in enumerate(pairs):
                Lc[b] += out[i]
        else:
            for b, a in pairs:
                Lc[b] += X.m2l(P_levels[l], M[a], cen[b] - cen[a], l)
    for b in range(nb):
        if T.box_leaf[b] and lv[b] >= l0:
            ts, te = st[b], en[b]
            for a in T.lists["list3"][b]:
                u[:, ts:te] += X.m2p(P_levels[lv[a]], M[a], pts[ts:te] - cen[a][None, :])
                if grad:
                    g[:, :, ts:te] += X.m2p_grad(P_levels[lv[a]], M[a], pts[ts:te] - cen[a][None, :])
    for b in range(nb):
        if lv[b] < l0:
            continue
        for a in T.lists["list4"][b]:
            s, e, sg, dp = src(a)
            Lc[b] += X.p2l(P_levels[lv[b]], pts[s:e] - cen[b][None, :], sg, dp)
    for l in range(l0 + 1, T.nlevels):
        kids = list(range(T.level_offset[l], T.level_offset[l + 1]))
        if batched and kids:
            out = X.l2l(P_levels[l - 1], P_levels[l], np.stack([Lc[T.box_parent[b]] for b in kids]),
                        np.stack([cen[b] - cen[T.box_parent[b]] for b in kids]), l)
            for i, b in enumerate(kids):
                Lc[b] += out[i]
        else:
            for b in kids:
                p = T.box_parent[b]
                Lc[b] += X.l2l(P_levels[l - 1], P_levels[l], Lc[p], cen[b] - cen[p], l)
    for b in range(nb):
        if T.box_leaf[b] and lv[b] >= l0:
            ts, te = st[b], en[b]
            u[:, ts:te] += X.l2p(P_levels[lv[b]], Lc[b], pts[ts:te] - cen[b][None, :])
            if grad:
                g[:, :, ts:te] += X.l2p_grad(P_levels[lv[b]], Lc[b], pts[ts:te] - cen[b][None, :])
    return (u, g) if grad else u


def apply(geom_re, geom_im, eps, N_s, k=1, sigma=None, tau=None, nrm_re=None, nrm_im=None,
          P_levels=None, T=None, ops=None):
    """User-order 3D FMM (Laplace unless ops is given); sigma/tau complex [nrhs, n] or [n].
    Returns (u, T)."""
    pts = np.asarray(geom_re) + 1j * np.asarray(geom_im)
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, eps=eps, helmholtz=False)
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
    nrm = None if tau is None else (np.asarray(nrm_re) + 1j * np.asarray(nrm_im))[perm]
    u_s = fmm3d(T, eps, pts[perm], sg, tu, nrm, P_levels, ops)
    u = np.empty_like(u_s)
    u[:, perm] = u_s
    return (u[0] if single else u), T


def apply_grad(geom_re, geom_im, eps, N_s, k=1, sigma=None, tau=None, nrm_re=None, nrm_im=None,
               P_levels=None, T=None, ops=None):
    """As ``apply``, also returning the target gradient: (u, g, T), g [nrhs, 3, n]
    (or [3, n]) in input order."""
    pts = np.asarray(geom_re) + 1j * np.asarray(geom_im)
    if T is None:
        T = tr.build_tree(geom_re, geom_im, N_s, k=k, eps=eps, helmholtz=False)
    perm = T.perm
    single = (sigma if sigma is not None else tau).ndim == 1
    prep = lambda v: None if v is None else np.atleast_2d(np.asarray(v, complex))[:, perm]
    nrm = None if tau is None else (np.asarray(nrm_re) + 1j * np.asarray(nrm_im))[perm]
    u_s, g_s = fmm3d(T, eps, pts[perm], prep(sigma), prep(tau), nrm, P_levels, ops, grad=True)
    u = np.empty_like(u_s)
    u[:, perm] = u_s
    g = np.empty_like(g_s)
    g[:, :, perm] = g_s
    return (u[0], g[0], T) if single else (u, g, T)
