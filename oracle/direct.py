"""Direct sums: the plain definition of what the FMM approximates.

Test infrastructure (oracle). Follows Sec. 2.1 (single/double layer, Eqs.
single_layer, double_layer), Sec. 2.3 Eq. evaluation_problem, and the
constant-free sums Eq. lap_2d_pot (2D Laplace, kernel log r), Eq. helm_2d_pot
(2D Helmholtz, H_0^(1)(kappa r)), Eq. lap_3d_pot (3D Laplace, 1/rho) and the
3D Helmholtz sum of Sec. 5.3 (exp(i kappa rho)/rho).

Readings taken here:

* the complex distance is r = sqrt((x-y).(x-y)) on the principal branch
  (Sec. 2.1, Def. 3.1); log r is evaluated as Log(r^2)/2, which equals
  Log(sqrt(r^2)) whenever Re r^2 > 0 (guaranteed by Assumptions 4.1/5.1);
* the double layer for complex points uses a caller-supplied complex normal n
  and is n . grad_y K(x, y) (Eq. double_layer with the unit normal replaced
  by the given vector, whose length carries the quadrature weight);
* a pair with x - y == 0 exactly (the self pair when sources are targets) is
  skipped;
* the kernels are constant-free (the paper drops -1/2pi, i/4, 1/4pi);
  ``green_scale`` restores them.
"""
from __future__ import annotations

import numpy as np
import scipy.special as sps

LAPLACE, HELMHOLTZ = 0, 1

GREEN_SCALE = {
    (2, LAPLACE): -1.0 / (2.0 * np.pi),
    (2, HELMHOLTZ): 0.25j,
    (3, LAPLACE): 1.0 / (4.0 * np.pi),
    (3, HELMHOLTZ): 1.0 / (4.0 * np.pi),
}


def kernel_pair(dim, kernel, kappa, d, nrm=None):
    """K(x, y) and n . grad_y K(x, y) for complex displacement d = x - y.

    d: complex array [..., dim]; nrm: complex [..., dim] or None.
    Returns (slp, dlp) complex arrays (dlp is None when nrm is None).
    """
    r2 = np.sum(d * d, axis=-1)
    nd = None if nrm is None else np.sum(nrm * d, axis=-1)
    dlp = None
    if dim == 2 and kernel == LAPLACE:
        # log r = Log(r^2)/2;  grad_y log r = (y - x)/r^2
        slp = 0.5 * np.log(r2)
        if nrm is not None:
            dlp = -nd / r2
    elif dim == 2 and kernel == HELMHOLTZ:
        r = np.sqrt(r2)
        z = kappa * r
        slp = sps.hankel1(0, z)
        if nrm is not None:
            # d/dy H0(kappa r) = -kappa H1(kappa r) dr/dy,  dr/dy = -(x-y)/r
            dlp = kappa * sps.hankel1(1, z) * nd / r
    elif dim == 3 and kernel == LAPLACE:
        r = np.sqrt(r2)
        slp = 1.0 / r
        if nrm is not None:
            # grad_y 1/r = (x-y)/r^3
            dlp = nd / (r2 * r)
    elif dim == 3 and kernel == HELMHOLTZ:
        r = np.sqrt(r2)
        e = np.exp(1j * kappa * r)
        slp = e / r
        if nrm is not None:
            # d/dr (e^{ikr}/r) = e^{ikr}(ikr-1)/r^2 ; dr/dy . n = -(n.d)/r
            dlp = nd * (1.0 - 1j * kappa * r) * e / (r2 * r)
    else:
        raise ValueError("unsupported dim/kernel")
    return slp, dlp


def kernel_pair_grad(dim, kernel, kappa, d, nrm=None):
    """grad_x K(x, y) and grad_x (n . grad_y K)(x, y) for d = x - y (Sec. 2.1:
    the target gradient of the single and double layer kernels, whose normal
    components give S' and D').

    With K = K(r), grad_x K = K'(r) d / r, and since n . grad_y K = -K'(r) (n.d)/r,
    grad_x (n . grad_y K) = -(K'(r)/r) n - (K''(r) - K'(r)/r) (n.d) d / r^2.
    d: complex [..., dim]; returns (gs, gd) complex [..., dim] (gd None without nrm).
    """
    r2 = np.sum(d * d, axis=-1)
    r = np.sqrt(r2)
    if dim == 2 and kernel == LAPLACE:
        k1 = 1.0 / r                              # K = log r
        k2 = -1.0 / r2
    elif dim == 2 and kernel == HELMHOLTZ:
        z = kappa * r
        h0, h1 = sps.hankel1(0, z), sps.hankel1(1, z)
        k1 = -kappa * h1                          # K = H0(kappa r)
        k2 = -kappa * kappa * (h0 - h1 / z)       # d/dr (-kappa H1) = -kappa^2 H1'(z)
    elif dim == 3 and kernel == LAPLACE:
        k1 = -1.0 / r2                            # K = 1/r
        k2 = 2.0 / (r2 * r)
    elif dim == 3 and kernel == HELMHOLTZ:
        e = np.exp(1j * kappa * r)                # K = e^{i kappa r}/r
        k1 = e * (1j * kappa * r - 1.0) / r2
        k2 = e * (2.0 - 2j * kappa * r - kappa * kappa * r2) / (r2 * r)
    else:
        raise ValueError("unsupported dim/kernel")
    gs = (k1 / r)[..., None] * d
    gd = None
    if nrm is not None:
        nd = np.sum(nrm * d, axis=-1)
        gd = -(k1 / r)[..., None] * nrm - ((k2 - k1 / r) * nd / r2)[..., None] * d
    return gs, gd


def direct_grad(dim, kernel, kappa, src, trg, sigma=None, tau=None, nrm=None, chunk=None):
    """grad_x u(x_i) for u of ``direct``: [nrhs][dim][N] (or [dim][N]); pairs
    with x - y == 0 are skipped."""
    src = np.asarray(src, dtype=np.complex128)
    trg = np.asarray(trg, dtype=np.complex128)
    single = True
    if sigma is not None:
        sigma = np.asarray(sigma, dtype=np.complex128)
        single = sigma.ndim == 1
    if tau is not None:
        tau = np.asarray(tau, dtype=np.complex128)
        single = tau.ndim == 1
        nrm = np.asarray(nrm, dtype=np.complex128)
    nrhs = (np.atleast_2d(sigma) if sigma is not None else np.atleast_2d(tau)).shape[0]
    N, M = trg.shape[0], src.shape[0]
    out = np.zeros((nrhs, dim, N), dtype=np.complex128)
    if chunk is None:
        chunk = max(1, min(N, 2_000_000 // max(M, 1)))
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        d = trg[a:b, None, :] - src[None, :, :]
        zero = np.all(d == 0, axis=-1)
        d = np.where(zero[..., None], 1.0, d)
        gs, gd = kernel_pair_grad(dim, kernel, kappa, d, None if tau is None else np.broadcast_to(nrm[None], d.shape))
        if sigma is not None:
            gs = np.where(zero[..., None], 0.0, gs)
            out[:, :, a:b] += np.einsum("tmk,rm->rkt", gs, np.atleast_2d(sigma))
        if tau is not None:
            gd = np.where(zero[..., None], 0.0, gd)
            out[:, :, a:b] += np.einsum("tmk,rm->rkt", gd, np.atleast_2d(tau))
    return out[0] if single else out


def direct(dim, kernel, kappa, src, trg, sigma=None, tau=None, nrm=None,
           chunk=None, green_scale=False):
    """u(x_i) = sum_j K(x_i, y_j) sigma_j + sum_j (n_j . grad_y K)(x_i, y_j) tau_j.

    src, trg: complex [M, dim], [N, dim]; sigma, tau: complex [M] or [nrhs, M];
    nrm: complex [M, dim] (required when tau is given). Pairs with x - y == 0
    are skipped. Returns complex [N] (or [nrhs, N]).
    """
    src = np.asarray(src, dtype=np.complex128)
    trg = np.asarray(trg, dtype=np.complex128)
    single = True
    rhs = []
    if sigma is not None:
        sigma = np.asarray(sigma, dtype=np.complex128)
        single = sigma.ndim == 1
        rhs.append(np.atleast_2d(sigma))
    if tau is not None:
        tau = np.asarray(tau, dtype=np.complex128)
        single = tau.ndim == 1
        if nrm is None:
            raise ValueError("double layer needs normals")
        nrm = np.asarray(nrm, dtype=np.complex128)
    nrhs = (np.atleast_2d(sigma) if sigma is not None else np.atleast_2d(tau)).shape[0]
    N, M = trg.shape[0], src.shape[0]
    out = np.zeros((nrhs, N), dtype=np.complex128)
    if chunk is None:
        chunk = max(1, min(N, 4_000_000 // max(M, 1)))
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        d = trg[a:b, None, :] - src[None, :, :]
        zero = np.all(d == 0, axis=-1)
        d = np.where(zero[..., None], 1.0, d)          # placeholder, masked below
        slp, dlp = kernel_pair(dim, kernel, kappa, d,
                               None if tau is None else np.broadcast_to(nrm[None], d.shape))
        if sigma is not None:
            slp = np.where(zero, 0.0, slp)
            out[:, a:b] += np.einsum("tm,rm->rt", slp, np.atleast_2d(sigma))
        if tau is not None:
            dlp = np.where(zero, 0.0, dlp)
            out[:, a:b] += np.einsum("tm,rm->rt", dlp, np.atleast_2d(tau))
    if green_scale:
        out *= GREEN_SCALE[(dim, kernel)]
    return out[0] if single else out


def relerr_paper(u, u0, sigma):
    """Eq. relerr: ||u - u0|| / (||u0|| + ||sigma||)."""
    return float(np.linalg.norm(u - u0) / (np.linalg.norm(u0) + np.linalg.norm(sigma)))


def relerr_l2(u, u0):
    """Plain relative l2 error ||u - u0|| / ||u0||."""
    return float(np.linalg.norm(u - u0) / np.linalg.norm(u0))
