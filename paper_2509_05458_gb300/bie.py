"""Complex-scaled boundary integral equation solved by GMRES with the FMM as
its matvec (Sec. 2.2, "Complex scaling and integral equations").

Sound-soft scattering on a perturbed half-space in 2D: the boundary
Gamma = {(t, gamma_2(t))} is deformed into the complex curve
    gamma~(t) = (t + i psi(t), gamma_2(t)),
psi smooth, odd, vanishing on [-t0, t0] and growing like a b |t| outside
(the auxiliary functions of Sec. 7: xi(s) = (s erfc(s) - e^{-s^2}/sqrt(pi))/2,
psi(t) = a (xi(b (t + t0)) - xi(b (t0 - t))), so psi' = (a b / 2) (erfc(b (t +
t0)) + erfc(b (t0 - t))) and |psi'| <= a b). The solution above the curve is
represented as a double layer potential u = D[sigma] over the deformed curve,
and the Dirichlet condition u = f on it gives Eq. complex_BIE,
    -sigma/2 + D[sigma] = f.
On the deformed curve f and sigma decay like e^{-kappa |psi|}, so the curve is
truncated to t in [-T, T] (Eq. fast_decay_bound).

Discretisation: the trapezoidal rule in t with spacing h (no quadrature
corrections: they are outside this library). The double layer kernel
(i/4) kappa H_1(kappa r) nu.(x - y)/r with the unnormalised normal
nu = (gamma_2', -gamma_1') (the library's DLP with CFMM_GREEN_SCALE and the
normal times h) is smooth on the curve; its limit at y = x,
    (gamma_2' gamma_1'' - gamma_1' gamma_2'') / (4 pi (gamma' . gamma')),
is the diagonal of the Nystrom matrix (the library skips the self pair).

Every application of the operator is one cfmm_apply on a plan built once
(the resident plan of a GMRES solve); the data come from cfmm_direct with a
single unit source, and the solution off the curve from cfmm_direct at the
targets. GMRES (restarted, modified Gram-Schmidt, Givens rotations) runs on
torch tensors on the plan's device: vector plumbing around the library's
kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import DLP, FP64, GREEN_SCALE, HELMHOLTZ, LAPLACE, SLP, direct, plan


def _xi(s, erfc):
    return 0.5 * (s * erfc(s) - np.exp(-s * s) / math.sqrt(math.pi))


class HalfSpaceCurve:
    """The truncated, deformed curve t -> (t + i psi(t), height e^{-t^2}) at the
    trapezoidal nodes t_j = -T + (j + 1/2) h, h = 2T/n, with the derivatives the
    double layer needs."""

    def __init__(self, n, T=10.0, height=0.5, a=0.5, b=1.0, t0=3.0):
        from scipy.special import erfc
        self.n, self.T, self.h = n, T, 2.0 * T / n
        t = -T + (np.arange(n) + 0.5) * self.h
        self.t = t
        psi = a * (_xi(b * (t + t0), erfc) - _xi(b * (t0 - t), erfc))
        dpsi = 0.5 * a * b * (erfc(b * (t + t0)) + erfc(b * (t0 - t)))
        d2psi = a * b * b / math.sqrt(math.pi) * (np.exp(-(b * (t0 - t)) ** 2) - np.exp(-(b * (t + t0)) ** 2))
        g2 = height * np.exp(-t * t)
        self.re = np.stack([t, g2], axis=1)
        self.im = np.stack([psi, np.zeros_like(t)], axis=1)
        d1 = 1.0 + 1j * dpsi                      # gamma_1'
        d2 = -2.0 * t * g2                        # gamma_2'
        dd1 = 1j * d2psi                          # gamma_1''
        dd2 = (4.0 * t * t - 2.0) * g2            # gamma_2''
        nu = np.stack([d2, -d1], axis=1) * self.h   # unnormalised normal times the weight
        self.nrm_re = np.ascontiguousarray(nu.real)
        self.nrm_im = np.ascontiguousarray(nu.imag)
        # limit of the (Green-scaled) double layer kernel at y = x, times the weight
        self.diag = self.h * (d2 * dd1 - d1 * dd2) / (4.0 * math.pi * (d1 * d1 + d2 * d2))
        self.slope = a * b
        self.psi = psi


def gmres(matvec, b, tol=1e-10, restart=60, maxiter=2000):
    """Restarted GMRES for complex torch vectors; returns (x, iterations,
    relative residual history)."""
    import torch
    x = torch.zeros_like(b)
    bn = float(torch.linalg.vector_norm(b))
    hist = []
    it = 0
    while it < maxiter:
        r = b - matvec(x)
        beta = float(torch.linalg.vector_norm(r))
        hist.append(beta / bn)
        if beta / bn <= tol:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for k in range(restart):
            w = matvec(V[k])
            for i in range(k + 1):
                hik = complex(torch.vdot(V[i], w))
                H[i, k] = hik
                w = w - hik * V[i]
            H[k + 1, k] = float(torch.linalg.vector_norm(w))
            if abs(H[k + 1, k]) > 0:
                V.append(w / H[k + 1, k])
            # earlier rotations G_i = [[conj c, conj s], [-s, c]] on the new column
            for i in range(k):
                t0 = np.conj(cs[i]) * H[i, k] + np.conj(sn[i]) * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t0
            den = math.hypot(abs(H[k, k]), abs(H[k + 1, k]))
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            hist.append(abs(g[k + 1]) / bn)
            if abs(g[k + 1]) / bn <= tol or it >= maxiter or len(V) <= k + 1:
                break
        m = k + 1
        y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
        for i in range(m):
            x = x + complex(y[i]) * V[i]
        if hist[-1] <= tol:
            break
    return x, it, hist


class DirichletHalfSpace:
    """-sigma/2 + D[sigma] = f on the deformed curve (Eq. complex_BIE), with
    kernel 'helmholtz' (wavenumber kappa) or 'laplace'."""

    def __init__(self, curve, kappa, eps=1e-10, device="cuda", leaf_size=64, precision=FP64, use_fmm=True):
        import torch
        self.c = curve
        self.kappa = kappa
        self.ker = HELMHOLTZ if kappa > 0 else LAPLACE
        self.dev = torch.device(device)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)
        self.re, self.im = t(curve.re), t(curve.im)
        self.nre, self.nim = t(curve.nrm_re), t(curve.nrm_im)
        self.diag = t(curve.diag)
        self.use_fmm = use_fmm
        self.flags = self.ker | DLP | GREEN_SCALE
        self.plan = plan(2, self.flags, kappa, eps, self.re, self.im, self.nre, self.nim,
                         leaf_size=leaf_size, precision=precision) if use_fmm else None
        self.matvecs = 0

    def matvec(self, sigma):
        import torch
        self.matvecs += 1
        d = sigma.reshape(1, 1, -1).contiguous()
        if self.use_fmm:
            Dsig = self.plan.apply(d)[0]
        else:
            Dsig = direct(2, self.flags, self.kappa, self.re, self.im, self.re, self.im, d, self.nre, self.nim)[0]
        return -0.5 * sigma + Dsig + self.diag * sigma

    def point_source_data(self, x0):
        """f = G(x, x0) on the curve (the library's direct sum with one unit
        source at the real point x0 and the Green's function constant)."""
        import torch
        src = torch.tensor([list(x0)], dtype=torch.float64, device=self.dev)
        one = torch.ones((1, 1, 1), dtype=torch.complex128, device=self.dev)
        return direct(2, self.ker | SLP | GREEN_SCALE, self.kappa, src, torch.zeros_like(src), self.re, self.im,
                      one)[0]

    def evaluate(self, sigma, targets):
        """u = D[sigma] at real targets (n, 2) off the curve."""
        import torch
        tr = torch.as_tensor(np.asarray(targets, dtype=np.float64), device=self.dev)
        d = sigma.reshape(1, 1, -1).contiguous()
        return direct(2, self.flags, self.kappa, self.re, self.im, tr, torch.zeros_like(tr), d, self.nre, self.nim)[0]

    def solve(self, f, tol=1e-10, restart=60, maxiter=2000):
        return gmres(self.matvec, f, tol=tol, restart=restart, maxiter=maxiter)
