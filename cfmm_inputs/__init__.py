"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds geometry and density generators only: none of the method's
arithmetic (no kernels, expansions, trees or lists). Every generator draws from
numpy's PCG64 with an explicit seed, in a fixed order, so both sides see the
same bits.

Families (they stand in for the paper's complexified wobbly curve/surface of
Sec. 7.1, Eqs. wobble_2D_cplx / complex_wobble, whose discretisations need
external packages):

* ``curve2d``: points on the curve t -> (t, h*exp(-t^2)), t uniform, with the
  x1 coordinate complexified by phi(t) = s*sign(t)*max(|t|-t_flat, 0)
  (Lipschitz constant s). Normals are (gamma_2'(t), -gamma_1'(t)) of the
  complexified curve, unnormalised (Sec. 2.1 double layer, read for complex
  points as a caller-supplied complex normal).
* ``surface3d``: (x, y) from the Halton sequence (bases 2, 3) scaled to a
  square, z = a*exp(-(x^2+y^2)/w^2), imaginary part
  s*max(rho-rho0, 0)*(x, y)/rho in (x1, x2) and 0 in x3.
* ``densities``: i.i.d. complex Gaussians (real and imaginary N(0,1)).
* ``wobble2d`` / ``wobble3d``: the paper's own test interfaces of Sec. 7.1
  (Eqs. wobble_2D_cplx and complex_wobble) with the deformation psi_{a,b,t0}
  built from xi (readings: xi(s) = (s erfc(s) - e^{-s^2}/sqrt(pi))/2, so that
  xi' = erfc/2; psi(t) = a (xi(b (t + t0)) - xi(b (t0 - t))), odd, flat on
  |t| < t0 and of slope a b beyond; the 2D bump's window is
  (erfc(2 (t - 6)) - erfc(2 (t + 6)))/2, one on [-6, 6] and zero outside).
  The paper discretises them with ChunkIE panels / a corrected trapezoidal
  rule and samples points; here t is uniform on [-20, 20] (2D, the range is
  not stated) and (t1, t2) are Halton points of [-25, 25]^2 (3D).
"""
from __future__ import annotations

import numpy as np

__all__ = ["curve2d", "surface3d", "densities", "halton", "Geometry",
           "curve2d_short", "curve2d_long", "plane3d", "plane3d_uneven", "wobble2d", "wobble3d", "psi_abt",
           "isotropic_pair3d"]


class Geometry:
    """Points (and optional normals) as real/imaginary [n][dim] float64 arrays."""

    def __init__(self, re, im, nrm_re=None, nrm_im=None, meta=None):
        self.re = np.ascontiguousarray(re, dtype=np.float64)
        self.im = np.ascontiguousarray(im, dtype=np.float64)
        self.nrm_re = None if nrm_re is None else np.ascontiguousarray(nrm_re, dtype=np.float64)
        self.nrm_im = None if nrm_im is None else np.ascontiguousarray(nrm_im, dtype=np.float64)
        self.meta = dict(meta or {})

    @property
    def n(self):
        return self.re.shape[0]

    @property
    def dim(self):
        return self.re.shape[1]

    def subset(self, idx):
        idx = np.asarray(idx)
        return Geometry(self.re[idx], self.im[idx],
                        None if self.nrm_re is None else self.nrm_re[idx],
                        None if self.nrm_im is None else self.nrm_im[idx],
                        self.meta)


def curve2d(n, seed=0, t_half=10.0, height=0.3, slope=0.5, t_flat=4.0,
            random_height=None):
    """Complexified bump curve in C x R.

    ``random_height=(lo, hi)`` draws the bump height once, before the t's.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if random_height is not None:
        height = float(rng.uniform(random_height[0], random_height[1]))
    t = rng.uniform(-t_half, t_half, size=n)
    g2 = height * np.exp(-t * t)
    re = np.stack([t, g2], axis=1)
    phi = slope * np.sign(t) * np.maximum(np.abs(t) - t_flat, 0.0)
    im = np.stack([phi, np.zeros_like(t)], axis=1)
    dphi = slope * (np.abs(t) > t_flat).astype(np.float64)
    # gamma' = (1 + i phi', -2 t h e^{-t^2}); normal = (gamma_2', -gamma_1')
    nrm_re = np.stack([-2.0 * t * g2, -np.ones_like(t)], axis=1)
    nrm_im = np.stack([np.zeros_like(t), -dphi], axis=1)
    return Geometry(re, im, nrm_re, nrm_im,
                    dict(family="curve2d", n=n, seed=seed, t_half=t_half,
                         height=height, slope=slope, t_flat=t_flat))


def halton(n, base, start=1):
    """Radical-inverse (van der Corput) sequence in `base` for indices start..start+n-1."""
    idx = np.arange(start, start + n, dtype=np.int64)
    out = np.zeros(n, dtype=np.float64)
    f = 1.0
    i = idx.copy()
    while np.any(i > 0):
        f /= base
        out += f * (i % base)
        i //= base
    return out


def surface3d(n, seed=0, half=20.0, amp=0.5, width=1.0, slope=0.4, rho0=6.0,
              random_shape=False):
    """Complexified plane with a Gaussian bump in C^2 x R.

    ``random_shape`` draws width ~ U[0.5, 3] and slope ~ U[0.2, 0.8] from the seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if random_shape:
        width = float(rng.uniform(0.5, 3.0))
        slope = float(rng.uniform(0.2, 0.8))
    x = (2.0 * halton(n, 2) - 1.0) * half
    y = (2.0 * halton(n, 3) - 1.0) * half
    z = amp * np.exp(-(x * x + y * y) / (width * width))
    rho = np.sqrt(x * x + y * y)
    fac = np.where(rho > 0, slope * np.maximum(rho - rho0, 0.0) / np.where(rho > 0, rho, 1.0), 0.0)
    re = np.stack([x, y, z], axis=1)
    im = np.stack([fac * x, fac * y, np.zeros_like(x)], axis=1)
    # normal of the real graph z(x, y), continued: (-z_x, -z_y, 1); the
    # complexification leaves x3 real, so the normal is kept real here.
    zx = -2.0 * x / (width * width) * z
    zy = -2.0 * y / (width * width) * z
    nrm_re = np.stack([-zx, -zy, np.ones_like(x)], axis=1)
    nrm_im = np.zeros_like(nrm_re)
    return Geometry(re, im, nrm_re, nrm_im,
                    dict(family="surface3d", n=n, seed=seed, half=half,
                         amp=amp, width=width, slope=slope, rho0=rho0))


def densities(n, seed=0, nrhs=1, ncomp=1):
    """Complex Gaussian densities, shape [nrhs][ncomp][n], complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((nrhs, ncomp, n, 2))
    return (a[..., 0] + 1j * a[..., 1]).astype(np.complex128)


# ---- the named workloads -------------------------------------------------

def curve2d_short(n=4000, seed=0):
    """The 2D Laplace SLP workload: N = 4000 on t in [-10, 10], bump height 0.3,
    imaginary slope 0.5 beyond |t| = 4."""
    return curve2d(n, seed=seed, t_half=10.0, height=0.3, slope=0.5, t_flat=4.0)


def curve2d_long(n=100000, seed=0):
    """The 2D Helmholtz SLP+DLP workload: N = 1e5 on t in [-40, 40], bump
    height ~ U[0.3, 1], imaginary slope 0.5 beyond |t| = 4."""
    return curve2d(n, seed=seed, t_half=40.0, slope=0.5, t_flat=4.0,
                   random_height=(0.3, 1.0))


def plane3d(n=1000000, seed=0):
    """The 3D workload: N = 1e6 Halton points of the complexified plane with a
    bump over [-20, 20]^2, imaginary slope 0.4 beyond rho = 6."""
    return surface3d(n, seed=seed, half=20.0, amp=0.5, width=1.0, slope=0.4, rho0=6.0)


def plane3d_uneven(count=32, seed0=100, nmin=10_000, nmax=200_000):
    """The uneven batch of the batched 3D Helmholtz workload: `count` surfaces
    of the ``surface3d`` family ([-20, 20]^2, bump 0.5, rho0 = 6), geometry i
    with N log-uniform in [nmin, nmax] (drawn from seed0) and its width ~
    U[0.5, 3] and slope ~ U[0.2, 0.8] drawn from seed0 + 1 + i."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=count))
    return [surface3d(int(round(n)), seed=seed0 + 1 + i, half=20.0, amp=0.5, rho0=6.0, random_shape=True)
            for i, n in enumerate(ns)]


# ---- the paper's test interfaces (Sec. 7.1) ---------------------------------

def _xi(s):
    from scipy.special import erfc
    return 0.5 * (s * erfc(s) - np.exp(-s * s) / np.sqrt(np.pi))


def psi_abt(t, a, b, t0):
    """psi_{a,b,t0}(t) = a (xi(b (t + t0)) - xi(b (t0 - t))) (see the module
    docstring for the reading of the printed formula)."""
    t = np.asarray(t, dtype=np.float64)
    return a * (_xi(b * (t + t0)) - _xi(b * (t0 - t)))


def wobble2d(n, seed=0, t_half=20.0, a=1.0 / 20.0, b=3.0, t0=13.0):
    """Eq. wobble_2D_cplx: (t + i psi(t), 2 e^{-t^2/16} cos(8t) w(t)), t uniform
    on [-t_half, t_half], w the window of the module docstring. No normals (the
    paper's timings are single-layer)."""
    from scipy.special import erfc
    rng = np.random.Generator(np.random.PCG64(seed))
    t = rng.uniform(-t_half, t_half, size=n)
    w = 0.5 * (erfc(2.0 * (t - 6.0)) - erfc(2.0 * (t + 6.0)))
    re = np.stack([t, 2.0 * np.exp(-t * t / 16.0) * np.cos(8.0 * t) * w], axis=1)
    im = np.stack([psi_abt(t, a, b, t0), np.zeros_like(t)], axis=1)
    return Geometry(re, im, meta=dict(family="wobble2d", n=n, seed=seed, a=a, b=b, t0=t0))


def wobble3d(n, half=25.0, a=0.2, b=0.75, t0=12.0):
    """Eq. complex_wobble: (u + i psi(u), v + i psi(v), e^{-(u^2+v^2)/8}
    (cos(1.9u + 0.95v) + sin(u + 1.55v))) with u = t1 (1 - e^{-(t1^2+t2^2)/300}/2),
    v likewise, (t1, t2) the Halton points (bases 2, 3) of [-half, half]^2."""
    t1 = (2.0 * halton(n, 2) - 1.0) * half
    t2 = (2.0 * halton(n, 3) - 1.0) * half
    e = np.exp(-(t1 * t1 + t2 * t2) / 300.0)
    u = t1 - 0.5 * t1 * e
    v = t2 - 0.5 * t2 * e
    z = np.exp(-(u * u + v * v) / 8.0) * (np.cos(1.9 * u + 0.95 * v) + np.sin(u + 1.55 * v))
    re = np.stack([u, v, z], axis=1)
    im = np.stack([psi_abt(u, a, b, t0), psi_abt(v, a, b, t0), np.zeros_like(u)], axis=1)
    return Geometry(re, im, meta=dict(family="wobble3d", n=n, a=a, b=b, t0=t0))


def isotropic_pair3d(seed=5, n_cluster=12, half=0.04):
    """A 3D point set whose tree (leaf size 8, separation 2) has a List-2 pair
    at level 3 with an isotropic complex shift: eight corner points fix the
    root cube [0, 8]^3 (width W = 8 (1 + 2^-20), level-3 boxes of width
    w = W/8), and two clusters of n_cluster points sit around the centres of
    the level-3 boxes (2, 3, 1) and (3, 3, 4), the second with imaginary part
    (0, w, 0). The complexified centres then differ by d = (w, i w, 3 w), so
    d1^2 + d2^2 = 0 with (d1, d2) != 0; the imaginary slope between the
    clusters is 1/sqrt(10)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W = 8.0 * (1.0 + 2.0 ** -20)
    lo = 4.0 - W / 2.0
    w = W / 8.0
    corners = np.array([[x, y, z] for x in (0.0, 8.0) for y in (0.0, 8.0) for z in (0.0, 8.0)])
    ca = lo + (np.array([2, 3, 1]) + 0.5) * w
    cb = lo + (np.array([3, 3, 4]) + 0.5) * w
    a = ca + rng.uniform(-half, half, (n_cluster, 3))
    b = cb + rng.uniform(-half, half, (n_cluster, 3))
    re = np.concatenate([corners, a, b])
    im = np.zeros_like(re)
    im[8 + n_cluster:, 1] = w
    return Geometry(re, im, meta={"family": "isotropic_pair3d", "w": w})
