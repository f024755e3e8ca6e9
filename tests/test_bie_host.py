"""The complex-scaled half-space BIE of the GMRES demo (Sec. 2.2, Eq.
complex_BIE) pinned on the CPU with the oracle's kernel: a dense Nystrom
solve of -sigma/2 + D[sigma] = f for the field of a point source below the
curve reproduces that field above the curve (the exact solution of the
Dirichlet problem), with the trapezoidal rule's convergence."""
import numpy as np
import pytest
import scipy.special as sps

from oracle.direct import kernel_pair
from paper_2509_05458_gb300.bie import HalfSpaceCurve

KAPPA = 5.0
X0 = np.array([0.0, -1.0])
TARGETS = np.array([[0.5, 1.5], [-2.0, 1.0], [3.0, 2.5]])


def _dense_solve(n):
    c = HalfSpaceCurve(n, T=10.0)
    pts = c.re + 1j * c.im
    nrm = c.nrm_re + 1j * c.nrm_im
    d = pts[:, None, :] - pts[None, :, :]
    d[np.arange(n), np.arange(n)] = 1.0            # placeholder, the diagonal is replaced below
    _, dl = kernel_pair(2, 1, KAPPA, d, np.broadcast_to(nrm[None], d.shape))
    A = 0.25j * dl
    A[np.arange(n), np.arange(n)] = c.diag
    A -= 0.5 * np.eye(n)
    r = np.sqrt(np.sum((pts - X0) ** 2, axis=1))
    f = 0.25j * sps.hankel1(0, KAPPA * r)
    sig = np.linalg.solve(A, f)
    dd = TARGETS[:, None, :] - pts[None, :, :]
    _, dl2 = kernel_pair(2, 1, KAPPA, dd, np.broadcast_to(nrm[None], dd.shape))
    u = (0.25j * dl2) @ sig
    ue = 0.25j * sps.hankel1(0, KAPPA * np.linalg.norm(TARGETS - X0, axis=1))
    return np.max(np.abs(u - ue) / np.abs(ue)), sig


def test_curve_is_lipschitz_and_decays():
    c = HalfSpaceCurve(1000, T=10.0)
    dpsi = np.diff(c.psi) / np.diff(c.t)
    assert np.max(np.abs(dpsi)) <= c.slope + 1e-12
    assert np.all(np.abs(c.psi[np.abs(c.t) < 1.0]) < 1e-3)      # psi is flat in the middle
    assert abs(c.psi[-1] + c.psi[0]) < 1e-12                    # odd


@pytest.mark.slow
def test_dense_nystrom_reproduces_point_source_field():
    e1, sig = _dense_solve(800)
    e2, _ = _dense_solve(1600)
    assert e1 < 5e-6 and e2 < 5e-7
    assert e1 / e2 > 4.0                       # trapezoidal rule on a C^2 kernel: about h^3
    assert np.max(np.abs(sig[:3])) < 1e-7 * np.max(np.abs(sig))  # exponential decay at the truncation


@pytest.mark.parametrize("restart", [5, 60])
def test_gmres_solves_complex_system(restart):
    """The solver the BIE demo uses, on a dense complex system with a known
    solution (CPU torch tensors): the iterate solves A x = b to the requested
    residual, also across restarts."""
    import torch
    from paper_2509_05458_gb300.bie import gmres
    rng = np.random.default_rng(3)
    n = 40
    A = np.eye(n) * (2.0 + 1.0j) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    x0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = A @ x0
    At = torch.from_numpy(A)
    x, its, hist = gmres(lambda v: At @ v, torch.from_numpy(b), tol=1e-13, restart=restart, maxiter=500)
    x = x.numpy()
    assert hist[-1] <= 1e-13
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x - x0) <= 1e-11 * np.linalg.norm(x0)
