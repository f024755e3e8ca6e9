"""GMRES on the complex-scaled half-space BIE (Sec. 2.2) with the FMM apply of a
resident plan as the matvec: the solution reproduces the exact field of a point
source above the curve, and matches the solve with the library's direct sum as
the matvec."""
import numpy as np
import pytest
import scipy.special as sps

pytestmark = pytest.mark.gpu


def test_gmres_fmm_half_space(cuda):
    import torch
    from paper_2509_05458_gb300.bie import HalfSpaceCurve, DirichletHalfSpace
    kap = 5.0
    c = HalfSpaceCurve(3200, T=10.0)
    x0 = (0.0, -1.0)
    tg = np.array([[0.5, 1.5], [-2.0, 1.0], [3.0, 2.5]])
    ue = 0.25j * sps.hankel1(0, kap * np.linalg.norm(tg - np.array(x0), axis=1))
    prob = DirichletHalfSpace(c, kap, eps=1e-12, device=cuda)
    f = prob.point_source_data(x0)
    sig, its, hist = prob.solve(f, tol=1e-12)
    assert hist[-1] <= 1e-12 and its < 200
    u = prob.evaluate(sig, tg).cpu().numpy()
    assert np.max(np.abs(u - ue) / np.abs(ue)) < 1e-7
    ref = DirichletHalfSpace(c, kap, device=cuda, use_fmm=False)
    sig2, _, _ = ref.solve(f, tol=1e-12)
    assert float(torch.linalg.vector_norm(sig - sig2) / torch.linalg.vector_norm(sig2)) < 1e-10
