"""GPU direct sum (cfmm_direct, Sec. 2.3 Eq. evaluation_problem + double layer)
against the oracle's direct sum, element by element, for all four kernels."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities
from oracle.direct import direct
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

KERNELS = [(2, 0, 0.0), (2, 1, 20.0), (2, 1, 0.7), (3, 0, 0.0), (3, 1, 10.0)]


@pytest.mark.parametrize("dim,ker,kap", KERNELS)
@pytest.mark.parametrize("layer", ["slp", "dlp", "both"])
def test_direct_matches_oracle(cuda, dim, ker, kap, layer):
    import paper_2509_05458_gb300 as cf
    g = curve2d(700, seed=4, t_half=6.0) if dim == 2 else surface3d(700, seed=4, half=3.0, rho0=1.0)
    pts = g.re + 1j * g.im
    nrm = g.nrm_re + 1j * g.nrm_im
    ncomp = 2 if layer == "both" else 1
    dens = densities(g.n, seed=5, nrhs=2, ncomp=ncomp)
    flag = {"slp": cf.SLP, "dlp": cf.DLP, "both": cf.SLP | cf.DLP}[layer]
    out = cf.direct(dim, ker | flag, kap, to_dev(g.re, cuda), to_dev(g.im, cuda), to_dev(g.re, cuda),
                    to_dev(g.im, cuda), to_dev(dens, cuda), to_dev(g.nrm_re, cuda), to_dev(g.nrm_im, cuda))
    out = out.cpu().numpy()
    for r in range(2):
        sg = dens[r, 0] if layer != "dlp" else None
        ta = dens[r, -1] if layer != "slp" else None
        ref = direct(dim, ker, kap, pts, pts, sigma=sg, tau=ta, nrm=nrm)
        err = np.abs(out[r] - ref) / np.max(np.abs(ref))
        assert err.max() < 1e-12, (r, err.max())


def test_direct_separate_targets_and_green_scale(cuda):
    import paper_2509_05458_gb300 as cf
    src = curve2d(300, seed=1)
    trg = curve2d(123, seed=2)
    dens = densities(src.n, seed=1)
    out = cf.direct(2, cf.HELMHOLTZ | cf.SLP | cf.GREEN_SCALE, 5.0, to_dev(src.re, cuda), to_dev(src.im, cuda),
                    to_dev(trg.re, cuda), to_dev(trg.im, cuda), to_dev(dens, cuda)).cpu().numpy()[0]
    ref = direct(2, 1, 5.0, src.re + 1j * src.im, trg.re + 1j * trg.im, sigma=dens[0, 0], green_scale=True)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("dim,ker,kap", KERNELS)
def test_direct_mixed_precision(cuda, dim, ker, kap):
    """Mixed precision (complex64 kernel arithmetic, FP32 hi/lo differences,
    compensated sums): relative l2 error against the FP64 oracle below 1e-6,
    max-norm error (relative to max |u|) below 5e-6."""
    import paper_2509_05458_gb300 as cf
    g = curve2d(900, seed=7, t_half=6.0) if dim == 2 else surface3d(900, seed=7, half=3.0, rho0=1.0)
    pts = g.re + 1j * g.im
    nrm = g.nrm_re + 1j * g.nrm_im
    dens = densities(g.n, seed=8, nrhs=1, ncomp=2)
    out = cf.direct(dim, ker | cf.SLP | cf.DLP, kap, to_dev(g.re, cuda), to_dev(g.im, cuda), to_dev(g.re, cuda),
                    to_dev(g.im, cuda), to_dev(dens, cuda), to_dev(g.nrm_re, cuda), to_dev(g.nrm_im, cuda),
                    precision=cf.MIXED).cpu().numpy()[0]
    ref = direct(dim, ker, kap, pts, pts, sigma=dens[0, 0], tau=dens[0, 1], nrm=nrm)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err < 5e-6, err
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-6
