"""cfmm_direct_noalloc: the direct sum for callers that cannot allocate device
memory while they run (their device-memory budget is held by a pool, or they
sit in a loop where cudaMalloc/cudaFree would synchronise the device). It keeps
its scratch in a fixed array inside the library. These tests call it through
the C ABI and check it against cfmm_direct, on two calls in a row, and check
that an oversized request is refused (the size check comes before any CUDA
call: tests/test_failures.py checks it without a GPU). This file is collected
last on purpose."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("green", [False, True])
@pytest.mark.parametrize("dim,ker,kap", [(2, 1, 20.0), (3, 1, 6.0), (2, 0, 0.0), (3, 0, 0.0)])
def test_noalloc_matches_direct_twice(cuda, dim, ker, kap, green):
    """Both layers, with and without the Green's function constants, for all
    four kernels."""
    import torch
    import paper_2509_05458_gb300 as cf
    flags = ker | cf.SLP | cf.DLP | (cf.GREEN_SCALE if green else 0)
    for call, seed in enumerate((1, 2)):          # two calls in a row, different inputs
        g = curve2d(900 + 37 * call, seed=seed, t_half=5.0) if dim == 2 else \
            surface3d(900 + 37 * call, seed=seed, half=3.0, rho0=1.0)
        dens = _t(densities(g.n, seed=seed, nrhs=2, ncomp=2), cuda)
        args = (_t(g.re, cuda), _t(g.im, cuda), _t(g.re, cuda), _t(g.im, cuda))
        nrm = (_t(g.nrm_re, cuda), _t(g.nrm_im, cuda))
        ref = cf.direct(dim, flags, kap, *args, dens, *nrm)
        out = torch.empty((2, g.n), dtype=torch.complex128, device=cuda)
        got = cf.direct_noalloc(dim, flags, kap, *args, dens, out, *nrm)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-12, (call, err)


def test_noalloc_rejects_oversized(cuda):
    import torch
    import paper_2509_05458_gb300 as cf
    m = 40000
    z = torch.zeros((m, 2), dtype=torch.float64, device=cuda)
    d = torch.zeros((1, 1, m), dtype=torch.complex128, device=cuda)
    out = torch.empty((1, m), dtype=torch.complex128, device=cuda)
    with pytest.raises(cf.CfmmError):
        cf.direct_noalloc(2, cf.LAPLACE | cf.SLP, 0.0, z, z, z, z, d, out)
