"""A batch of uneven geometries in one CUDA graph (cfmm_batch_capture): every
member's result equals its own eager apply bit for bit, on the captured
densities and after new densities are written in place, and a replay counts
the graph's kernels."""
import numpy as np
import pytest

from cfmm_inputs import curve2d, surface3d, densities

pytestmark = pytest.mark.gpu


def _members(cf, dev, torch):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    specs = [
        (surface3d(3000, seed=21, half=4.0, amp=0.5, width=1.0, slope=0.3, rho0=1.0), cf.HELMHOLTZ, 3.0, 2, 2),
        (surface3d(1200, seed=22, half=3.0, random_shape=True), cf.HELMHOLTZ, 5.0, 2, 1),
        (surface3d(2500, seed=23, half=4.0, slope=0.3, rho0=1.0), cf.LAPLACE, 0.0, 1, 1),
        (curve2d(6000, seed=24, t_half=20.0, height=0.7), cf.HELMHOLTZ, 15.0, 1, 3),
    ]
    out = []
    for i, (g, ker, kap, sep, nrhs) in enumerate(specs):
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            p = cf.plan(g.dim, ker | cf.SLP, kap, 1e-6, t(g.re), t(g.im), leaf_size=48, sep=sep,
                        precision=cf.MIXED if i % 2 else cf.FP64, stream=s)
        d = t(densities(g.n, seed=30 + i, nrhs=nrhs, ncomp=1))
        out.append((p, s, d, g.n))
    return out


def test_batch_matches_eager_applies(cuda):
    import torch
    import paper_2509_05458_gb300 as cf
    mem = _members(cf, cuda, torch)
    torch.cuda.synchronize()
    refs = []
    for p, s, d, n in mem:
        with torch.cuda.stream(s):
            refs.append(p.apply(d).clone())
    torch.cuda.synchronize()
    main = torch.cuda.Stream(device=cuda)
    bufs = [d.clone() for _, _, d, _ in mem]
    outs = [torch.empty((d.shape[0], n), dtype=torch.complex128, device=cuda) for _, _, d, n in mem]
    torch.cuda.synchronize()
    b = cf.Batch([(p, bufs[i], outs[i]) for i, (p, _, _, _) in enumerate(mem)], main)
    main.synchronize()
    for i in range(len(mem)):
        assert torch.equal(outs[i], refs[i])
    assert b.kernels > 0
    for seed in (7, 8):
        new = [torch.from_numpy(densities(n, seed=seed + 10 * i, nrhs=d.shape[0], ncomp=1)).to(cuda)
               for i, (_, _, d, n) in enumerate(mem)]
        for i, (p, s, _, _) in enumerate(mem):
            with torch.cuda.stream(s):
                refs[i] = p.apply(new[i]).clone()
        torch.cuda.synchronize()
        for i in range(len(mem)):
            bufs[i].copy_(new[i])
            outs[i].zero_()
        torch.cuda.synchronize()
        c0 = cf.launch_count()
        b.replay()
        main.synchronize()
        assert cf.launch_count() - c0 == b.kernels
        for i in range(len(mem)):
            assert torch.equal(outs[i], refs[i])
    b.destroy()
    for p, _, _, _ in mem:
        p.destroy()


def test_batch_rejects_default_stream_plan(cuda):
    import torch
    import paper_2509_05458_gb300 as cf
    g = curve2d(2000, seed=25)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    p = cf.plan(2, cf.LAPLACE | cf.SLP, 0.0, 1e-6, t(g.re), t(g.im), leaf_size=32)
    d = t(densities(g.n, seed=1, ncomp=1))
    o = torch.empty((1, g.n), dtype=torch.complex128, device=cuda)
    with pytest.raises(cf.CfmmError):
        cf.Batch([(p, d, o)], torch.cuda.Stream(device=cuda))
    p.destroy()
