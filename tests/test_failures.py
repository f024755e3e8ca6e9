"""Failure detection on the host: every ABI call returns a status, and a
failing call leaves the library usable.

CPU (no GPU touched): argument validation of cfmm_plan_ex, cfmm_apply,
cfmm_batch_capture and the injection hook returns CFMM_EINVAL with a message
before any CUDA call. GPU: NaN points give CFMM_ENONFINITE, injected device
allocation failures give CFMM_ENOMEM from a plan or an apply, and the next
call succeeds with the reference result; in the serving loop a bad request
fails alone while the others complete."""
import ctypes as C

import numpy as np
import pytest

from cfmm_inputs import curve2d, densities


def _lib():
    import paper_2509_05458_gb300 as cf
    try:
        return cf, cf.lib()
    except ImportError:
        pytest.skip("library not built")


EINVAL, ENONFINITE, ENOMEM = -1, -2, -4


def _plan_status(L, cf, dim=2, kernel=None, k=10.0, eps=1e-6, n=8, pts=True, nrm=False, opts=None):
    kernel = cf.HELMHOLTZ | cf.SLP if kernel is None else kernel
    x = np.zeros((max(n, 1), dim))
    p = x.ctypes.data if pts else None
    q = x.ctypes.data if nrm else None
    h = L.cfmm_plan_ex(dim, kernel, k, eps, p, p, q, q, n, C.byref(opts) if opts is not None else None)
    return h, L.cfmm_last_status(), L.cfmm_last_error().decode()


@pytest.mark.parametrize("case", ["dim", "kernel", "flags", "k", "eps_low", "eps_high", "n", "pts", "normals",
                                  "leaf", "sep", "precision"])
def test_plan_rejects_bad_arguments_without_gpu(case):
    cf, L = _lib()
    kw = {}
    if case == "dim":
        kw = dict(dim=4)
    elif case == "kernel":
        kw = dict(kernel=7)
    elif case == "flags":
        kw = dict(kernel=cf.LAPLACE | (1 << 9))
    elif case == "k":
        kw = dict(k=0.0)
    elif case == "eps_low":
        kw = dict(eps=1e-20)
    elif case == "eps_high":
        kw = dict(eps=0.5)
    elif case == "n":
        kw = dict(n=0)
    elif case == "pts":
        kw = dict(pts=False)
    elif case == "normals":
        kw = dict(kernel=cf.HELMHOLTZ | cf.DLP)
    else:
        o = cf._Opts(64, 1, 0, 0, None)
        if case == "leaf":
            o.leaf_size = 5000
        elif case == "sep":
            o.sep = 4
        else:
            o.precision = 7
        kw = dict(opts=o)
    h, st, msg = _plan_status(L, cf, **kw)
    assert not h
    assert st == EINVAL and msg


def test_other_calls_reject_bad_arguments_without_gpu():
    cf, L = _lib()
    out = np.zeros(4)
    assert L.cfmm_apply(None, out.ctypes.data, 1, out.ctypes.data) == EINVAL
    assert "null plan" in L.cfmm_last_error().decode()
    assert L.cfmm_destroy(None) == 0
    assert not L.cfmm_batch_capture(None, 0, None, None, None, None)
    assert L.cfmm_last_status() == EINVAL
    assert L.cfmm_debug_fail_allocs(-1) == EINVAL
    assert L.cfmm_debug_fail_allocs(0) == 0
    # a later valid call clears nothing it should not: the status is per call
    assert L.cfmm_destroy(None) == 0


def test_direct_noalloc_rejects_oversized_without_gpu():
    """cfmm_direct_noalloc checks its sizes and arguments on the host before its
    first CUDA call: with host pointers and no GPU the size limit is what it
    reports."""
    cf, L = _lib()
    m = 40000
    x = np.zeros((m, 2))
    d = np.zeros(2 * m)
    h = x.ctypes.data
    st = L.cfmm_direct_noalloc(2, cf.LAPLACE | cf.SLP, 0.0, h, h, None, None, m, h, h, 8, d.ctypes.data, 1,
                               d.ctypes.data, None)
    assert st == EINVAL
    assert "32768" in L.cfmm_last_error().decode()
    st = L.cfmm_direct_noalloc(4, cf.LAPLACE | cf.SLP, 0.0, h, h, None, None, 8, h, h, 8, d.ctypes.data, 1,
                               d.ctypes.data, None)
    assert st == EINVAL and "dim" in L.cfmm_last_error().decode()


def _geom_dev(cuda, n=3000, seed=5):
    import torch
    g = curve2d(n, seed=seed, t_half=10.0, height=0.5)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    return g, t(g.re), t(g.im)


@pytest.mark.gpu
def test_nonfinite_points(cuda):
    import paper_2509_05458_gb300 as cf
    g, re, im = _geom_dev(cuda)
    im[17, 0] = float("nan")
    with pytest.raises(cf.CfmmError) as e:
        cf.plan(2, cf.HELMHOLTZ | cf.SLP, 10.0, 1e-6, re, im, leaf_size=32)
    assert e.value.status == ENONFINITE


@pytest.mark.gpu
@pytest.mark.parametrize("where", ["plan", "apply"])
def test_injected_allocation_failure_recovers(cuda, where):
    import torch
    import paper_2509_05458_gb300 as cf
    L = cf.lib()
    g, re, im = _geom_dev(cuda)
    d = torch.from_numpy(densities(g.n, seed=2, nrhs=1, ncomp=1)).to(cuda)
    ref_plan = cf.plan(2, cf.HELMHOLTZ | cf.SLP, 10.0, 1e-6, re, im, leaf_size=32)
    ref = ref_plan.apply(d).clone()
    ref_plan.destroy()
    try:
        if where == "plan":
            assert L.cfmm_debug_fail_allocs(1) == 0
            with pytest.raises(cf.CfmmError) as e:
                cf.plan(2, cf.HELMHOLTZ | cf.SLP, 10.0, 1e-6, re, im, leaf_size=32)
            assert e.value.status == ENOMEM
            p = cf.plan(2, cf.HELMHOLTZ | cf.SLP, 10.0, 1e-6, re, im, leaf_size=32)
        else:
            p = cf.plan(2, cf.HELMHOLTZ | cf.SLP, 10.0, 1e-6, re, im, leaf_size=32)
            d3 = torch.from_numpy(densities(g.n, seed=2, nrhs=3, ncomp=1)).to(cuda)
            assert L.cfmm_debug_fail_allocs(1) == 0      # the first apply must allocate its workspaces
            with pytest.raises(cf.CfmmError) as e:
                p.apply(d3)
            assert e.value.status == ENOMEM
    finally:
        L.cfmm_debug_fail_allocs(0)
    got = p.apply(d)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    p.destroy()


@pytest.mark.gpu
def test_serving_bad_request_fails_alone(cuda):
    from paper_2509_05458_gb300.serving import Server, make_stream, summarize
    reqs = make_stream(6, seed=11, rate_hz=500.0, nmin=2000, nmax=8000, max_matvec=2)
    reqs[2].eps = 0.5                      # outside [1e-15, 0.1]
    res = Server(slots=3).run(reqs, realtime=False)
    bad = [r for r in res if r.error]
    assert [r.rid for r in bad] == [reqs[2].rid]
    assert "cfmm error -1" in bad[0].error
    assert all(len(r.outputs) == len(q.rhs) for r, q in zip(res, sorted(reqs, key=lambda q: q.arrival))
               if not r.error)
    st = summarize(res, 1.0)
    assert st["errors"] == 1 and sum(st["error_kinds"].values()) == 1
