"""Host logic of the serving loop, on CPU: the request stream generator, the
memory estimate used for admission, and the latency summary."""
import numpy as np

from paper_2509_05458_gb300.serving import Request, Result, estimate_bytes, make_stream, summarize


def test_stream_is_seeded_and_within_bounds():
    a = make_stream(40, seed=5, rate_hz=10.0, nmin=1000, nmax=50_000, dims=(2, 3), max_matvec=7)
    b = make_stream(40, seed=5, rate_hz=10.0, nmin=1000, nmax=50_000, dims=(2, 3), max_matvec=7)
    assert [r.n for r in a] == [r.n for r in b]
    assert all(np.array_equal(x.pts_re, y.pts_re) for x, y in zip(a, b))
    arr = [r.arrival for r in a]
    assert arr == sorted(arr) and arr[0] > 0
    for r in a:
        assert 1000 <= r.n <= 50_000 and r.dim in (2, 3)
        assert r.eps in (1e-3, 1e-6, 1e-9) and 1 <= len(r.rhs) <= 7
        assert r.pts_re.shape == (r.n, r.dim) and r.rhs[0].shape == (1, r.n)
        helm = (r.kernel & 0xF) == 1
        assert (r.kappa > 0) == helm
        if r.dim == 3:
            assert r.sep == 2 and r.kappa <= 50.0
    assert {r.dim for r in a} == {2, 3}
    # kappa ~ U[1, 50] in both dimensions (no remapping)
    big = make_stream(400, seed=6, rate_hz=10.0, nmin=1000, nmax=2000, dims=(2, 3), max_matvec=1, lazy=True)
    assert max(r.kappa for r in big if r.dim == 3) > 40.0


def test_lazy_stream_materializes_the_same_data():
    a = make_stream(6, seed=8, nmin=1000, nmax=5000, dims=(2, 3), max_matvec=3)
    b = make_stream(6, seed=8, nmin=1000, nmax=5000, dims=(2, 3), max_matvec=3, lazy=True)
    for x, y in zip(a, b):
        assert y.pts_re is None and y.n == x.n and y.nrhs == len(x.rhs)
        y.materialize()
        assert np.array_equal(x.pts_re, y.pts_re) and np.array_equal(x.pts_im, y.pts_im)
        assert all(np.array_equal(p, q) for p, q in zip(x.rhs, y.rhs))
        y.release()
        assert y.pts_re is None


def test_memory_estimate_grows_with_size_and_kernel():
    def req(n, kernel):
        x = np.zeros((n, 2))
        return Request(0, 2, kernel, 1.0, 1e-6, x, x, [np.zeros((1, n), complex)])
    small, big = estimate_bytes(req(1000, 0)), estimate_bytes(req(100_000, 0))
    assert big > small > 0
    assert estimate_bytes(req(100_000, 1)) > big     # Helmholtz tables cost more


def test_memory_estimate_counts_3d_helmholtz_operators():
    """3D Helmholtz plans hold the M2L coaxial operators of a level (more with
    smaller leaves), bounded by the library's per-launch operator budget."""
    def req(n, dim, kernel, leaf):
        x = np.zeros((n, dim))
        return Request(0, dim, kernel, 5.0, 1e-6, x, x, [np.zeros((1, n), complex)], leaf_size=leaf)
    lap, helm = estimate_bytes(req(200_000, 3, 0, 64)), estimate_bytes(req(200_000, 3, 1, 64))
    assert helm - lap > 200_000 * 4500       # the operators on top of the expansions
    assert estimate_bytes(req(200_000, 3, 1, 32)) > helm > estimate_bytes(req(200_000, 3, 1, 256))
    huge = estimate_bytes(req(10_000_000, 3, 1, 16)) - estimate_bytes(req(10_000_000, 3, 0, 16))
    assert huge < 10_000_000 * 2500 + (6 << 30) + (1 << 20)   # operator term capped at 6 GiB
    # 2D plans have no such term
    assert estimate_bytes(req(200_000, 2, 1, 64)) < helm


def test_summary_percentiles_and_errors():
    res = [Result(i, [np.zeros(10, complex)], arrival=0.0, admitted=0.0, done=float(i + 1)) for i in range(100)]
    res.append(Result(100, [], 0.0, 0.0, 1.0, error="CfmmError: cfmm error -1: eps must be in [1e-15, 0.1]"))
    st = summarize(res, wall_s=10.0)
    assert st["requests"] == 101 and st["errors"] == 1
    assert st["error_kinds"] == {"CfmmError: cfmm error -1: eps must be in [1e-15, 0.1]": 1}
    assert st["p50_s"] in (50.0, 51.0) and st["p99_s"] in (99.0, 100.0)
    assert abs(st["mean_s"] - 50.5) < 1e-12
    assert abs(st["points_per_s"] - 100 * 10 / 10.0) < 1e-12
