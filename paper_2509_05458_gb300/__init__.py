"""Python binding of the GB300 complex-coordinate FMM (C ABI in include/cfmm.h).

Argument marshalling only: every step of the method runs in the CUDA library
``libcfmm.so`` built in-tree by ``paper_2509_05458_gb300._build``. There is no
CPU fallback: importing the binding without the built library raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays. Points and normals
are float64 [n, dim] (real and imaginary parts separately); densities are
complex128 [nrhs, ncomp, n] (ncomp = 1 for SLP or DLP, 2 for SLP+DLP, sigma
first); results are complex128 [nrhs, n].
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["LAPLACE", "HELMHOLTZ", "SLP", "DLP", "GREEN_SCALE", "FP64", "MIXED", "AUTO",
           "TOP_FIT", "Plan", "plan", "plan_targets", "Batch", "direct", "direct_noalloc", "lib", "launch_count", "CfmmError", "library_path"]

LAPLACE, HELMHOLTZ = 0, 1
SLP, DLP, GREEN_SCALE = 1 << 4, 1 << 5, 1 << 6
FP64, MIXED, AUTO = 0, 1, 2
TOP_FIT = -1   # top_level: the rule's level, deeper until the 3D Helmholtz order fits the library's limit
# status codes (include/cfmm.h)
OK, EINVAL, ENONFINITE, EGEOM, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libcfmm.so")


class CfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cfmm error {status}: {msg}")
        self.status = status


class _Opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int), ("sep", C.c_int), ("precision", C.c_int),
                ("top_level", C.c_int), ("stream", C.c_void_p)]


class _Info(C.Structure):
    _fields_ = [("dim", C.c_int), ("kernel", C.c_int), ("sep", C.c_int), ("leaf_size", C.c_int),
                ("precision", C.c_int), ("nlevels", C.c_int), ("nboxes", C.c_int), ("nleaves", C.c_int),
                ("l0", C.c_int), ("n", C.c_int64), ("list_len", C.c_int64 * 4), ("p2p_pairs", C.c_int64),
                ("m2l_pairs", C.c_int64), ("root_lo", C.c_double * 3), ("root_width", C.c_double),
                ("lipschitz", C.c_double), ("n_src", C.c_int64), ("n_trg", C.c_int64)]


_lib = None


def lib():
    """The loaded CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        raise ImportError(f"{library_path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(library_path)
    vp, i64, dbl, ci = C.c_void_p, C.c_int64, C.c_double, C.c_int
    L.cfmm_plan.restype = vp
    L.cfmm_plan.argtypes = [ci, ci, dbl, dbl, vp, vp, i64]
    L.cfmm_plan_ex.restype = vp
    L.cfmm_plan_ex.argtypes = [ci, ci, dbl, dbl, vp, vp, vp, vp, i64, C.POINTER(_Opts)]
    L.cfmm_apply_grad.restype = ci
    L.cfmm_apply_grad.argtypes = [vp, vp, ci, vp, vp]
    L.cfmm_plan_targets.restype = vp
    L.cfmm_plan_targets.argtypes = [ci, ci, dbl, dbl, vp, vp, vp, vp, i64, vp, vp, i64, C.POINTER(_Opts)]
    L.cfmm_apply.restype = ci
    L.cfmm_apply.argtypes = [vp, vp, ci, vp]
    L.cfmm_apply_capture.restype = ci
    L.cfmm_apply_capture.argtypes = [vp, vp, ci, vp]
    L.cfmm_apply_replay.restype = ci
    L.cfmm_apply_replay.argtypes = [vp]
    L.cfmm_batch_capture.restype = vp
    L.cfmm_batch_capture.argtypes = [C.POINTER(vp), ci, C.POINTER(vp), C.POINTER(ci), C.POINTER(vp), vp]
    L.cfmm_batch_replay.restype = ci
    L.cfmm_batch_replay.argtypes = [vp]
    L.cfmm_batch_kernels.restype = i64
    L.cfmm_batch_kernels.argtypes = [vp]
    L.cfmm_batch_destroy.restype = ci
    L.cfmm_batch_destroy.argtypes = [vp]
    L.cfmm_debug_fail_allocs.restype = ci
    L.cfmm_debug_fail_allocs.argtypes = [ci]
    L.cfmm_destroy.restype = ci
    L.cfmm_destroy.argtypes = [vp]
    L.cfmm_direct.restype = ci
    L.cfmm_direct.argtypes = [ci, ci, dbl, vp, vp, vp, vp, i64, vp, vp, i64, vp, ci, vp, ci, vp]
    L.cfmm_direct_noalloc.restype = ci
    L.cfmm_direct_noalloc.argtypes = [ci, ci, dbl, vp, vp, vp, vp, i64, vp, vp, i64, vp, ci, vp, vp]
    L.cfmm_plan_get_info.restype = ci
    L.cfmm_plan_get_info.argtypes = [vp, C.POINTER(_Info)]
    L.cfmm_plan_get_orders.restype = ci
    L.cfmm_plan_get_orders.argtypes = [vp, vp, ci]
    L.cfmm_plan_export_tree.restype = ci
    L.cfmm_plan_export_tree.argtypes = [vp] * 11
    L.cfmm_plan_export_list.restype = ci
    L.cfmm_plan_export_list.argtypes = [vp, ci, vp, vp]
    L.cfmm_plan_timings.restype = ci
    L.cfmm_plan_timings.argtypes = [vp, vp, ci]
    L.cfmm_plan_set_timing.restype = ci
    L.cfmm_plan_set_timing.argtypes = [vp, ci]
    L.cfmm_launch_count.restype = i64
    L.cfmm_last_status.restype = ci
    L.cfmm_last_error.restype = C.c_char_p
    L.cfmm_version.restype = C.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        L = lib()
        raise CfmmError(rc, L.cfmm_last_error().decode())
    return rc


def launch_count():
    return int(lib().cfmm_launch_count())


def _ptr(a):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _as_f64(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Plan:
    """A resident plan: sorted points, tree, lists and translation tables on the GPU."""

    def __init__(self, handle, dim, ncomp, n, keep, nsrc=None, nout=None):
        self._h = handle
        self.dim = dim
        self.ncomp = ncomp
        self.n = n                                 # points of the tree
        self.nsrc = n if nsrc is None else nsrc    # densities per component
        self.nout = n if nout is None else nout    # outputs (the separate targets, if any)
        self._keep = keep

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self._h:
            lib().cfmm_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def apply(self, densities, out=None):
        """densities: complex128 [nrhs, ncomp, nsrc] (or [nsrc] / [nrhs, nsrc] when
        ncomp == 1), torch (CUDA or CPU) or numpy. Returns complex128 [nrhs, nout]
        of the same kind (nsrc = nout = n without separate targets)."""
        d = densities
        is_torch = hasattr(d, "data_ptr")
        if is_torch:
            import torch
            if d.dim() == 1:
                d = d.reshape(1, 1, -1)
            elif d.dim() == 2:
                d = d.reshape(d.shape[0], 1, -1) if self.ncomp == 1 else d.reshape(1, *d.shape)
            d = d.to(torch.complex128).contiguous()
            nrhs = d.shape[0]
            if out is None:
                out = torch.empty((nrhs, self.nout), dtype=torch.complex128, device=d.device)
        else:
            d = np.asarray(d, dtype=np.complex128)
            if d.ndim == 1:
                d = d.reshape(1, 1, -1)
            elif d.ndim == 2:
                d = d.reshape(d.shape[0], 1, -1) if self.ncomp == 1 else d.reshape(1, *d.shape)
            d = np.ascontiguousarray(d)
            nrhs = d.shape[0]
            if out is None:
                out = np.empty((nrhs, self.nout), dtype=np.complex128)
        if d.shape[1] != self.ncomp or d.shape[2] != self.nsrc:
            raise ValueError(f"densities must be [nrhs, {self.ncomp}, {self.nsrc}]")
        _check(lib().cfmm_apply(self._h, _ptr(d), nrhs, _ptr(out)))
        return out

    def apply_grad(self, densities, out=None, grad=None, potential=True):
        """cfmm_apply_grad: (potential [nrhs, nout] or None, gradient [nrhs, dim, nout]),
        complex128, of the same kind (torch CUDA/CPU or numpy) as densities."""
        d = densities
        is_torch = hasattr(d, "data_ptr")
        if is_torch:
            import torch
            if d.dim() == 1:
                d = d.reshape(1, 1, -1)
            elif d.dim() == 2:
                d = d.reshape(d.shape[0], 1, -1) if self.ncomp == 1 else d.reshape(1, *d.shape)
            d = d.to(torch.complex128).contiguous()
            nrhs = d.shape[0]
            if potential and out is None:
                out = torch.empty((nrhs, self.nout), dtype=torch.complex128, device=d.device)
            if grad is None:
                grad = torch.empty((nrhs, self.dim, self.nout), dtype=torch.complex128, device=d.device)
        else:
            d = np.asarray(d, dtype=np.complex128)
            if d.ndim == 1:
                d = d.reshape(1, 1, -1)
            elif d.ndim == 2:
                d = d.reshape(d.shape[0], 1, -1) if self.ncomp == 1 else d.reshape(1, *d.shape)
            d = np.ascontiguousarray(d)
            nrhs = d.shape[0]
            if potential and out is None:
                out = np.empty((nrhs, self.nout), dtype=np.complex128)
            if grad is None:
                grad = np.empty((nrhs, self.dim, self.nout), dtype=np.complex128)
        if d.shape[1] != self.ncomp or d.shape[2] != self.nsrc:
            raise ValueError(f"densities must be [nrhs, {self.ncomp}, {self.nsrc}]")
        _check(lib().cfmm_apply_grad(self._h, _ptr(d), nrhs, _ptr(out), _ptr(grad)))
        return out, grad

    def capture(self, densities, out):
        """Record one apply of CUDA tensors (densities [nrhs, ncomp, n] complex128,
        out [nrhs, n]) into a CUDA graph owned by the plan; replay() reruns it.
        The tensors must stay alive and in place while the graph is used."""
        if not (densities.is_cuda and out.is_cuda and densities.is_contiguous() and out.is_contiguous()):
            raise ValueError("capture takes contiguous CUDA tensors")
        self._graph_keep = (densities, out)
        _check(lib().cfmm_apply_capture(self._h, _ptr(densities), densities.shape[0], _ptr(out)))

    def replay(self):
        _check(lib().cfmm_apply_replay(self._h))

    def info(self):
        inf = _Info()
        _check(lib().cfmm_plan_get_info(self._h, C.byref(inf)))
        return {"dim": inf.dim, "kernel": inf.kernel, "sep": inf.sep, "leaf_size": inf.leaf_size,
                "precision": inf.precision, "nlevels": inf.nlevels, "nboxes": inf.nboxes,
                "nleaves": inf.nleaves, "l0": inf.l0, "n": inf.n, "list_len": list(inf.list_len),
                "p2p_pairs": inf.p2p_pairs, "m2l_pairs": inf.m2l_pairs,
                "root_lo": list(inf.root_lo)[: inf.dim], "root_width": inf.root_width,
                "lipschitz": inf.lipschitz, "n_src": inf.n_src, "n_trg": inf.n_trg}

    def orders(self):
        nl = self.info()["nlevels"]
        p = np.zeros(nl, dtype=np.int32)
        _check(lib().cfmm_plan_get_orders(self._h, p.ctypes.data, nl))
        return p

    def export_tree(self):
        inf = self.info()
        nb, n, dim = inf["nboxes"], self.n, self.dim
        perm = np.zeros(n, np.int64)
        keys = np.zeros(n, np.uint64)
        lv = np.zeros(nb, np.int32)
        pre = np.zeros(nb, np.uint64)
        st = np.zeros(nb, np.int32)
        en = np.zeros(nb, np.int32)
        lf = np.zeros(nb, np.int32)
        par = np.zeros(nb, np.int32)
        cre = np.zeros((nb, dim))
        cim = np.zeros((nb, dim))
        _check(lib().cfmm_plan_export_tree(self._h, *[a.ctypes.data for a in
                                                      (perm, keys, lv, pre, st, en, lf, par, cre, cim)]))
        return dict(perm=perm, keys=keys, level=lv, prefix=pre, start=st, end=en, leaf=lf.astype(bool),
                    parent=par, center_re=cre, center_im=cim)

    def export_list(self, which):
        inf = self.info()
        nb = inf["nboxes"]
        off = np.zeros(nb + 1, np.int64)
        ent = np.zeros(max(1, inf["list_len"][which - 1]), np.int32)
        _check(lib().cfmm_plan_export_list(self._h, which, off.ctypes.data, ent.ctypes.data))
        return off, ent[: inf["list_len"][which - 1]]

    def set_timing(self, on=True):
        """0/False: off; 1/True: per-step events (the near field beside the far
        field); 2: serialised (the near field in line, so no step absorbs the
        other stream's kernels)."""
        _check(lib().cfmm_plan_set_timing(self._h, int(on)))

    def timings(self):
        t = np.zeros(9)
        _check(lib().cfmm_plan_timings(self._h, t.ctypes.data, 9))
        return t



class Batch:
    """One CUDA graph over one apply of each of several plans (cfmm_batch_capture).

    members: list of (plan, densities, out) with CUDA tensors as in
    Plan.capture; each plan must have been created with its own (non-default)
    stream. The tensors are kept alive here; replay() reruns every apply, the
    members on different streams concurrently."""

    def __init__(self, members, stream):
        n = len(members)
        for p, d, o in members:
            if not (d.is_cuda and o.is_cuda and d.is_contiguous() and o.is_contiguous()):
                raise ValueError("a batch takes contiguous CUDA tensors")
        self._keep = list(members)
        hp = (C.c_void_p * n)(*[p.handle for p, _, _ in members])
        dp = (C.c_void_p * n)(*[_ptr(d) for _, d, _ in members])
        nr = (C.c_int * n)(*[int(d.shape[0]) for _, d, _ in members])
        op = (C.c_void_p * n)(*[_ptr(o) for _, _, o in members])
        self._stream = stream
        self._h = lib().cfmm_batch_capture(hp, n, dp, nr, op, _stream_ptr(stream))
        if not self._h:
            _check(lib().cfmm_last_status() or -5)

    def replay(self):
        _check(lib().cfmm_batch_replay(self._h))

    @property
    def kernels(self):
        return int(lib().cfmm_batch_kernels(self._h))

    def destroy(self):
        if self._h:
            lib().cfmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

def plan(dim, kernel, k, eps, pts_re, pts_im, nrm_re=None, nrm_im=None, leaf_size=64, sep=1,
         precision=FP64, top_level=0, stream=None):
    """cfmm_plan_ex. kernel: LAPLACE/HELMHOLTZ or-ed with SLP/DLP/GREEN_SCALE."""
    re, im = _as_f64(pts_re), _as_f64(pts_im)
    nre, nim = _as_f64(nrm_re), _as_f64(nrm_im)
    n = int(re.shape[0])
    opts = _Opts(int(leaf_size), int(sep), int(precision), int(top_level), _stream_ptr(stream))
    h = lib().cfmm_plan_ex(int(dim), int(kernel), float(k), float(eps), _ptr(re), _ptr(im),
                           _ptr(nre), _ptr(nim), n, C.byref(opts))
    if not h:
        _check(lib().cfmm_last_status() or -5)
    dlp = bool(kernel & DLP)
    slp = bool(kernel & SLP) or not dlp
    return Plan(h, dim, int(slp) + int(dlp), n, (re, im, nre, nim))


def plan_targets(dim, kernel, k, eps, src_re, src_im, trg_re, trg_im, nrm_re=None, nrm_im=None, leaf_size=64,
                 sep=1, precision=FP64, top_level=0, stream=None):
    """cfmm_plan_targets: the potential of the sources at separate targets (their
    own imaginary parts allowed). apply() takes densities [nrhs, ncomp, m] and
    returns [nrhs, n_targets]."""
    re, im = _as_f64(src_re), _as_f64(src_im)
    tre, tim = _as_f64(trg_re), _as_f64(trg_im)
    nre, nim = _as_f64(nrm_re), _as_f64(nrm_im)
    m, n = int(re.shape[0]), int(tre.shape[0])
    opts = _Opts(int(leaf_size), int(sep), int(precision), int(top_level), _stream_ptr(stream))
    h = lib().cfmm_plan_targets(int(dim), int(kernel), float(k), float(eps), _ptr(re), _ptr(im), _ptr(nre),
                                _ptr(nim), m, _ptr(tre), _ptr(tim), n, C.byref(opts))
    if not h:
        _check(lib().cfmm_last_status() or -5)
    dlp = bool(kernel & DLP)
    slp = bool(kernel & SLP) or not dlp
    return Plan(h, dim, int(slp) + int(dlp), m + n, (re, im, tre, tim, nre, nim), nsrc=m, nout=n)


def direct(dim, kernel, k, src_re, src_im, trg_re, trg_im, densities, nrm_re=None, nrm_im=None,
           precision=FP64, stream=None, out=None):
    """cfmm_direct on CUDA torch tensors. densities complex128 [nrhs, ncomp, m]."""
    import torch
    sr, si, tr, ti = (t.to(torch.float64).contiguous() for t in (src_re, src_im, trg_re, trg_im))
    nr = None if nrm_re is None else nrm_re.to(torch.float64).contiguous()
    ni = None if nrm_im is None else nrm_im.to(torch.float64).contiguous()
    d = densities.to(torch.complex128)
    if d.dim() == 1:
        d = d.reshape(1, 1, -1)
    d = d.contiguous()
    m, n, nrhs = sr.shape[0], tr.shape[0], d.shape[0]
    if out is None:
        out = torch.empty((nrhs, n), dtype=torch.complex128, device=tr.device)
    _check(lib().cfmm_direct(int(dim), int(kernel), float(k), _ptr(sr), _ptr(si), _ptr(nr), _ptr(ni), m,
                             _ptr(tr), _ptr(ti), n, _ptr(d), nrhs, _ptr(out), int(precision),
                             _stream_ptr(stream)))
    return out


def direct_noalloc(dim, kernel, k, src_re, src_im, trg_re, trg_im, densities, out, nrm_re=None, nrm_im=None,
                   stream=None):
    """cfmm_direct_noalloc on CUDA torch tensors: the direct sum without any device
    allocation inside the library (for callers that cannot allocate while they run).
    Points [m or n, dim] float64, densities complex128 [nrhs, ncomp, m], out
    complex128 [nrhs, n], all contiguous CUDA tensors owned by the caller."""
    for t in (src_re, src_im, trg_re, trg_im, densities, out):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("cfmm_direct_noalloc takes contiguous CUDA tensors")
    m, n, nrhs = src_re.shape[0], trg_re.shape[0], densities.shape[0]
    _check(lib().cfmm_direct_noalloc(int(dim), int(kernel), float(k), _ptr(src_re), _ptr(src_im),
                                     _ptr(nrm_re), _ptr(nrm_im), m, _ptr(trg_re), _ptr(trg_im), n,
                                     _ptr(densities), nrhs, _ptr(out), _stream_ptr(stream)))
    return out
