"""The C ABI library loads and exports every function declared in include/cfmm.h
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cfmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    return g.build()


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_error_state(libpath):
    import paper_2509_05458_gb300 as cf
    L = cf.lib()
    assert b"sm_103a" in L.cfmm_version()
    assert L.cfmm_destroy(None) == 0


def test_binding_rejects_bad_arguments_without_gpu(libpath):
    import numpy as np
    import paper_2509_05458_gb300 as cf
    z = np.zeros((4, 2))
    with pytest.raises(cf.CfmmError):
        cf.plan(4, cf.LAPLACE, 0.0, 1e-6, z, z)          # bad dim, rejected before any CUDA call
    with pytest.raises(cf.CfmmError):
        cf.plan(2, cf.HELMHOLTZ, -1.0, 1e-6, z, z)       # k <= 0
    with pytest.raises(cf.CfmmError):
        cf.plan(2, cf.LAPLACE, 0.0, 1.0, z, z)           # eps out of range


def test_binding_declares_every_entry_point(libpath):
    """The ctypes binding sets a result type for every function of the header
    (a missing one would silently truncate 64-bit pointers or sizes)."""
    import paper_2509_05458_gb300 as cf
    src = open(os.path.join(ROOT, "paper_2509_05458_gb300", "__init__.py")).read()
    bound = set(re.findall(r"L\.(cfmm_[a-z0-9_]+)\.restype", src))
    missing = [n for n in _declared() if n not in bound]
    assert not missing, missing
    cf.lib()
