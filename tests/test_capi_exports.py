"""The C-ABI library builds, loads and exports every function include/feti.h declares (no GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "feti.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(feti_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["feti_create", "feti_solve", "feti_newton", "feti_get_index_maps", "feti_last_error",
              "feti_destroy", "feti_dual_apply"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02599_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == _declared()


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    from feti_inputs import mesh
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    try:
        FetiSolver(mesh.cube_problem(2, (1, 1, 1)))
    except FetiError as e:
        assert e.status == 11
    else:
        raise AssertionError("feti_create must fail without a CUDA device")
