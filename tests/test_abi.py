"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/p3t.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(p3t_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2007_15432_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("p3t_create", "p3t_destroy", "p3t_build_tree", "p3t_soft_force",
              "p3t_neighbours", "p3t_hard_step", "p3t_kick", "p3t_energy", "p3t_status",
              "p3t_strerror", "p3t_cutoffs"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in sorted(_declared()):
        assert hasattr(lib, n), n


def test_strerror_and_invalid_arguments_without_gpu(lib):
    lib.p3t_strerror.restype = ctypes.c_char_p
    assert lib.p3t_strerror(0) == b"ok"
    assert b"capacity" in lib.p3t_strerror(-3)
    # null context / null params are rejected on the host, before any CUDA call
    assert lib.p3t_create(None, None, 0) == -1
    assert lib.p3t_status(None, None) == -1
    assert lib.p3t_tree_stats(None, None) == -1


def test_binding_imports_and_mirrors_names():
    from paper_2007_15432_gb300 import p3t
    for n in _declared():
        assert hasattr(p3t, n), n


def test_ensemble_descriptor_table():
    """Ensemble host logic: disks laid end to end in the shared arrays."""
    from paper_2007_15432_gb300 import ensemble as EN
    t = EN.descriptor_table([5, 0, 3, 7])
    assert t.tolist() == [[0, 5], [5, 0], [5, 3], [8, 7]]
    assert EN.size_class(512) == 9 and EN.size_class(16383) == 13
