"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dpvo_ba.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_2208_04726_b300 import ba, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dpvo_ba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpvo_ba_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "dpvo_ba_solve" in names and "dpvo_ba_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(ba.EXPORTS) == names


def test_struct_layouts_match_header():
    assert ctypes.sizeof(ba.Dims) == 36
    assert ctypes.sizeof(ba.Problem) == 64
    assert ctypes.sizeof(ba.Config) == 24


def test_strerror_without_gpu():
    lib = ba.load()
    assert lib.dpvo_ba_strerror(0) == b"ok"
    assert lib.dpvo_ba_strerror(-1) == b"invalid argument"


def test_null_arguments_are_rejected_without_touching_the_gpu():
    lib = ba.load()
    assert lib.dpvo_ba_create(None, None) == ba.EINVAL
    assert lib.dpvo_ba_solve(None, None, None, 1, None) == ba.EINVAL
    assert lib.dpvo_ba_destroy(None) == ba.EINVAL
