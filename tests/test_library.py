"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dpvo_ba.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

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


def test_struct_layouts_match_header(tmp_path):
    """Every binding structure has the size and field offsets the C compiler
    gives the header's structure (a small C program prints them)."""
    pairs = {"dpvo_ba_dims": ba.Dims, "dpvo_ba_problem": ba.Problem, "dpvo_ba_config": ba.Config,
             "dpvo_ba_grads": ba.Grads, "dpvo_ba_pose_loss_problem": ba.PoseLossProblem,
             "dpvo_ba_window_params": ba.WindowParams, "dpvo_ba_corr_dims": ba.CorrDims}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpvo_ba.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for cname, cls in pairs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def test_strerror_without_gpu():
    lib = ba.load()
    assert lib.dpvo_ba_strerror(0) == b"ok"
    assert lib.dpvo_ba_strerror(-1) == b"invalid argument"


def test_null_arguments_are_rejected_without_touching_the_gpu():
    lib = ba.load()
    assert lib.dpvo_ba_create(None, None) == ba.EINVAL
    assert lib.dpvo_ba_solve(None, None, None, 1, None) == ba.EINVAL
    assert lib.dpvo_ba_destroy(None) == ba.EINVAL
