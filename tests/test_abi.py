"""The C-ABI library loads and exports every entry point include/*.h
declares; host-only logic (pass planning, status strings, argument checks)
works without a GPU."""
import ctypes
import glob
import os
import re

import pytest
import torch

from paper_1006_3148_gb300 import build, jacobi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(jacobi_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = ctypes.CDLL(build.LIB)
    names = _declared_functions()
    assert "jacobi_sweep" in names and "jacobi_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_version():
    L = jacobi.load()
    assert L.jacobi_version() >= 10000
    for code in range(-9, 1):
        assert jacobi.jacobi_status_string(code) != "unknown status"
    assert jacobi.jacobi_status_string(-123) == "unknown status"


@pytest.mark.parametrize("T", list(range(0, 41)))
@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 16])
def test_pass_planning(T, d):
    depths = jacobi.jacobi_plan_passes(T, d)
    assert sum(depths) == T
    assert all(1 <= x <= d for x in depths)
    assert len(depths) % 2 == T % 2   # result lands where single sweeps put it
    if T:
        import math
        assert len(depths) <= math.ceil(T / d) + 1
        assert max(depths) - min(depths) <= 1


def test_pass_planning_rejects_bad_arguments():
    L = jacobi.load()
    buf = (ctypes.c_int * 4)()
    assert L.jacobi_plan_passes(-1, 2, buf, 4) == -1
    assert L.jacobi_plan_passes(5, 0, buf, 4) == -1
    assert L.jacobi_plan_passes(100, 1, buf, 4) == -1


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    L = jacobi.load()
    h = ctypes.c_void_p(1)
    assert L.jacobi_create(ctypes.byref(h), 0, 4, 4, 0) == -1
    assert h.value is None
    assert L.jacobi_create(ctypes.byref(h), 4, 4, 4, 7) == -2
    assert L.jacobi_create(None, 4, 4, 4, 0) == -1
    assert L.jacobi_destroy(None) == 0
    assert L.jacobi_sweep(None, None, None, 1, None) == -1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error():
    L = jacobi.load()
    h = ctypes.c_void_p()
    assert L.jacobi_create(ctypes.byref(h), 4, 4, 4, 0) == -4
    assert L.jacobi_last_cuda_error() != b""
