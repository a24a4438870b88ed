"""Mutation check of the oracle's pins.

Plants plausible mistakes in a private copy of the oracle's C source (a
dropped term, a wrong index, a transposed operand, a reordered sum, a
reciprocal multiply, a missed halo copy), compiles each copy on the CPU and
asserts that at least one pin fails for it.  The shipped oracle is never
modified.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "jacobi_oracle.c")

# (name, original text in sweep_f64/oracle_jacobi_f64, replacement)
MUTANTS = [
    ("drop_k_plus", "s = s + src[IDX(i, j, k + 1)];\n                dst[IDX(i, j, k)] = s / 6.0;",
     "dst[IDX(i, j, k)] = s / 6.0;"),
    ("wrong_index_k", "s = s + src[IDX(i, j, k + 1)];\n                dst[IDX(i, j, k)] = s / 6.0;",
     "s = s + src[IDX(i, j, k - 1)];\n                dst[IDX(i, j, k)] = s / 6.0;"),
    ("transposed_i_j", "double s = src[IDX(i - 1, j, k)];\n                s = s + src[IDX(i + 1, j, k)];\n                s = s + src[IDX(i, j - 1, k)];",
     "double s = src[IDX(j - 1, i, k)];\n                s = s + src[IDX(i + 1, j, k)];\n                s = s + src[IDX(i, j - 1, k)];"),
    ("reordered_sum", "double s = src[IDX(i - 1, j, k)];\n                s = s + src[IDX(i + 1, j, k)];\n                s = s + src[IDX(i, j - 1, k)];\n                s = s + src[IDX(i, j + 1, k)];\n                s = s + src[IDX(i, j, k - 1)];\n                s = s + src[IDX(i, j, k + 1)];\n                dst[IDX(i, j, k)] = s / 6.0;",
     "double s = src[IDX(i, j, k + 1)];\n                s = s + src[IDX(i, j, k - 1)];\n                s = s + src[IDX(i, j + 1, k)];\n                s = s + src[IDX(i, j - 1, k)];\n                s = s + src[IDX(i + 1, j, k)];\n                s = s + src[IDX(i - 1, j, k)];\n                dst[IDX(i, j, k)] = s / 6.0;"),
    ("reciprocal_multiply", "dst[IDX(i, j, k)] = s / 6.0;\n            }\n}\n\nstatic void sweep_f32",
     "dst[IDX(i, j, k)] = s * (1.0 / 6.0);\n            }\n}\n\nstatic void sweep_f32"),
    ("sign_error", "s = s + src[IDX(i, j - 1, k)];\n                s = s + src[IDX(i, j + 1, k)];\n                s = s + src[IDX(i, j, k - 1)];\n                s = s + src[IDX(i, j, k + 1)];\n                dst[IDX(i, j, k)] = s / 6.0;\n            }\n}\n\nstatic void sweep_f32",
     "s = s + src[IDX(i, j - 1, k)];\n                s = s - src[IDX(i, j + 1, k)];\n                s = s + src[IDX(i, j, k - 1)];\n                s = s + src[IDX(i, j, k + 1)];\n                dst[IDX(i, j, k)] = s / 6.0;\n            }\n}\n\nstatic void sweep_f32"),
    ("no_halo_copy", "    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;\n    oracle_halo_copy_f64(A, B, nx, ny, nz);\n    for (long s = 0; s < T; ++s) {\n        if (s % 2 == 0) sweep_f64",
     "    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;\n    for (long s = 0; s < T; ++s) {\n        if (s % 2 == 0) sweep_f64"),
]


def _build(src_text, tmpdir, name):
    c = os.path.join(tmpdir, name + ".c")
    so = os.path.join(tmpdir, name + ".so")
    with open(c, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", so, c, "-lm"], check=True)
    L = ctypes.CDLL(so)
    L.oracle_jacobi_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_long] * 4
    return L


def _run(L, A0, T):
    a = A0.copy()
    b = np.full_like(a, np.nan)
    nz, ny, nx = (s - 2 for s in a.shape)
    w = L.oracle_jacobi_f64(a.ctypes.data, b.ctypes.data, nx, ny, nz, T)
    return a if w == 0 else b


def _pins_pass(L):
    """The pins of test_oracle_jacobi, restated against a given library."""
    # linear integer field fixed point
    k, j, i = np.meshgrid(np.arange(7), np.arange(6), np.arange(8), indexing="ij")
    lin = (3.0 + 2 * i - j + 5 * k).astype(np.float64)
    if not np.array_equal(_run(L, lin, 2), lin):
        return False
    # sine-mode decay
    nx, ny, nz = 11, 9, 13
    for pqr in ((2, 3, 1), (9, 1, 5)):
        phi = inputs.mode_only_grid(nx, ny, nz, pqr).numpy()
        lam = sum(math.cos(math.pi * p / (n + 1)) for n, p in zip((nx, ny, nz), pqr)) / 3.0
        if np.abs(_run(L, phi, 4) - lam ** 4 * phi).max() > 32 * 2.0 ** -53:
            return False
    # summation order fixture (first two lines) and division
    b = 2.0 ** -53
    for vals, exp in (([1, b, b, 0, 0, 0], 1.0 / 6.0), ([b, b, 1, 0, 0, 0], (1 + 2.0 ** -52) / 6.0)):
        A = np.zeros((3, 3, 3))
        A[1, 1, 0], A[1, 1, 2], A[1, 0, 1], A[1, 2, 1], A[0, 1, 1], A[2, 1, 1] = vals
        if _run(L, A, 1)[1, 1, 1] != exp:
            return False
    s = float.fromhex("0x1.254a19a30774ep+2")
    A = np.zeros((3, 3, 3))
    A[1, 1, 0] = s
    if _run(L, A, 1)[1, 1, 1] != s / 6.0:
        return False
    # halo of the result grid equals the input halo (odd T: result in B)
    A = inputs.uniform_grid(4, 3, 5, seed=1).numpy()
    r = _run(L, A, 1)
    halo = np.ones(A.shape, bool)
    halo[1:-1, 1:-1, 1:-1] = False
    return bool(np.array_equal(r[halo], A[halo]))


def test_pins_pass_for_shipped_oracle(tmp_path):
    with open(SRC) as fh:
        assert _pins_pass(_build(fh.read(), str(tmp_path), "orig"))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    with open(SRC) as fh:
        text = fh.read()
    assert text.count(old) >= 1, name
    mutated = text.replace(old, new, 1)
    assert mutated != text
    assert not _pins_pass(_build(mutated, str(tmp_path), name)), name
