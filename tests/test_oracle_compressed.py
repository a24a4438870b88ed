"""Pins of the oracle's compressed grid (Sect. 2.1).

The sequential compressed-grid sweeps keep ONE array, write every result
shifted by (-1,-1,-1) and (+1,+1,+1) on alternate sweeps and reverse the
loops on every second sweep.  The paper's point is that this is exact: the
result must equal plain Jacobi (Eq. 1, two grids) bit for bit.  Pinned by
brute force against the oracle's two-grid sweeps on small grids of every
shape class, by the closed-form decay of a sine mode, and by planted
mistakes (loops not reversed, no shift, halo not carried along) that these
pins must catch.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "jacobi_oracle.c")

SHAPES = [(1, 1, 1), (2, 1, 3), (1, 5, 2), (3, 4, 5), (7, 2, 6), (9, 9, 9), (6, 8, 3)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_compressed_equals_two_grid_jacobi_bitwise(dtype):
    for g, (nx, ny, nz) in enumerate(SHAPES):
        a = inputs.uniform_grid(nx, ny, nz, seed=50 + g).to(dtype).numpy()
        for T in range(0, 10):
            got = oracle.jacobi_compressed(a, T)
            assert got.dtype == a.dtype
            assert np.array_equal(got, oracle.jacobi_result(a, T)), (nx, ny, nz, T)


def test_compressed_sine_mode_decay():
    # phi_{pqr} is an eigenvector of the Jacobi sweep with eigenvalue
    # (cos(p pi/(nx+1)) + cos(q pi/(ny+1)) + cos(r pi/(nz+1))) / 3
    nx, ny, nz = 11, 9, 13
    for pqr in ((1, 1, 1), (2, 3, 1), (9, 1, 5)):
        phi = inputs.mode_only_grid(nx, ny, nz, pqr).numpy()
        lam = sum(math.cos(math.pi * p / (n + 1)) for n, p in zip((nx, ny, nz), pqr)) / 3.0
        for T in (1, 4, 7):
            assert np.abs(oracle.jacobi_compressed(phi, T) - lam ** T * phi).max() <= 64 * 2.0 ** -53


def test_compressed_halo_carried_and_argument_errors():
    a = inputs.uniform_grid(5, 4, 3, seed=9).numpy()
    halo = np.ones(a.shape, bool)
    halo[1:-1, 1:-1, 1:-1] = False
    for T in (1, 2, 3):
        assert np.array_equal(oracle.jacobi_compressed(a, T)[halo], a[halo])
    with pytest.raises(ValueError):
        oracle.jacobi_compressed(a, -1)


# ------------------------------------------------------------ planted mistakes

def _mutant_lib(tmp_path, old, new, name):
    with open(SRC) as fh:
        text = fh.read()
    assert text.count(old) >= 1, name
    mutated = text.replace(old, new, 1)
    c, so = str(tmp_path / (name + ".c")), str(tmp_path / (name + ".so"))
    with open(c, "w") as fh:
        fh.write(mutated)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", so, c, "-lm"], check=True)
    L = ctypes.CDLL(so)
    L.oracle_jacobi_compressed_f64.argtypes = [ctypes.c_void_p] + [ctypes.c_long] * 4
    return L


def _compressed_with(L, a, T):
    nz, ny, nx = (s - 2 for s in a.shape)
    E = np.zeros((nz + 3, ny + 3, nx + 3))
    E[1:, 1:, 1:] = a
    pos = L.oracle_jacobi_compressed_f64(E.ctypes.data, nx, ny, nz, T)
    return E[pos:pos + nz + 2, pos:pos + ny + 2, pos:pos + nx + 2]


def _pins_pass(L):
    for g, (nx, ny, nz) in enumerate(SHAPES):
        a = inputs.uniform_grid(nx, ny, nz, seed=70 + g).numpy()
        for T in (1, 2, 3):
            if not np.array_equal(_compressed_with(L, a, T), oracle.jacobi_result(a, T)):
                return False
    return True


MUTANTS = [
    ("loops_not_reversed", "        const long k = from ? kk : nz + 1 - kk;\n        for (long jj = 0; jj <= ny + 1; ++jj) {\n"
     "            const long j = from ? jj : ny + 1 - jj;",
     "        const long k = kk;\n        for (long jj = 0; jj <= ny + 1; ++jj) {\n            const long j = jj;"),
    ("no_shift", "    const long o = from, w = 1 - from;", "    const long o = from, w = from;"),
    ("halo_not_carried", "                if (is_halo(i, j, k, nx, ny, nz)) {\n                    v = E[EIDX(i + o, j + o, k + o)];",
     "                if (is_halo(i, j, k, nx, ny, nz)) {\n                    continue;"),
    ("shift_in_x_only", "                E[EIDX(i + w, j + w, k + w)] = v;", "                E[EIDX(i + w, j + o, k + o)] = v;"),
]


def test_pins_pass_for_shipped_compressed_oracle(tmp_path):
    L = _mutant_lib(tmp_path, "static void cg_sweep_f64", "static void cg_sweep_f64", "orig")
    assert _pins_pass(L)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_compressed_mutant(tmp_path, name, old, new):
    assert not _pins_pass(_mutant_lib(tmp_path, old, new, name)), name
