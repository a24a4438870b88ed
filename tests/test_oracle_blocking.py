"""Brute-force agreement of blocked and naive orderings on tiny grids.

The pipelined temporal blocking order of Sect. 2.1 (teams of threads, T
updates per thread, blocks shifted by one cell per update, distances of
Eq. 3) and the multi-layer halo decomposition of Sect. 3.1 reach exactly the
result of plain sweeps, because each cell sees the same operands in the same
order.  Every grid with 1..5 cells per axis is checked bitwise.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs

SHAPES = list(itertools.product(range(1, 6), repeat=3))


def _naive(A, T):
    return oracle.jacobi_result(A, T)


@pytest.mark.parametrize("shape", SHAPES)
def test_pipelined_equals_naive(shape):
    nx, ny, nz = shape
    A0 = inputs.uniform_grid(nx, ny, nz, seed=100 + nx * 36 + ny * 6 + nz).numpy()
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    for _ in range(4):
        T = int(rng.integers(0, 10))
        n_teams = int(rng.integers(1, 3))
        t_team = int(rng.integers(1, 4))
        T_upd = int(rng.integers(1, 3))
        d_l = int(rng.integers(1, 3))
        d_t = int(rng.integers(0, 3))
        bx, by, bz = (int(rng.integers(1, 4)) for _ in range(3))
        exp = _naive(A0, T)
        A = A0.copy()
        B = np.empty_like(A)
        where = oracle.jacobi_pipelined(A, B, T, n_teams, t_team, T_upd, d_l, d_t, bx, by, bz)
        got = A if where == 0 else B
        assert where == T % 2
        assert np.array_equal(got, exp), (shape, T, n_teams, t_team, T_upd, d_l, d_t, bx, by, bz)


@pytest.mark.parametrize("shape", SHAPES)
def test_multihalo_equals_naive(shape):
    nx, ny, nz = shape
    A0 = inputs.uniform_grid(nx, ny, nz, seed=200 + nx * 36 + ny * 6 + nz).numpy()
    rng = np.random.default_rng(7 + nx * 100 + ny * 10 + nz)
    for _ in range(4):
        depths = [int(x) for x in rng.integers(1, 5, size=int(rng.integers(0, 4)))]
        bx, by = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        exp = _naive(A0, sum(depths))
        A = A0.copy()
        B = np.empty_like(A)
        where = oracle.jacobi_multihalo(A, B, depths, bx, by)
        got = A if where == 0 else B
        assert np.array_equal(got, exp), (shape, depths, bx, by)


def test_pipelined_zero_distance_is_rejected():
    # d_l = 0 would let a thread update a block before its predecessor
    # finished it (the race Eq. 3's first condition averts).
    A = inputs.uniform_grid(4, 4, 4, seed=1).numpy()
    with pytest.raises(ValueError):
        oracle.jacobi_pipelined(A, np.empty_like(A), 4, 1, 2, 1, 0, 0, 2, 2, 2)
