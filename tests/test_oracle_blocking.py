"""Brute-force agreement of blocked and naive orderings on tiny grids.

The pipelined temporal blocking order of Sect. 2.1 (teams of threads, T
updates per thread, blocks shifted by one cell per update, distances of
Eq. 3) and the multi-layer halo decomposition of Sect. 3.1 reach exactly the
result of plain sweeps, because each cell sees the same operands in the same
order.  Every grid with 1..9 cells per axis is checked bitwise, with sweep
counts T = 0..12 and blocking depths d in {1, 2, 3, 4, 8} (d = threads per
team x updates per thread for the pipelined order; the depth of each pass
for the multi-layer halo); the sequential compressed grid (Sect. 2.1) is
checked over the same grids.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs

N = range(1, 10)
# (threads per team, updates per thread) giving team depths 1, 2, 3, 4 and 8
TEAM_DEPTHS = [(1, 1), (2, 1), (1, 2), (3, 1), (1, 3), (4, 1), (2, 2), (1, 4), (8, 1), (4, 2), (2, 4)]
PASS_DEPTHS = [1, 2, 3, 4, 8]


def _naive(A, T):
    return oracle.jacobi_result(A, T)


def _grid(nx, ny, nz, base):
    return inputs.uniform_grid(nx, ny, nz, seed=base + nx * 100 + ny * 10 + nz).numpy()


@pytest.mark.parametrize("nx", N)
def test_pipelined_equals_naive(nx):
    for ny, nz in itertools.product(N, N):
        A0 = _grid(nx, ny, nz, 100)
        rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
        for _ in range(3):
            T = int(rng.integers(0, 13))
            n_teams = int(rng.integers(1, 3))
            t_team, T_upd = TEAM_DEPTHS[int(rng.integers(0, len(TEAM_DEPTHS)))]
            d_l = int(rng.integers(1, 3))
            d_t = int(rng.integers(0, 3))
            bx, by, bz = (int(rng.integers(1, 4)) for _ in range(3))
            exp = _naive(A0, T)
            A = A0.copy()
            B = np.empty_like(A)
            where = oracle.jacobi_pipelined(A, B, T, n_teams, t_team, T_upd, d_l, d_t, bx, by, bz)
            got = A if where == 0 else B
            assert where == T % 2
            assert np.array_equal(got, exp), ((nx, ny, nz), T, n_teams, t_team, T_upd, d_l, d_t, bx, by, bz)


@pytest.mark.parametrize("nx", N)
def test_multihalo_equals_naive(nx):
    for ny, nz in itertools.product(N, N):
        A0 = _grid(nx, ny, nz, 200)
        rng = np.random.default_rng(7 + nx * 100 + ny * 10 + nz)
        for _ in range(3):
            depths = []
            while True:  # passes of the listed depths, T = sum <= 12
                d = PASS_DEPTHS[int(rng.integers(0, len(PASS_DEPTHS)))]
                if sum(depths) + d > 12 or rng.random() < 0.2:
                    break
                depths.append(d)
            bx, by = int(rng.integers(1, 4)), int(rng.integers(1, 4))
            exp = _naive(A0, sum(depths))
            A = A0.copy()
            B = np.empty_like(A)
            where = oracle.jacobi_multihalo(A, B, depths, bx, by)
            got = A if where == 0 else B
            assert np.array_equal(got, exp), ((nx, ny, nz), depths, bx, by)


@pytest.mark.parametrize("nx", N)
def test_compressed_equals_naive(nx):
    for ny, nz in itertools.product(N, N):
        A0 = _grid(nx, ny, nz, 300)
        T = (nx + ny + nz) % 13
        assert np.array_equal(oracle.jacobi_compressed(A0, T), _naive(A0, T)), ((nx, ny, nz), T)


def test_pipelined_zero_distance_is_rejected():
    # d_l = 0 would let a thread update a block before its predecessor
    # finished it (the race Eq. 3's first condition averts).
    A = inputs.uniform_grid(4, 4, 4, seed=1).numpy()
    with pytest.raises(ValueError):
        oracle.jacobi_pipelined(A, np.empty_like(A), 4, 1, 2, 1, 0, 0, 2, 2, 2)
