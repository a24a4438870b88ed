"""Pins for the CPU oracle's Jacobi sweeps (Eq. 1, Sect. 1.1).

Each test checks the oracle against something other than itself: a fixed
point of Eq. (1), the closed-form eigenvalue of a discrete sine mode, a
hand-derived summation-order fixture, the maximum principle, and a dense
Kronecker-sum matrix built independently of the stencil loops.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _linear_field(nx, ny, nz, a, b, c, e, dtype):
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    return (a + b * i + c * j + e * k).astype(dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("T", [1, 2, 5])
def test_linear_integer_field_is_fixed_point(dtype, T):
    # sum of the six neighbours of a linear integer field is exactly 6u
    # (integers < 2^24), and 6u/6 (or 6u*RN(1/6) in FP32) rounds back to u.
    A = _linear_field(7, 5, 6, 3, 2, -1, 5, dtype)
    ref = A.copy()
    r = oracle.jacobi_result(A, T)
    assert np.array_equal(r, ref)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("c", [1.0, 0.5, 3.0, -0.25])
def test_dyadic_constant_is_fixed_point(dtype, c):
    A = np.full((6, 5, 7), c, dtype=dtype)
    r = oracle.jacobi_result(A, 3)
    assert np.array_equal(r, A)


def test_nonlinear_field_is_not_fixed_point():
    # guards the fixed-point tests against an oracle that does nothing
    A = _linear_field(5, 5, 5, 0, 1, 0, 0, np.float64) ** 2
    r = oracle.jacobi_result(A, 1)
    assert not np.array_equal(r, A)
    # discrete Laplacian of i^2 is 2 -> Jacobi adds 2/6 on the interior
    assert np.allclose(r[1:-1, 1:-1, 1:-1], A[1:-1, 1:-1, 1:-1] + 1.0 / 3.0, rtol=0, atol=1e-12)


def _parse_value(tok):
    b = 2.0 ** -53
    return {"0": 0.0, "1": 1.0, "b": b}[tok]


def test_summation_order_golden():
    rows = []
    with open(os.path.join(GOLD, "eq1_term_order.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            rows.append(([_parse_value(x) for x in t[:6]], t[6]))
    assert len(rows) == 7
    closed = {"1/6": 1.0 / 6.0, "(1+2^-52)/6": (1.0 + 2.0 ** -52) / 6.0}
    assert closed["1/6"] != closed["(1+2^-52)/6"]
    for vals, exp in rows:
        A = np.zeros((3, 3, 3))
        A[1, 1, 0], A[1, 1, 2] = vals[0], vals[1]   # i-1, i+1
        A[1, 0, 1], A[1, 2, 1] = vals[2], vals[3]   # j-1, j+1
        A[0, 1, 1], A[2, 1, 1] = vals[4], vals[5]   # k-1, k+1
        r = oracle.jacobi_result(A, 1)
        assert r[1, 1, 1] == closed[exp], (vals, exp, r[1, 1, 1].hex())


def test_division_not_reciprocal_multiply():
    # s/6 and s*RN(1/6) differ for this s; Eq. (1) read as true division.
    s = float.fromhex("0x1.254a19a30774ep+2")
    assert s / 6.0 != s * (1.0 / 6.0)
    A = np.zeros((3, 3, 3))
    A[1, 1, 0] = s
    r = oracle.jacobi_result(A, 1)
    assert r[1, 1, 1] == s / 6.0


def _decay(nx, ny, nz, p, q, r):
    return (math.cos(math.pi * p / (nx + 1)) + math.cos(math.pi * q / (ny + 1))
            + math.cos(math.pi * r / (nz + 1))) / 3.0


@pytest.mark.parametrize("pqr", [(1, 1, 1), (2, 3, 1), (9, 1, 5), (11, 9, 13), (6, 5, 7)])
def test_sine_mode_decays_by_closed_form(pqr):
    # J phi = lambda phi with lambda = (cos(pi p/(nx+1)) + ...)/3 because
    # sin(t(i-1)) + sin(t(i+1)) = 2 cos(t) sin(t i); zero halo.
    nx, ny, nz = 11, 9, 13
    phi = inputs.mode_only_grid(nx, ny, nz, pqr).numpy()
    lam = _decay(nx, ny, nz, *pqr)
    for T in (1, 4, 15):
        u = oracle.jacobi_result(phi, T)
        exp = lam ** T * phi
        err = np.abs(u - exp).max()
        assert err <= 8 * T * 2.0 ** -53 * np.abs(phi).max() + 1e-300, (pqr, T, err)


def test_sine_mode_decay_fp32():
    nx, ny, nz = 15, 12, 10
    pqr = (3, 2, 4)
    phi64 = inputs.mode_only_grid(nx, ny, nz, pqr).numpy()
    phi = phi64.astype(np.float32)
    lam = _decay(nx, ny, nz, *pqr)
    T = 20
    u = oracle.jacobi_result(phi, T).astype(np.float64)
    err = np.abs(u - lam ** T * phi.astype(np.float64)).max()
    assert err <= 8 * T * 2.0 ** -24


def test_maximum_principle():
    A = inputs.uniform_grid(9, 8, 7, seed=11).numpy()
    lo, hi = A.min(), A.max()
    for T in (1, 3, 8):
        u = oracle.jacobi_result(A, T)
        assert u.min() >= lo and u.max() <= hi


def _jacobi_matrix(n):
    """1D path adjacency (neighbours i-1, i+1 within 1..n)."""
    return np.eye(n, k=1) + np.eye(n, k=-1)


def test_dense_kronecker_matrix_agrees():
    # Independent route: u_{t+1} = (Kx + Ky + Kz) u_t / 6 + boundary / 6 with
    # Kronecker sums of 1D adjacency matrices (x fastest in the flat order).
    nx, ny, nz = 4, 3, 5
    A = inputs.uniform_grid(nx, ny, nz, seed=5).numpy()
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    K = (np.kron(np.kron(Iz, Iy), _jacobi_matrix(nx)) + np.kron(np.kron(Iz, _jacobi_matrix(ny)), Ix)
         + np.kron(np.kron(_jacobi_matrix(nz), Iy), Ix))
    bnd = np.zeros((nz, ny, nx))
    bnd[:, :, 0] += A[1:-1, 1:-1, 0]
    bnd[:, :, -1] += A[1:-1, 1:-1, -1]
    bnd[:, 0, :] += A[1:-1, 0, 1:-1]
    bnd[:, -1, :] += A[1:-1, -1, 1:-1]
    bnd[0, :, :] += A[0, 1:-1, 1:-1]
    bnd[-1, :, :] += A[-1, 1:-1, 1:-1]
    v = A[1:-1, 1:-1, 1:-1].reshape(-1).copy()
    for T in range(1, 7):
        v = (K @ v + bnd.reshape(-1)) / 6.0
        u = oracle.jacobi_result(A, T)
        assert np.abs(u[1:-1, 1:-1, 1:-1].reshape(-1) - v).max() < 1e-14


def test_halo_untouched_and_result_parity():
    A = inputs.uniform_grid(6, 5, 4, seed=3).numpy()
    A0 = A.copy()
    B = np.full_like(A, -7.0)
    where = oracle.jacobi(A, B, 3)
    assert where == 1
    halo = np.ones(A.shape, bool)
    halo[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(A[halo], A0[halo])
    assert np.array_equal(B[halo], A0[halo])
    A = A0.copy()
    assert oracle.jacobi(A, np.empty_like(A), 0) == 0
    assert np.array_equal(A, A0)
    with pytest.raises(ValueError):
        oracle.jacobi(A, np.empty_like(A), -1)


def test_fp32_close_to_fp64():
    A64 = inputs.uniform_grid(10, 9, 8, seed=4).numpy()
    A32 = A64.astype(np.float32)
    r64 = oracle.jacobi_result(A32.astype(np.float64), 12)
    r32 = oracle.jacobi_result(A32, 12).astype(np.float64)
    assert np.abs(r64 - r32).max() <= 1e-5 * np.abs(r64).max()
    assert not np.array_equal(r64, r32)
