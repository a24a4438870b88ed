"""Pins for the oracle's Poisson pieces: residual, plain FP64 Jacobi with a
right-hand side, and mixed-precision refinement.

Independent routes: SciPy's DST-I solves -Lap_h u = f exactly (the 7-point
Laplacian is diagonal in the sine basis), and a single sine mode is an
eigenvector with a closed-form eigenvalue.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs


def _lap_eig(n3, pqr, h):
    return sum((2.0 - 2.0 * math.cos(math.pi * p / (n + 1))) / (h * h) for n, p in zip(n3, pqr))


@pytest.mark.parametrize("pqr", [(1, 1, 1), (3, 2, 5), (7, 6, 8)])
def test_residual_of_sine_mode(pqr):
    nx, ny, nz = 8, 7, 9
    h = 1.0 / 9.0
    phi = inputs.mode_only_grid(nx, ny, nz, pqr).numpy()
    lam = _lap_eig((nx, ny, nz), pqr, h)
    f = lam * phi
    r = oracle.poisson_residual(phi, f, h)
    assert np.abs(r).max() <= 1e-12 * np.abs(f).max()
    r0 = oracle.poisson_residual(phi, np.zeros_like(phi), h)
    assert np.allclose(-r0, f, rtol=0, atol=1e-12 * np.abs(f).max())


def test_dst_solution_has_tiny_residual():
    n = 12
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=5).numpy()
    u = oracle.poisson_dst(f, h)
    rel = oracle.norm2(oracle.poisson_residual(u, f, h)) / oracle.norm2(f)
    assert rel < 1e-13


def test_norm2_matches_numpy():
    x = inputs.uniform_grid(5, 4, 3, seed=2).numpy()
    assert abs(oracle.norm2(x) - np.linalg.norm(x[1:-1, 1:-1, 1:-1])) < 1e-14 * np.linalg.norm(x)


def test_plain_jacobi_error_contracts_at_spectral_radius():
    # Error of Jacobi for -Lap_h u = f shrinks per sweep by at most
    # rho = cos(pi h) (largest |eigenvalue| of J = (cos+cos+cos)/3, p=q=r=1);
    # the slowest mode decays at exactly rho.
    n = 10
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=6).numpy()
    us = oracle.poisson_dst(f, h)
    u = np.zeros_like(f)
    oracle.poisson_jacobi(u, f, h, 200)
    e1 = np.linalg.norm(u - us)
    oracle.poisson_jacobi(u, f, h, 100)
    e2 = np.linalg.norm(u - us)
    rho = math.cos(math.pi * h)
    ratio = (e2 / e1) ** (1.0 / 100)
    assert abs(ratio - rho) < 2e-3


def test_refine_converges_to_dst_solution():
    n = 16
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=5).numpy()
    u = np.zeros_like(f)
    st, outer, rel = oracle.refine(u, f, h, 1e-10, 200, 100)
    assert st == 0 and rel <= 1e-10 and outer >= 2
    rel2 = oracle.norm2(oracle.poisson_residual(u, f, h)) / oracle.norm2(f)
    assert rel2 == rel
    us = oracle.poisson_dst(f, h)
    # ||u-u*||/||u*|| <= kappa * rel with kappa = lam_max/lam_min of A_h
    kappa = (1 + math.cos(math.pi * h)) / (1 - math.cos(math.pi * h))
    assert np.linalg.norm(u - us) / np.linalg.norm(us) <= kappa * 1e-10


def test_refine_stops_at_max_outer():
    n = 8
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=8).numpy()
    u = np.zeros_like(f)
    st, outer, rel = oracle.refine(u, f, h, 1e-30, 5, 3)
    assert st == 1 and outer == 3 and rel > 0
