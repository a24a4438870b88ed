"""GPU Poisson pieces against the oracle: plain FP64 Jacobi with a source
term (bitwise), the FP64 residual, and mixed-precision refinement (the
workload: 96^3, h = 1/97, f ~ N(0,1) seed 5, zero halo, relative residual
1e-10 with 500 FP32 inner sweeps per outer step)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


def test_plain_fp64_poisson_jacobi_bit_exact():
    nx, ny, nz = 12, 10, 9
    h = 1.0 / 11.0
    f = inputs.normal_rhs(nx, ny, nz, seed=9)
    u0 = inputs.uniform_grid(nx, ny, nz, seed=10)
    for sweeps in (1, 7, 8):
        H = J.Handle(nx, ny, nz, torch.float64)
        u = u0.cuda()
        tmp = torch.full_like(u, float("nan"))
        out = J.jacobi_poisson_jacobi(H, u, tmp, f.cuda(), h, sweeps)
        torch.cuda.synchronize()
        exp = oracle.poisson_jacobi(u0.numpy().copy(), f.numpy(), h, sweeps)
        assert np.array_equal(out.cpu().numpy(), exp), sweeps


def test_plain_fp64_poisson_jacobi_graph_replays_and_tail_bit_exact():
    # 1025 sweeps: two replays of a 512-sweep graph, then one launch
    nx, ny, nz = 9, 7, 6
    h = 1.0 / 10.0
    f = inputs.normal_rhs(nx, ny, nz, seed=19)
    u0 = inputs.uniform_grid(nx, ny, nz, seed=20)
    H = J.Handle(nx, ny, nz, torch.float64)
    u = u0.cuda()
    tmp = torch.full_like(u, float("nan"))
    out = J.jacobi_poisson_jacobi(H, u, tmp, f.cuda(), h, 1025)
    torch.cuda.synchronize()
    exp = oracle.poisson_jacobi(u0.numpy().copy(), f.numpy(), h, 1025)
    assert out is tmp and np.array_equal(out.cpu().numpy(), exp)


@pytest.mark.parametrize("n", [15, 16])
def test_refine_outer_steps_match_oracle_odd_and_even_nx(n):
    # odd nx runs the scalar FP32 sweep, even nx the two-cells-per-thread one.
    # The residual's 1/h^2 product (the oracle divides by h^2) may move the
    # last bits of the source term, so the outer counts may differ by one.
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n - 1, n - 2, seed=21)
    H = J.Handle(n, n - 1, n - 2, torch.float64)
    u = torch.zeros_like(f).cuda()
    st, outer, rel = J.jacobi_refine(H, u, f.cuda(), h, 1e-10, 60, 100)
    st_o, outer_o, rel_o = oracle.refine(np.zeros_like(f.numpy()), f.numpy(), h, 1e-10, 60, 100)
    assert st == 0 and st_o == 0 and abs(outer - outer_o) <= 1 and rel <= 1e-10
    uh = u.cpu().numpy()
    assert oracle.norm2(oracle.poisson_residual(uh, f.numpy(), h)) / oracle.norm2(f.numpy()) <= 1.01e-10


def test_residual_matches_oracle():
    nx, ny, nz = 20, 18, 16
    h = 1.0 / 21.0
    f = inputs.normal_rhs(nx, ny, nz, seed=11)
    u = inputs.uniform_grid(nx, ny, nz, seed=12)
    H = J.Handle(nx, ny, nz, torch.float64)
    rel = J.jacobi_poisson_residual(H, u.cuda(), f.cuda(), h)
    exp = oracle.norm2(oracle.poisson_residual(u.numpy(), f.numpy(), h)) / oracle.norm2(f.numpy())
    assert abs(rel - exp) <= 1e-12 * exp


def _kappa(n):
    c = math.cos(math.pi / (n + 1))
    return (1 + c) / (1 - c)


def test_refine_small_matches_dst_solution():
    n = 16
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=5)
    H = J.Handle(n, n, n, torch.float64)
    u = torch.zeros_like(f).cuda()
    st, outer, rel = J.jacobi_refine(H, u, f.cuda(), h, 1e-10, 200, 100)
    assert st == 0 and rel <= 1e-10
    uh = u.cpu().numpy()
    rel_cpu = oracle.norm2(oracle.poisson_residual(uh, f.numpy(), h)) / oracle.norm2(f.numpy())
    assert rel_cpu <= 1.01e-10
    us = oracle.poisson_dst(f.numpy(), h)
    assert np.linalg.norm(uh - us) / np.linalg.norm(us) <= _kappa(n) * 1.01e-10
    st_o, outer_o, _ = oracle.refine(np.zeros_like(f.numpy()), f.numpy(), h, 1e-10, 200, 100)
    assert st_o == 0 and abs(outer - outer_o) <= 1


def test_refine_reports_not_converged():
    n = 10
    h = 1.0 / (n + 1)
    f = inputs.normal_rhs(n, n, n, seed=6)
    H = J.Handle(n, n, n, torch.float64)
    u = torch.zeros_like(f).cuda()
    st, outer, rel = J.jacobi_refine(H, u, f.cuda(), h, 1e-30, 5, 2)
    assert st == -7 and outer == 2 and rel > 0


def test_refine_workload_96cubed():
    n = 96
    h = 1.0 / 97.0
    f = inputs.normal_rhs(n, n, n, seed=5)
    H = J.Handle(n, n, n, torch.float64)
    u = torch.zeros_like(f).cuda()
    st, outer, rel = J.jacobi_refine(H, u, f.cuda(), h, 1e-10, 500, 400)
    assert st == 0 and rel <= 1e-10, (st, outer, rel)
    uh = u.cpu().numpy()
    rel_cpu = oracle.norm2(oracle.poisson_residual(uh, f.numpy(), h)) / oracle.norm2(f.numpy())
    assert rel_cpu <= 1.01e-10
    us = oracle.poisson_dst(f.numpy(), h)
    assert np.linalg.norm(uh - us) / np.linalg.norm(us) <= _kappa(n) * 1.01e-10
    # each outer step contracts the error at least by rho^500 of FP32 Jacobi
    rho = math.cos(math.pi / 97)
    assert outer <= math.ceil(math.log(1e-10) / math.log(rho ** 500)) + 8
