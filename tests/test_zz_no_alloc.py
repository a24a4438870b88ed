"""The allocation-free residual entry point.

jacobi_poisson_residual_noalloc serves callers that may not allocate device
memory themselves or through the library: code whose device memory is owned
entirely by another allocator (a framework's caching pool or a fixed memory
budget), and latency-critical code that cannot accept an allocation's
implicit device synchronisation or its failure under memory pressure.  It
keeps its partial sums in a fixed device array inside the library instead.

Its result is compared with the CPU oracle's residual (r = f - A_h u from
oracle.poisson_residual, norms taken on the host) and with the allocating
entry point jacobi_poisson_residual, within the residual tolerance used
elsewhere in the tests, on consecutive calls that reuse the shared array,
and at the largest accepted number of planes.  This file is named so that
pytest collects it last.
"""
import ctypes

import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # same bound as the residual parity test


def _case(nx, ny, nz, seed):
    f = inputs.normal_rhs(nx, ny, nz, seed=seed)
    u = inputs.uniform_grid(nx, ny, nz, seed=seed + 1)
    return u, f, 1.0 / (max(nx, ny, nz) + 1)


def _oracle_rel(u, f, h):
    r = oracle.poisson_residual(u.numpy(), f.numpy(), h)
    return oracle.norm2(r) / oracle.norm2(f.numpy())


def _check(u, f, h):
    nz, ny, nx = (s - 2 for s in u.shape)
    ud, fd = u.cuda(), f.cuda()
    got = J.jacobi_poisson_residual_noalloc(ud, fd, h)
    exp = _oracle_rel(u, f, h)
    assert abs(got - exp) <= REL_TOL * exp, (got, exp)
    ref = J.jacobi_poisson_residual(J.Handle(nx, ny, nz, torch.float64), ud, fd, h)
    assert abs(got - ref) <= REL_TOL * ref, (got, ref)


def test_noalloc_residual_matches_oracle_twice_in_a_row():
    a, b = _case(24, 27, 22, 31), _case(40, 43, 38, 41)
    _check(*a)  # two calls in a row on different grids
    _check(*b)
    _check(*a)  # and the first grid again after the second one


def test_noalloc_residual_at_the_plane_limit():
    # a thin grid with nz = JACOBI_NOALLOC_MAX_NZ planes: accepted, correct
    _check(*_case(2, 3, 16384, 51))


def test_noalloc_rejects_too_many_planes():
    L = J.load()
    rel = ctypes.c_double()
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    code = L.jacobi_poisson_residual_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, 1,
                                             16385, 0.5, J._stream(None), ctypes.byref(rel))
    assert code == -1
