"""The allocation-free residual entry point.

jacobi_poisson_residual_noalloc serves callers that may not allocate device
memory themselves or through the library: code whose device memory is owned
entirely by another allocator (a framework's caching pool or a fixed memory
budget), and latency-critical code that cannot accept an allocation's
implicit device synchronisation or its failure under memory pressure.  It
keeps its partial sums in a fixed device array inside the library instead.

Its result must equal, within the residual tolerance used elsewhere in the
tests, that of jacobi_poisson_residual (which allocates scratch on its
handle), and stay correct on consecutive calls that reuse the shared array.
This file is named so that pytest collects it last.
"""
import ctypes

import pytest
import torch

from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # same bound as the residual parity test


def _case(n, seed):
    f = inputs.normal_rhs(n, n + 3, n - 2, seed=seed)
    u = inputs.uniform_grid(n, n + 3, n - 2, seed=seed + 1)
    return u.cuda(), f.cuda(), 1.0 / (n + 1)


def test_noalloc_residual_matches_allocating_entry_point_twice_in_a_row():
    cases = [_case(24, 31), _case(40, 41)]
    for u, f, h in cases:  # two calls in a row, different grids
        nz, ny, nx = (s - 2 for s in u.shape)
        ref = J.jacobi_poisson_residual(J.Handle(nx, ny, nz, torch.float64), u, f, h)
        got = J.jacobi_poisson_residual_noalloc(u, f, h)
        assert abs(got - ref) <= REL_TOL * ref, (got, ref)
    u, f, h = cases[0]  # and the first grid again after the second one
    nz, ny, nx = (s - 2 for s in u.shape)
    ref = J.jacobi_poisson_residual(J.Handle(nx, ny, nz, torch.float64), u, f, h)
    assert abs(J.jacobi_poisson_residual_noalloc(u, f, h) - ref) <= REL_TOL * ref


def test_noalloc_rejects_too_many_planes():
    L = J.load()
    rel = ctypes.c_double()
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    code = L.jacobi_poisson_residual_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, 1,
                                             16385, 0.5, J._stream(None), ctypes.byref(rel))
    assert code == -1
