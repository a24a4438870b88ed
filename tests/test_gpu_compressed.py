"""GPU parity of the compressed-grid sweeps (one buffer, shift of S planes
alternating in direction, Sect. 2.1) against the CPU oracle.

Every result is read at the position the call reports and compared bit for
bit with the oracle's two-grid sweeps (FP64; FP32 with the oracle's FP32
loop, plus 1e-5 * max|u| against the FP64 oracle) and with the oracle's
sequential compressed grid.  The buffer cells outside the grid's position
start as NaN, so a read outside the grid would show.  Shapes are ragged
(no tile divides them), odd and even row pitches occur, z chunks are as
small as the plan allows so that many chunks run at once, and sweep counts
leave a shallower last pass.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _input(shape, seed, dtype):
    return inputs.uniform_grid(*shape, seed, dtype=torch.float64).to(dtype)


def _run(shape, dtype, T, plan=None, upper=1, seed=31, a0=None):
    nx, ny, nz = shape
    h = J.Handle(nx, ny, nz, dtype)
    if plan is not None:
        J.jacobi_compressed_set_plan(h, *plan)
    a0 = _input(shape, seed, dtype) if a0 is None else a0
    U = J.compressed_buffer(h)
    U.fill_(float("nan"))
    J.compressed_view(h, U, upper).copy_(a0)
    pos = J.jacobi_sweep_compressed(h, U, T, upper)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    info = J.jacobi_compressed_get_plan(h)
    d = info["depth"]
    passes = 0 if T == 0 else (T + d - 1) // d
    assert pos == upper ^ (passes % 2)
    out = J.compressed_view(h, U, pos).cpu().numpy()
    h.close()
    return out, a0.numpy()


def _check(shape, dtype, T, plan=None, upper=1, seed=31):
    got, a = _run(shape, dtype, T, plan, upper, seed)
    exp = oracle.jacobi_result(a, T)
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, (shape, T, plan, upper, bad[0], got.flat[bad[0]], exp.flat[bad[0]])
    if dtype == torch.float32:
        e64 = oracle.jacobi_result(a.astype(np.float64), T)
        assert np.abs(got.astype(np.float64) - e64).max() <= 1e-5 * max(np.abs(e64).max(), 1e-300)
    return got, a


SHAPES = [(70, 45, 37), (67, 33, 41), (150, 37, 29), (1, 1, 1), (3, 70, 5), (129, 2, 66)]


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_fp32_compressed_every_depth_bitwise(depth):
    bz = 2 * depth + 2  # the smallest chunk: many chunks in flight
    for shape in SHAPES:
        for T in sorted({1, depth, depth + 1, 2 * depth + 1, 3 * depth}):
            for upper in (1, 0):
                _check(shape, torch.float32, T, (depth, bz, 2), upper)


@pytest.mark.parametrize("waves", [1, 2, 3])
def test_fp32_compressed_waves_and_chunks(waves):
    for bz in (8, 13, 64):
        _check((90, 61, 77), torch.float32, 7, (3, bz, waves))


def test_fp64_compressed_bitwise():
    for shape in SHAPES:
        for bz, waves in ((4, 1), (5, 2), (64, 2)):
            for T in (1, 2, 5):
                _check(shape, torch.float64, T, (1, bz, waves), upper=T % 2)


def test_compressed_defaults_zero_sweeps_and_sequential_oracle():
    h = J.Handle(20, 20, 20, torch.float32)
    assert J.jacobi_compressed_get_plan(h) == {"depth": 3, "bz": 128, "waves": 1, "shift_planes": 128 + 3 + 1}
    h.close()
    h = J.Handle(20, 20, 20, torch.float64)
    assert J.jacobi_compressed_get_plan(h) == {"depth": 1, "bz": 64, "waves": 1, "shift_planes": 64 + 1 + 1}
    h.close()
    got, a = _run((40, 30, 50), torch.float32, 0)
    assert np.array_equal(got, a)
    for dt in (torch.float64, torch.float32):
        got, a = _run((33, 18, 40), dt, 6, seed=8)
        assert np.array_equal(got, oracle.jacobi_compressed(a, 6))


def test_compressed_argument_errors():
    L = J.load()
    h = J.Handle(16, 16, 16, torch.float32)
    assert L.jacobi_compressed_set_plan(h.ptr, 3, 7, 2) == -1   # bz < 2*depth + 2
    assert L.jacobi_compressed_set_plan(h.ptr, 5, 64, 2) == -1
    assert L.jacobi_compressed_set_plan(h.ptr, 2, 64, -1) == -1
    assert L.jacobi_compressed_set_plan(h.ptr, 2, 64, 9) == -1
    assert J.jacobi_compressed_get_plan(h)["bz"] == 128        # unchanged by the refused plans
    J.jacobi_compressed_set_plan(h, 2)                          # zero fields: the defaults
    assert J.jacobi_compressed_get_plan(h) == {"depth": 2, "bz": 128, "waves": 1, "shift_planes": 131}
    U = J.compressed_buffer(h)
    assert L.jacobi_sweep_compressed(h.ptr, U.data_ptr(), 3, 2, None, None) == -1
    assert L.jacobi_sweep_compressed(h.ptr, U.data_ptr(), -1, 1, None, None) == -1
    assert L.jacobi_sweep_compressed(h.ptr, U.data_ptr() + 4, 3, 1, None, None) == -8  # JACOBI_ERR_ALIGN
    h64 = J.Handle(16, 16, 16, torch.float64)
    assert L.jacobi_compressed_set_plan(h64.ptr, 2, 64, 2) == -9  # FP64: depth 1 only
    h.close()
    h64.close()


def test_compressed_wait_timeout_reports_status():
    # the first item never reports: the items two chunks on wait, give up
    # after the limit and record JACOBI_ERR_TIMEOUT; no fault, no hang
    shape = (40, 30, 60)
    h = J.Handle(*shape, torch.float32)
    J.jacobi_compressed_set_plan(h, 2, 6, 2)
    a0 = _input(shape, 4, torch.float32)
    U = J.compressed_buffer(h)
    J.compressed_view(h, U, 1).copy_(a0)
    J.jacobi_debug_set_fault(h, 1, 300)
    J.jacobi_sweep_compressed(h, U, 2, 1)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == -5  # JACOBI_ERR_TIMEOUT
    J.jacobi_debug_set_fault(h, 0, 2000)
    J.compressed_view(h, U, 1).copy_(a0)
    pos = J.jacobi_sweep_compressed(h, U, 2, 1)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert np.array_equal(J.compressed_view(h, U, pos).cpu().numpy(), oracle.jacobi_result(a0.numpy(), 2))
    h.close()


def test_fp32_compressed_256cubed_against_oracle():
    # many items in flight (32 chunks of 8 planes, 5 x 10 tiles) over twelve
    # sweeps: every cell against the oracle
    n = 256
    got, a = _run((n, n, n), torch.float32, 12, (3, 8, 2), seed=5)
    assert np.array_equal(got, oracle.jacobi_result(a, 12))
