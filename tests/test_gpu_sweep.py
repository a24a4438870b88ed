"""GPU parity of jacobi_sweep against the CPU oracle (through the C ABI).

FP64 must be bit-identical (fixed left-to-right sum, division by 6.0).
FP32 is compared bitwise against the oracle's FP32 loop (same operation
order) and within 1e-5 * max|u| against the FP64 oracle run on the widened
FP32 inputs.
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
    nx, ny, nz = shape
    return inputs.uniform_grid(nx, ny, nz, seed, dtype=torch.float64).to(dtype)


@functools.lru_cache(maxsize=None)
def _expected(shape, seed, dtype, T):
    a = _input(shape, seed, dtype).numpy()
    return oracle.jacobi_result(a, T)


def _gpu(shape, seed, dtype, T, plan=None, A0=None):
    nx, ny, nz = shape
    h = J.Handle(nx, ny, nz, dtype)
    if plan is not None:
        J.jacobi_set_plan(h, *plan)
    A = (A0 if A0 is not None else _input(shape, seed, dtype)).cuda()
    B = torch.full_like(A, float("nan"))
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    h.close()
    return out.cpu().numpy()


SHAPES = [(1, 1, 1), (2, 3, 1), (5, 4, 3), (7, 9, 11), (13, 6, 17), (33, 31, 29), (67, 45, 33)]
PLANS = [
    (J.KERNEL_PLAIN, 1, 32, 8, 8),
    (J.KERNEL_TB, 1, 4, 3, 2),
    (J.KERNEL_TB, 1, 8, 8, 8),
    (J.KERNEL_TB, 1, 64, 16, 64),
    (J.KERNEL_TB, 2, 4, 4, 3),
    (J.KERNEL_TB, 3, 8, 5, 4),
    (J.KERNEL_TB, 4, 16, 8, 7),
    (J.KERNEL_TB, 5, 5, 7, 9),
    (J.KERNEL_TB, 8, 32, 16, 16),
    (J.KERNEL_TB, 8, 3, 3, 2),
    (J.KERNEL_TB, 2, 8, 8, 8, 16),
    (J.KERNEL_TB, 4, 16, 8, 20, 4),
    (J.KERNEL_TB, 1, 32, 8, 16, 8),
    (J.KERNEL_TB, 2, 16, 8, 8, 4, 128),
    (J.KERNEL_TB, 3, 24, 12, 8, 8, 512),
    (J.KERNEL_PLAIN, 1, 64, 4, 1),
    (J.KERNEL_PLAIN, 1, 128, 8, 3),
    (J.KERNEL_PLAIN, 1, 32, 32, 32),
    (J.KERNEL_TB_CTA, 2, 8, 8, 8, 0, 256),
    (J.KERNEL_TB_CTA, 3, 16, 8, 5, 0, 512),
    (J.KERNEL_TB_CTA, 4, 32, 16, 16, 0, 512),
    (J.KERNEL_TB_CTA, 4, 5, 7, 3, 0, 256),
    (J.KERNEL_TB_CTA, 2, 64, 32, 64, 0, 512),
    (J.KERNEL_TB_CTA, 4, 64, 32, 64, 0, 512),
    (J.KERNEL_TB_CTA, 1, 16, 8, 5, 0, 256),
    (J.KERNEL_TB_CTA, 1, 64, 32, 64, 0, 512),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("plan", PLANS, ids=lambda p: "k%d_d%d_%dx%dx%d" % p[:5] + "".join("_%d" % v for v in p[5:]))
def test_fp64_bit_exact_small(shape, plan):
    for T in (1, 2, 3, 7, 12):
        got = _gpu(shape, 11, torch.float64, T, plan)
        exp = _expected(shape, 11, torch.float64, T)
        assert np.array_equal(got, exp), (shape, plan, T, np.abs(got - exp).max())


@pytest.mark.parametrize("shape", [(5, 4, 3), (33, 31, 29), (67, 45, 33)])
@pytest.mark.parametrize("plan", [PLANS[0], PLANS[3], PLANS[6], PLANS[8], PLANS[-1], PLANS[-4]],
                         ids=lambda p: "k%d_d%d_%dx%d" % p[:4])
def test_fp32_bitwise_vs_fp32_oracle_and_tolerance_vs_fp64(shape, plan):
    for T in (1, 4, 9):
        got = _gpu(shape, 12, torch.float32, T, plan)
        exp32 = _expected(shape, 12, torch.float32, T)
        assert np.array_equal(got, exp32), (shape, plan, T)
        a64 = _input(shape, 12, torch.float32).to(torch.float64).numpy()
        exp64 = oracle.jacobi_result(a64, T)
        assert np.abs(got.astype(np.float64) - exp64).max() <= 1e-5 * np.abs(exp64).max()


def test_workload_64cubed_fp64_all_depths():
    # 64^3 interior, interior and halo U[0,1) from seed 1, T = 10
    shape = (64, 64, 64)
    exp = _expected(shape, 1, torch.float64, 10)
    for plan in [None, (J.KERNEL_PLAIN, 1, 0, 0, 0)] + [(J.KERNEL_TB, d, 32, 16, 32) for d in (1, 2, 4, 8)] + \
            [(J.KERNEL_TB_CTA, d, 32, 16, 24, 0, 512) for d in (1, 2, 3, 4)]:
        got = _gpu(shape, 1, torch.float64, 10, plan)
        assert np.array_equal(got, exp), plan


def test_t_zero_is_noop_and_parity():
    shape = (9, 8, 7)
    A0 = _input(shape, 3, torch.float64)
    h = J.Handle(*shape, torch.float64)
    A = A0.cuda()
    B = torch.zeros_like(A)
    assert J.jacobi_sweep(h, A, B, 0) is A
    assert torch.equal(A.cpu(), A0) and torch.count_nonzero(B) == 0
    out = J.jacobi_sweep(h, A, B, 5)
    assert out is B
    halo = torch.ones(A.shape, dtype=torch.bool)
    halo[1:-1, 1:-1, 1:-1] = False
    assert torch.equal(B.cpu()[halo], A0[halo]) and torch.equal(A.cpu()[halo], A0[halo])


def test_argument_errors():
    h = J.Handle(8, 8, 8, torch.float64)
    A = torch.zeros(h.shape, dtype=torch.float64, device="cuda")
    B = torch.zeros_like(A)
    L = J.load()
    s = J._stream(None)
    import ctypes
    pa, pb = ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr())
    assert L.jacobi_sweep(h.ptr, pa, pb, -1, s) == -1
    assert L.jacobi_sweep(h.ptr, pa, pa, 1, s) == -1
    assert L.jacobi_sweep(h.ptr, ctypes.c_void_p(A.data_ptr() + 8), pb, 1, s) == -8
    assert L.jacobi_sweep(h.ptr, pa, ctypes.c_void_p(A.data_ptr() + 16), 1, s) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB, 0, 8, 8, 8, 0, 0) == -1
    assert L.jacobi_set_plan(h.ptr, 9, 1, 8, 8, 8, 0, 0) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB, 1, 8, 8, 8, 5, 0) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB, 1, 8, 8, 8, 4, 96) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB, 8, 512, 512, 8, 0, 0) == -9
    # TB_CTA: depth 1..4, 256 or 512 threads, a bounded widened tile per thread
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CTA, 5, 8, 8, 8, 0, 512) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CTA, 0, 8, 8, 8, 0, 512) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CTA, 2, 8, 8, 8, 0, 128) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CTA, 4, 128, 64, 8, 0, 256) == -9
    # PLAIN: CTA x extent a multiple of 32, at most 1024 threads, planes >= 0
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_PLAIN, 1, 48, 4, 8, 0, 0) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_PLAIN, 1, 64, 32, 8, 0, 0) == -1
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_PLAIN, 1, 32, 8, -1, 0, 0) == -1
    J.jacobi_set_plan(h, J.KERNEL_PLAIN)
    p = J.jacobi_get_plan(h)
    assert (p["kernel"], p["depth"], p["bx"], p["by"], p["bz"]) == (J.KERNEL_PLAIN, 1, 32, 8, 8)
    J.jacobi_set_plan(h, J.KERNEL_TB, 2)
    p = J.jacobi_get_plan(h)
    assert (p["kernel"], p["depth"], p["bx"], p["by"], p["bz"]) == (J.KERNEL_TB, 2, 8, 8, 8)


X2_SHAPES = [(2, 3, 1), (4, 5, 6), (32, 7, 9), (62, 33, 17), (64, 31, 29), (66, 45, 33), (130, 9, 20)]
X2_PLANS = [(J.KERNEL_PLAIN_X2, 1, 32, 1, 1), (J.KERNEL_PLAIN_X2, 1, 32, 8, 16), (J.KERNEL_PLAIN_X2, 1, 64, 4, 3),
            (J.KERNEL_PLAIN_X2, 1, 128, 8, 32)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("shape", X2_SHAPES)
@pytest.mark.parametrize("plan", X2_PLANS, ids=lambda p: "x2_%dx%dx%d" % p[2:5])
def test_two_cells_per_thread_bitwise(shape, plan, dtype):
    # Eq. (1)'s left-to-right order per cell (FP32: packed additions) gives
    # the oracle's bits
    for T in (1, 4, 9):
        got = _gpu(shape, 14, dtype, T, plan)
        assert np.array_equal(got, _expected(shape, 14, dtype, T)), (shape, plan, T)


def test_two_cells_per_thread_needs_even_nx():
    L = J.load()
    for dt in (torch.float64, torch.float32):
        h_odd = J.Handle(9, 8, 8, dt)
        assert L.jacobi_set_plan(h_odd.ptr, J.KERNEL_PLAIN_X2, 1, 32, 8, 8, 0, 0) == -9
    h = J.Handle(10, 8, 8, torch.float32)
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_PLAIN_X2, 1, 48, 8, 8, 0, 0) == -1
    J.jacobi_set_plan(h, J.KERNEL_PLAIN_X2)
    p = J.jacobi_get_plan(h)
    assert (p["kernel"], p["bx"], p["by"], p["bz"]) == (J.KERNEL_PLAIN_X2, 32, 8, 16)


@pytest.mark.parametrize("shape,plan", [((1, 70000, 2), (J.KERNEL_PLAIN, 1, 32, 1, 1)),
                                        ((3, 1, 70001), (J.KERNEL_PLAIN, 1, 32, 1, 1)),
                                        ((40, 3, 65600), (J.KERNEL_PLAIN, 1, 32, 1, 1)),
                                        ((2, 70000, 2), (J.KERNEL_PLAIN_X2, 1, 32, 1, 1)),
                                        ((40, 3, 65600), (J.KERNEL_PLAIN_X2, 1, 32, 1, 1))])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_plain_beyond_65535_row_blocks_or_z_chunks(shape, plan, dt):
    # more (row block, z chunk) pairs than grid y holds: they spill into grid z
    for T in (1, 2):
        got = _gpu(shape, 13, dt, T, plan)
        assert np.array_equal(got, _expected(shape, 13, dt, T)), (shape, T)


def test_bounded_wait_timeout_reports_status_and_context_survives():
    # Failure detection without a fault: the test hook drops one mbarrier
    # arrival; every wait is bounded, so the kernel records TIMEOUT and exits.
    shape = (40, 24, 30)
    h = J.Handle(*shape, torch.float64)
    J.jacobi_set_plan(h, J.KERNEL_TB, 2, 16, 8, 10)
    A = _input(shape, 4, torch.float64).cuda()
    B = torch.zeros_like(A)
    J.jacobi_debug_set_fault(h, 1, 50)
    J.jacobi_sweep(h, A, B, 2)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == -5
    # the context is still usable and the next sweep is exact
    A = _input(shape, 4, torch.float64).cuda()
    out = J.jacobi_sweep(h, A, B, 2)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert np.array_equal(out.cpu().numpy(), _expected(shape, 4, torch.float64, 2))


def test_host_entry_point_matches_oracle():
    shape = (30, 20, 25)
    h = J.Handle(*shape, torch.float64)
    A0 = _input(shape, 6, torch.float64).pin_memory()
    out = torch.empty_like(A0).pin_memory()
    J.jacobi_sweep_host(h, A0, out, 7)
    assert np.array_equal(out.numpy(), _expected(shape, 6, torch.float64, 7))


def test_tuner_picks_a_plan_and_result_is_plan_independent():
    shape = (96, 80, 72)
    h = J.Handle(*shape, torch.float64)
    sa = torch.zeros(h.shape, dtype=torch.float64, device="cuda")
    sb = torch.zeros_like(sa)
    g = J.jacobi_tune(h, sa, sb)
    assert g > 0
    p = J.jacobi_get_plan(h)
    assert p["kernel"] in (J.KERNEL_PLAIN, J.KERNEL_TB, J.KERNEL_PLAIN_X2, J.KERNEL_TB_CTA)
    assert 1 <= p["depth"] <= 16
    got = _gpu(shape, 7, torch.float64, 9)
    assert np.array_equal(got, _expected(shape, 7, torch.float64, 9))
