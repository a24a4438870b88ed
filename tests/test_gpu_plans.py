"""Parity of every plan the autotuner can choose, and of the default plans.

The tuner's first-stage candidates for the benchmark workloads (FP64 512^3,
FP32 1024^3) are read through jacobi_tune_candidates and each one is forced
(jacobi_set_plan) on ragged grids whose sizes are not multiples of the
tiles, with sweep counts that leave a remainder pass (T mod d != 0).  Every
result is compared with the CPU oracle: FP64 bit for bit; FP32 bit for bit
with the oracle's FP32 loop (same operation order, Eq. 1) and within
1e-5 * max|u| of the FP64 oracle started from the same FP32 values.

The FP32 workload recipe (sine mode (16,16,16) plus U[0,1) noise, zero
halo, T = 200) is also run at 256^3 with every one-CTA blocked candidate,
and handles that were never tuned must be within 10 % of the tuned speed.
"""
import functools
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@functools.lru_cache(maxsize=None)
def _candidates(n, dtype):
    h = J.Handle(n, n, n, dtype)
    c = J.jacobi_tune_candidates(h)
    h.close()
    return tuple(c)


def _plan_id(p):
    names = {J.KERNEL_PLAIN: "plain", J.KERNEL_TB: "tb", J.KERNEL_PLAIN_X2: "x2", J.KERNEL_TB_CTA: "cta"}
    return "%s_d%d_%dx%dx%d_r%d_t%d" % ((names.get(p[0], str(p[0])),) + tuple(p[1:]))


@functools.lru_cache(maxsize=None)
def _input(shape, seed, dtype):
    nx, ny, nz = shape
    return inputs.uniform_grid(nx, ny, nz, seed, dtype=torch.float64).to(dtype)


@functools.lru_cache(maxsize=None)
def _oracle(shape, seed, dtype, T, wide=False):
    a = _input(shape, seed, dtype).numpy()
    if wide:
        a = a.astype(np.float64)
    return oracle.jacobi_result(a, T)


def _run(shape, A0, T, plan):
    nx, ny, nz = shape
    h = J.Handle(nx, ny, nz, A0.dtype)
    if plan is not None:
        J.jacobi_set_plan(h, *plan)
    A = A0.cuda()
    B = torch.full_like(A, float("nan"))
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    h.close()
    return out.cpu().numpy()


def _check(shape, seed, dtype, T, plan):
    got = _run(shape, _input(shape, seed, dtype), T, plan)
    exp = _oracle(shape, seed, dtype, T)
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, (plan, shape, T, bad[0], got.flat[bad[0]], exp.flat[bad[0]])
    if dtype == torch.float32:
        e64 = _oracle(shape, seed, dtype, T, wide=True)
        assert np.abs(got.astype(np.float64) - e64).max() <= FP32_TOL * np.abs(e64).max()


# Ragged shapes: no tile of the candidate lists divides them; nx even so
# that the two-cells-per-thread kernel is among the candidates.
RAGGED = [(150, 70, 45), (66, 37, 29)]


FAMILIES = [J.KERNEL_PLAIN, J.KERNEL_PLAIN_X2, J.KERNEL_TB_CTA, J.KERNEL_TB, J.KERNEL_TB_REG, J.KERNEL_TB_CHAIN]
FAMILY_IDS = ["plain", "x2", "cta", "tb", "reg", "chain"]
FAMILIES64 = FAMILIES[:4]  # the register-blocked families are FP32 only


# The candidate lists are read inside the tests (they need the GPU), one
# test per kernel family.
@pytest.mark.parametrize("family", FAMILIES, ids=FAMILY_IDS)
def test_fp32_every_tuner_candidate_bitwise(family):
    plans = [p for p in _candidates(1024, torch.float32) if p[0] == family]
    assert plans
    for plan in plans:
        d = plan[1]
        for shape in RAGGED:
            for T in sorted({1, d + 1, 2 * d + 1, 3}):
                _check(shape, 21, torch.float32, T, plan)


@pytest.mark.parametrize("family", FAMILIES64, ids=FAMILY_IDS[:4])
def test_fp64_every_tuner_candidate_bitwise(family):
    plans = [p for p in _candidates(512, torch.float64) if p[0] == family]
    assert plans
    for plan in plans:
        d = plan[1]
        for shape in RAGGED:
            for T in sorted({1, d + 1, 2 * d + 1}):
                _check(shape, 22, torch.float64, T, plan)


# odd row pitch (nx odd): the register-blocked kernel copies single cells
@pytest.mark.parametrize("shape", [(67, 45, 33), (129, 31, 19), (1, 1, 1), (3, 70, 5)])
def test_fp32_register_blocked_candidates_odd_and_tiny(shape):
    plans = [p for p in _candidates(1024, torch.float32) if p[0] == J.KERNEL_TB_REG]
    assert plans
    for plan in plans:
        d = plan[1]
        for T in sorted({1, d + 1, 2 * d + 1}):
            _check(shape, 24, torch.float32, T, plan)


def test_fp64_grids_reject_the_register_blocked_family():
    h = J.Handle(40, 30, 20, torch.float64)
    assert J.load().jacobi_set_plan(h.ptr, J.KERNEL_TB_REG, 2, 64, 32, 16, 0, 0) == -9
    h32 = J.Handle(40, 30, 20, torch.float32)
    L = J.load()
    assert L.jacobi_set_plan(h32.ptr, J.KERNEL_TB_REG, 5, 64, 32, 16, 0, 0) == -1
    assert L.jacobi_set_plan(h32.ptr, J.KERNEL_TB_REG, 2, 96, 32, 16, 0, 0) == -1
    J.jacobi_set_plan(h32, J.KERNEL_TB_REG, 2)
    p = J.jacobi_get_plan(h32)
    assert (p["kernel"], p["bx"], p["by"], p["bz"], p["threads"]) == (J.KERNEL_TB_REG, 64, 32, 20, 128)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (17, 9, 13), (150, 70, 45), (131, 67, 41)])
def test_default_plan_bitwise(shape, dtype):
    for T in (1, 2, 3, 7):
        _check(shape, 23, dtype, T, None)


PQR = (16, 16, 16)


@functools.lru_cache(maxsize=None)
def _mode_case(n, T):
    A0 = inputs.mode_grid(n, n, n, seed=3, pqr=PQR, dtype=torch.float32, device="cpu")
    a32 = A0.numpy()
    return A0, oracle.jacobi_result(a32, T), oracle.jacobi_result(a32.astype(np.float64), T)


def test_fp32_mode_workload_256cubed_every_blocked_candidate():
    # the 1024^3 FP32 workload's recipe at 256^3 (the oracle finishes in
    # seconds), T = 200: the default plan and every one-CTA blocked candidate
    # of the tuner with its 1024^3 z chunk
    n, T = 256, 200
    A0, e32, e64 = _mode_case(n, T)
    plans = [None] + [p for p in _candidates(1024, torch.float32)
                      if p[0] in (J.KERNEL_TB_CTA, J.KERNEL_TB_REG) and p[4] == 128]
    scale = np.abs(e64).max()
    for plan in plans:
        got = _run((n, n, n), A0, T, plan)
        assert np.array_equal(got, e32), plan
        err = np.abs(got.astype(np.float64) - e64).max()
        assert err <= FP32_TOL * scale, (plan, err / scale)


def _glups(h, A, B, T, reps=3):
    J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        t0 = time.perf_counter()
        J.jacobi_sweep(h, A, B, T)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return h.nx * h.ny * h.nz * T / best / 1e9


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_untuned_handle_within_ten_percent_of_tuned(dtype):
    # 512 x 512 x 500: a size no other test tunes (tuned plans are cached per
    # process by grid size, and every untuned handle of a tuned size uses them)
    nx, ny, nz, T = 512, 512, 500, 40
    A = inputs.uniform_grid(nx, ny, nz, seed=2, dtype=torch.float64, device="cuda").to(dtype)
    B = torch.empty_like(A)
    h0 = J.Handle(nx, ny, nz, dtype)
    plan0 = J.jacobi_get_plan(h0)
    g_default = _glups(h0, A, B, T)
    h1 = J.Handle(nx, ny, nz, dtype)
    J.jacobi_tune(h1, torch.empty_like(A), torch.empty_like(A))
    g_tuned = _glups(h1, A, B, T)
    assert g_default >= 0.9 * g_tuned, (g_default, g_tuned, plan0, J.jacobi_get_plan(h1))
