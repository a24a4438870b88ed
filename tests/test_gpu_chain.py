"""Temporal blocking by a chain of CTAs (the team x T updates product of
Sect. 2.1): a thread-block cluster of c CTAs, each applying t levels of the
register-blocked step and handing its last level to the next CTA through
distributed shared memory, so that one pass applies d = c x t sweeps.

FP32 results must equal the oracle's FP32 loop bit for bit (same operation
order as Eq. 1) on ragged grids for d in {4, 6, 8, 12, 16}, including
passes of uneven depth and passes shallower than the chain (sweep counts
that are not multiples of d); a dropped hand-off must end in a bounded-wait
timeout that leaves the context usable.  FP64 depths 12 and 16 run on the
one-level-per-CTA cluster pipeline (where the device allows such clusters).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


def _run(shape, dtype, plan, T, seed=31):
    a0 = inputs.uniform_grid(*shape, seed=seed, dtype=torch.float64).to(dtype)
    h = J.Handle(*shape, dtype)
    J.jacobi_set_plan(h, *plan)
    A = a0.cuda()
    B = torch.full_like(A, float("nan"))
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    got = out.cpu().numpy()
    h.close()
    return got, oracle.jacobi_result(a0.numpy(), T)


# (depth, CTAs, region height): d up to 15 fits 64 x 32 regions, 16 needs 64 x 64
CHAINS = [(4, 2, 32), (4, 4, 64), (6, 2, 32), (6, 3, 64), (8, 2, 64), (8, 4, 32), (12, 3, 64), (12, 4, 64),
          (16, 4, 64)]


@pytest.mark.parametrize("d,c,by", CHAINS, ids=lambda v: str(v))
@pytest.mark.parametrize("shape", [(150, 70, 45), (67, 131, 29), (3, 2, 40)])
def test_fp32_chain_bitwise(shape, d, c, by):
    plan = (J.KERNEL_TB_CHAIN, d, 64, by, 16, c)
    for T in sorted({1, c - 1, d, d + 1, 2 * d + 3} - {0}):
        got, exp = _run(shape, torch.float32, plan, T)
        bad = np.flatnonzero(got != exp)
        assert bad.size == 0, (shape, plan, T, bad.size)


def test_fp32_chain_dropped_handoff_times_out_and_context_survives():
    shape = (60, 40, 30)
    a0 = inputs.uniform_grid(*shape, seed=4, dtype=torch.float64).to(torch.float32)
    h = J.Handle(*shape, torch.float32)
    J.jacobi_set_plan(h, J.KERNEL_TB_CHAIN, 4, 64, 32, 16, 2)
    A = a0.cuda()
    B = torch.zeros_like(A)
    J.jacobi_debug_set_fault(h, 1, 50)
    J.jacobi_sweep(h, A, B, 4)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == -5  # JACOBI_ERR_TIMEOUT
    A = a0.cuda()
    out = J.jacobi_sweep(h, A, B, 4)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert np.array_equal(out.cpu().numpy(), oracle.jacobi_result(a0.numpy(), 4))


def test_chain_plan_checks():
    L = J.load()
    h = J.Handle(40, 30, 20, torch.float32)
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CHAIN, 8, 64, 64, 16, 1, 0) == -1   # one CTA is no chain
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CHAIN, 17, 64, 64, 16, 4, 0) == -1  # deeper than 4 per CTA
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CHAIN, 16, 64, 32, 16, 4, 0) == -1  # tile height 0
    assert L.jacobi_set_plan(h.ptr, J.KERNEL_TB_CHAIN, 3, 64, 64, 16, 4, 0) == -1   # fewer levels than CTAs
    h64 = J.Handle(40, 30, 20, torch.float64)
    assert L.jacobi_set_plan(h64.ptr, J.KERNEL_TB_CHAIN, 4, 64, 64, 16, 2, 0) == -9  # FP32 only
    J.jacobi_set_plan(h, J.KERNEL_TB_CHAIN, 6)
    p = J.jacobi_get_plan(h)
    assert (p["kernel"], p["depth"], p["bx"], p["by"], p["bz"], p["ring"]) == (J.KERNEL_TB_CHAIN, 6, 64, 64, 20, 2)


@pytest.mark.parametrize("d", [12, 16])
def test_fp64_deep_cluster_pipeline_bitwise(d):
    # one level per CTA: clusters of 12 or 16 CTAs (non-portable sizes)
    shape = (45, 37, 29)
    h = J.Handle(*shape, torch.float64)
    code = J.load().jacobi_set_plan(h.ptr, J.KERNEL_TB, d, 8, 8, 8, 4, 0)
    if code == -9:
        pytest.skip("clusters of %d CTAs are not launchable on this device" % d)
    assert code == 0
    for T in (d, d + 1, 2 * d + 3):
        got, exp = _run(shape, torch.float64, (J.KERNEL_TB, d, 8, 8, 8, 4), T)
        assert np.array_equal(got, exp), (d, T)
