"""Full-size parity in the launch configuration the benchmark times.

512^3 FP64, interior U[0,1) (seed 2), halo 0 except the k=0 plane = 1,
T = 100: the whole result grid is compared bitwise with the CPU oracle, for
the tuned plan and for forced depths 1, 2, 4 and 8.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

N, T = 512, 100


@pytest.fixture(scope="module")
def c2():
    A0 = inputs.dirichlet_z0_grid(N, N, N, seed=2)
    exp = oracle.jacobi_result(A0.numpy(), T)
    return A0, exp


def _run(A0, plan):
    h = J.Handle(N, N, N, torch.float64)
    A = A0.cuda()
    B = torch.empty_like(A)
    if plan == "tuned":
        J.jacobi_tune(h, B, torch.empty_like(A))
    elif plan is not None:
        J.jacobi_set_plan(h, *plan)
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    res = out.cpu().numpy()
    del A, B
    torch.cuda.empty_cache()
    return res


@pytest.mark.parametrize("plan", ["tuned", (J.KERNEL_TB_CTA, 4, 64, 32, 64, 0, 512), (J.KERNEL_TB_CTA, 3, 32, 32, 128, 0, 256),
                                  (J.KERNEL_TB_CTA, 1, 64, 32, 64, 0, 512),
                                  (J.KERNEL_TB, 1, 64, 16, 64), (J.KERNEL_TB, 2, 64, 16, 64),
                                  (J.KERNEL_TB, 4, 64, 16, 128), (J.KERNEL_TB, 8, 32, 32, 128)],
                         ids=["tuned", "cta_d4", "cta_d3", "cta_d1", "d1", "d2", "d4", "d8"])
def test_512cubed_fp64_bit_exact(c2, plan):
    A0, exp = c2
    got = _run(A0, plan)
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, "first mismatch at flat index %d: %r vs %r" % (bad[0], got.flat[bad[0]], exp.flat[bad[0]])


def test_512cubed_fp32_chain_bitwise():
    # the same recipe in FP32 through a chain of 2 CTAs of 4 levels each
    # (depth 8 per pass), compared bitwise with the oracle's FP32 loop
    A0 = inputs.dirichlet_z0_grid(N, N, N, seed=2).to(torch.float32)
    exp = oracle.jacobi_result(A0.numpy(), T)
    h = J.Handle(N, N, N, torch.float32)
    J.jacobi_set_plan(h, J.KERNEL_TB_CHAIN, 8, 64, 64, 128, 2)
    A = A0.cuda()
    B = torch.empty_like(A)
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    got = out.cpu().numpy()
    del A, B, out
    torch.cuda.empty_cache()
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, bad.size
