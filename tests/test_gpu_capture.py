"""Sweeps captured into a CUDA graph.

After one uncaptured call with the same plan (which sets the kernels'
shared-memory limits and allocates the compressed grid's counters), a
jacobi_sweep or jacobi_sweep_compressed call is stream work only: kernel
launches (and, for the compressed grid, a memset), so it can be captured
with torch.cuda.graph in its default (global) capture mode and replayed on
new inputs written into the same buffers.  Every replay is compared with
the oracle bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

SHAPE = (70, 45, 37)
T = 7


def _inputs(dtype, seeds):
    return [inputs.uniform_grid(*SHAPE, seed=s, dtype=torch.float64).to(dtype) for s in seeds]


PLANS = [
    (torch.float64, None),
    (torch.float32, None),
    (torch.float32, (J.KERNEL_TB_REG, 3, 64, 32, 16)),
    (torch.float32, (J.KERNEL_TB_CTA, 2, 16, 8, 8, 0, 256)),
    (torch.float64, (J.KERNEL_TB, 2, 16, 8, 8)),
]


@pytest.mark.parametrize("dtype,plan", PLANS, ids=["f64_default", "f32_default", "f32_reg", "f32_cta", "f64_tb"])
def test_sweep_captured_and_replayed(dtype, plan):
    h = J.Handle(*SHAPE, dtype)
    if plan is not None:
        J.jacobi_set_plan(h, *plan)
    hosts = _inputs(dtype, (61, 62, 63))
    A = hosts[0].cuda()
    B = torch.empty_like(A)
    J.jacobi_sweep(h, A, B, T)  # uncaptured first call
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    A.copy_(hosts[0].cuda())
    with torch.cuda.graph(g):
        out = J.jacobi_sweep(h, A, B, T)
    for x in hosts:
        A.copy_(x.cuda())
        g.replay()
        torch.cuda.synchronize()
        assert J.jacobi_get_status(h) == 0
        assert np.array_equal(out.cpu().numpy(), oracle.jacobi_result(x.numpy(), T))
    h.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_compressed_sweep_captured_and_replayed(dtype):
    h = J.Handle(*SHAPE, dtype)
    J.jacobi_compressed_set_plan(h, 0, 8, 1)
    hosts = _inputs(dtype, (71, 72))
    U = J.compressed_buffer(h)
    J.compressed_view(h, U, 1).copy_(hosts[0].cuda())
    J.jacobi_sweep_compressed(h, U, T, 1)  # uncaptured first call
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pos = J.jacobi_sweep_compressed(h, U, T, 1)
    for x in hosts:
        J.compressed_view(h, U, 1).copy_(x.cuda())
        g.replay()
        torch.cuda.synchronize()
        assert J.jacobi_get_status(h) == 0
        got = J.compressed_view(h, U, pos).cpu().numpy()
        assert np.array_equal(got, oracle.jacobi_result(x.numpy(), T))
    h.close()
