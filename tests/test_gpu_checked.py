"""The bounds-checked build (compiled with -DJACOBI_CHECKED).

Every global, shared and distributed-shared-memory access of the sweep,
batch, compressed-grid and refinement kernels is checked against the buffer it belongs to;
an access outside records JACOBI_ERR_BOUNDS in the status word and is
skipped (no trap).  This stands in for a memory checker.  The checked library is built
beside the normal one (libjacobi_checked.so) and the small-shape parity
suites run against it in a subprocess: every result must still equal the
oracle's and every status word must read 0.  A test hook then declares the
grids one element shorter than they are, so that accesses which are in fact
valid trip the checks: the status must read JACOBI_ERR_BOUNDS, nothing may
fault, and the next sweep must be exact again.
"""
import os
import subprocess
import sys

import pytest

from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED_ENV = dict(os.environ, JACOBI_BUILD_TAG="checked", JACOBI_NVCC_FLAGS="-DJACOBI_CHECKED")


@pytest.fixture(scope="module")
def checked_build():
    r = subprocess.run([sys.executable, "-c", "from paper_1006_3148_gb300 import build; print(build.build())"],
                       env=CHECKED_ENV, cwd=ROOT, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip().endswith("libjacobi_checked.so")
    return r.stdout.strip()


def _run_checked(code):
    r = subprocess.run([sys.executable, "-c", code], env=CHECKED_ENV, cwd=ROOT, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-3000:])
    return r.stdout


def test_normal_build_is_unchecked_and_refuses_the_bounds_hook():
    assert J.load().jacobi_build_checked() == 0
    h = J.Handle(8, 8, 8)
    assert J.load().jacobi_debug_set_fault(h.ptr, 2, 2000) == -9


def test_checked_build_parity_suites_status_zero(checked_build):
    # the small-shape parity tests of every kernel family, the batch engines
    # and refinement, against the checked library (full-size grids and
    # timing tests left out: the checked kernels are slow)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu",
                        "tests/test_gpu_sweep.py", "tests/test_gpu_batch.py", "tests/test_gpu_refine.py",
                        "tests/test_gpu_plans.py", "tests/test_gpu_compressed.py",
                        "-k", "not untuned and not 256cubed and not workload_96cubed and not 65535 and not tuner"],
                       env=CHECKED_ENV, cwd=ROOT, capture_output=True, text=True, timeout=3600)
    assert r.returncode == 0, r.stdout[-4000:]
    assert " passed" in r.stdout


def test_checked_build_reports_out_of_bounds_without_fault(checked_build):
    out = _run_checked(r'''
import numpy as np, torch
import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J
assert J.load().jacobi_build_checked() == 1
shape = (37, 21, 13)
for dt, plan in ((torch.float64, (J.KERNEL_PLAIN, 1, 32, 4, 4)), (torch.float32, (J.KERNEL_TB_REG, 2, 64, 32, 8)),
                 (torch.float64, (J.KERNEL_TB, 2, 16, 8, 8)), (torch.float32, (J.KERNEL_TB_CTA, 2, 16, 8, 8, 0, 256))):
    a0 = inputs.uniform_grid(*shape, seed=5, dtype=torch.float64).to(dt)
    h = J.Handle(*shape, dt)
    J.jacobi_set_plan(h, *plan)
    J.jacobi_debug_set_fault(h, 2, 2000)       # grids declared one element short
    A, B = a0.cuda(), torch.empty_like(a0.cuda())
    J.jacobi_sweep(h, A, B, 3)
    torch.cuda.synchronize()
    st = J.jacobi_get_status(h)
    assert st == -6, (plan, st)                 # JACOBI_ERR_BOUNDS
    J.jacobi_debug_set_fault(h, 0, 2000)
    A = a0.cuda()
    out = J.jacobi_sweep(h, A, B, 3)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert np.array_equal(out.cpu().numpy(), oracle.jacobi_result(a0.numpy(), 3)), plan
dims = [(9, 7, 5), (12, 4, 6)]
b = J.Batch(dims, [torch.float64, torch.float32], [3, 3])
J.jacobi_batch_debug_set_fault(b, 2, 2000)
A = [inputs.uniform_grid(*d, seed=9).to(t).cuda() for d, t in zip(dims, (torch.float64, torch.float32))]
J.jacobi_batch_run(b, A, [torch.empty_like(x) for x in A])
torch.cuda.synchronize()
assert J.jacobi_batch_get_status(b) == -6
for dt, plan in ((torch.float32, (2, 6, 2)), (torch.float64, (1, 4, 2))):
    h = J.Handle(*shape, dt)
    J.jacobi_compressed_set_plan(h, *plan)
    U = J.compressed_buffer(h)
    a0 = inputs.uniform_grid(*shape, seed=6, dtype=torch.float64).to(dt)
    J.compressed_view(h, U, 1).copy_(a0)
    J.jacobi_debug_set_fault(h, 2, 2000)
    J.jacobi_sweep_compressed(h, U, 3, 1)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == -6, dt
    J.jacobi_debug_set_fault(h, 0, 2000)
    J.compressed_view(h, U, 1).copy_(a0)
    pos = J.jacobi_sweep_compressed(h, U, 3, 1)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert np.array_equal(J.compressed_view(h, U, pos).cpu().numpy(), oracle.jacobi_result(a0.numpy(), 3)), dt
print("bounds reported")
''')
    assert "bounds reported" in out
