"""FP32 workload parity: 1024^3 with one sine mode (16,16,16), T = 200.

The result of the tuned plan at full size (the size and plan the benchmark
times) is compared element by element with the oracle: bitwise with its
FP32 loop (same operation order, Eq. 1) and within 1e-5 * max|u| of the
FP64 oracle started from the same FP32 values.  Two properties that hold at
any size are checked as well: the maximum principle, and the projection onto
the sine mode, which Jacobi with a zero halo multiplies by lambda per sweep
(lambda = (cos(16 pi/1025) * 3)/3).  The same recipe at 256^3 with the
default plan gets the same checks.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu

PQR = (16, 16, 16)


def _lam(n):
    return sum(math.cos(math.pi * p / (n + 1)) for p in PQR) / 3.0


def _phi_planes(n, device):
    s = inputs.sine_mode_1d(n, PQR[0]).to(device)
    return s


def _projection(u, n):
    """<u, phi> / <phi, phi> in FP64, plane by plane on the device."""
    s = _phi_planes(n, u.device)
    sxy = s[:, None] * s[None, :]
    num = torch.zeros((), dtype=torch.float64, device=u.device)
    for k in range(1, n + 1):
        num += (u[k].to(torch.float64) * sxy).sum() * s[k]
    den = (s * s).sum() ** 3
    return float(num / den)


@pytest.mark.parametrize("n,T,tuned", [(256, 200, False), (1024, 200, True)])
def test_fp32_mode_workload(n, T, tuned):
    A0 = inputs.mode_grid(n, n, n, seed=3, pqr=PQR, dtype=torch.float32, device="cuda")
    lo, hi = float(A0.min()), float(A0.max())
    p0 = _projection(A0, n)
    h = J.Handle(n, n, n, torch.float32)
    B = torch.empty_like(A0)
    if tuned:
        sa = torch.empty_like(A0)
        J.jacobi_tune(h, sa, B)
        del sa
    A = A0.clone()
    out = J.jacobi_sweep(h, A, B, T)
    torch.cuda.synchronize()
    assert J.jacobi_get_status(h) == 0
    assert float(out.min()) >= lo and float(out.max()) <= hi
    pT = _projection(out, n)
    assert abs(pT - _lam(n) ** T * p0) <= 1e-4 * abs(_lam(n) ** T * p0), (pT, _lam(n) ** T * p0)
    a32 = A0.cpu().numpy()
    got = out.cpu().numpy()
    del A, B, out, A0
    torch.cuda.empty_cache()
    # element by element against the oracle's FP32 loop: bitwise
    e32 = oracle.jacobi_result(a32, T)
    bad = np.flatnonzero(got != e32)
    assert bad.size == 0, (bad.size, bad[0], got.flat[bad[0]], e32.flat[bad[0]])
    del e32
    # and against the FP64 oracle from the widened FP32 inputs (in place, to
    # bound host memory at full size)
    a64 = a32.astype(np.float64)
    b64 = np.empty_like(a64)
    e64 = a64 if oracle.jacobi(a64, b64, T) == 0 else b64
    err, scale = 0.0, 0.0
    for k in range(n + 2):
        err = max(err, float(np.abs(got[k].astype(np.float64) - e64[k]).max()))
        scale = max(scale, float(np.abs(e64[k]).max()))
    print("FP32 workload %d^3 T=%d: max|u_fp32 - u_fp64| / max|u_fp64| = %.3e" % (n, T, err / scale))
    assert err <= 1e-5 * scale, err / scale
