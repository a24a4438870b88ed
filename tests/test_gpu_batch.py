"""GPU parity of the batched persistent sweep (one launch, CUDA graph)
against the CPU oracle, grid by grid."""
import numpy as np
import pytest
import torch

import oracle
from paper_1006_3148_gb300 import inputs
from paper_1006_3148_gb300 import jacobi as J

pytestmark = pytest.mark.gpu


def _make(dims, f32, seed):
    hosts = []
    for g, (nx, ny, nz) in enumerate(dims):
        a = inputs.uniform_grid(nx, ny, nz, seed + g)
        hosts.append(a.to(torch.float32) if f32[g] else a)
    return hosts


def _check(b, hosts, Ts, tol_fp64=True):
    A = [h.cuda() for h in hosts]
    B = [torch.full_like(x, float("nan")) for x in A]
    outs = J.jacobi_batch_run(b, A, B)
    torch.cuda.synchronize()
    assert J.jacobi_batch_get_status(b) == 0
    for g, (h, T) in enumerate(zip(hosts, Ts)):
        got = outs[g].cpu().numpy()
        exp = oracle.jacobi_result(h.numpy(), T)
        assert np.array_equal(got, exp), (g, h.dtype, T)
        if h.dtype == torch.float32 and tol_fp64:
            e64 = oracle.jacobi_result(h.to(torch.float64).numpy(), T)
            assert np.abs(got.astype(np.float64) - e64).max() <= 1e-5 * max(np.abs(e64).max(), 1e-300)


def test_small_mixed_batch_all_tiles():
    rng = np.random.default_rng(3)
    n = 14
    dims = [tuple(int(v) for v in rng.integers(1, 25, size=3)) for _ in range(n)]
    f32 = [bool(v) for v in rng.integers(0, 2, size=n)]
    Ts = [int(v) for v in rng.integers(0, 8, size=n)]
    hosts = _make(dims, f32, 40)
    b = J.Batch(dims, [torch.float32 if f else torch.float64 for f in f32], Ts)
    for tile in [(32, 8), (4, 2), (1, 1), (64, 4), (7, 3), (8, 4, 3), (16, 2, 1)]:
        J.jacobi_batch_set_tile(b, *tile)
        _check(b, hosts, Ts)
    b.close()


def test_graph_replay_with_new_inputs():
    dims = [(20, 17, 9), (33, 8, 12), (5, 40, 6)]
    Ts = [5, 6, 3]
    b = J.Batch(dims, [torch.float64, torch.float32, torch.float64], Ts)
    for seed in (1, 2, 3):
        hosts = _make(dims, [False, True, False], 100 * seed)
        _check(b, hosts, Ts)


def test_bounded_wait_timeout_reports_status():
    dims = [(40, 24, 10), (16, 16, 16)]
    Ts = [6, 6]
    b = J.Batch(dims, [torch.float64, torch.float64], Ts)
    J.jacobi_batch_set_tile(b, 8, 8)
    J.jacobi_batch_debug_set_fault(b, 1, 50)
    hosts = _make(dims, [False, False], 7)
    A = [h.cuda() for h in hosts]
    B = [torch.zeros_like(x) for x in A]
    J.jacobi_batch_run(b, A, B)
    torch.cuda.synchronize()
    assert J.jacobi_batch_get_status(b) == -5
    J.jacobi_batch_debug_set_fault(b, 0, 2000)
    _check(b, hosts, Ts)


def test_batch_workload_256_grids_32_to_192():
    # 256 grids, sizes U{32..192} per axis (seed 4), half FP64 / half FP32,
    # interior and halo U[0,1), T = 50 each: every grid against the oracle.
    dims, f32 = inputs.batch_dims(256, seed=4)
    Ts = [50] * 256
    hosts = _make(dims, f32, 1000)
    b = J.Batch(dims, [torch.float32 if f else torch.float64 for f in f32], Ts)
    info = J.jacobi_batch_get_info(b)
    assert info["items"] > 0 and info["blocks"] > 0 and info["bz"] == 0
    _check(b, hosts, Ts)
