"""GPU parity of the batched sweeps (CUDA graph; sweep-per-launch engine and
persistent engine) against the CPU oracle, grid by grid."""
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


def _check(b, hosts, Ts, tol_fp64=True, expected=None):
    A = [h.cuda() for h in hosts]
    B = [torch.full_like(x, float("nan")) for x in A]
    outs = J.jacobi_batch_run(b, A, B)
    torch.cuda.synchronize()
    assert J.jacobi_batch_get_status(b) == 0
    for g, (h, T) in enumerate(zip(hosts, Ts)):
        got = outs[g].cpu().numpy()
        exp = expected[g] if expected is not None else oracle.jacobi_result(h.numpy(), T)
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


@pytest.mark.parametrize("kz", [1, 3, 8, 64])
def test_small_mixed_batch_sweep_engine(kz):
    rng = np.random.default_rng(5)
    n = 17
    dims = [tuple(int(v) for v in rng.integers(1, 40, size=3)) for _ in range(n)]
    f32 = [bool(v) for v in rng.integers(0, 2, size=n)]
    Ts = [int(v) for v in rng.integers(0, 9, size=n)]
    hosts = _make(dims, f32, 60)
    b = J.Batch(dims, [torch.float32 if f else torch.float64 for f in f32], Ts)
    J.jacobi_batch_set_engine(b, J.BATCH_SWEEPS, kz)
    assert J.jacobi_batch_get_engine(b) == {"engine": J.BATCH_SWEEPS, "kz": kz}
    _check(b, hosts, Ts)
    b.close()


def test_single_dtype_batches_sweep_engine():
    for dt in (torch.float64, torch.float32):
        dims = [(9, 33, 5), (40, 3, 17), (1, 1, 1)]
        Ts = [4, 7, 2]
        hosts = _make(dims, [dt == torch.float32] * 3, 80)
        b = J.Batch(dims, [dt] * 3, Ts)
        J.jacobi_batch_set_engine(b, J.BATCH_SWEEPS, 4)
        _check(b, hosts, Ts)
        b.close()


def test_batch_source_term_both_engines():
    # Poisson form: FP64 grids with g = h^2 f against the oracle's plain FP64
    # Jacobi with a source; one grid without a source term
    dims = [(12, 10, 9), (7, 15, 6), (20, 4, 11)]
    Ts = [6, 5, 3]
    hg = [1.0 / 11.0, 1.0 / 16.0, 1.0 / 21.0]
    fs = [inputs.normal_rhs(*d, seed=30 + g) for g, d in enumerate(dims)]
    us = [inputs.uniform_grid(*d, seed=40 + g) for g, d in enumerate(dims)]
    exp = [oracle.poisson_jacobi(us[g].numpy().copy(), fs[g].numpy(), hg[g], Ts[g]) for g in range(2)]
    exp.append(oracle.jacobi_result(us[2].numpy(), Ts[2]))
    b = J.Batch(dims, [torch.float64] * 3, Ts)
    for engine in (J.BATCH_SWEEPS, J.BATCH_PERSISTENT):
        if engine == J.BATCH_SWEEPS:
            J.jacobi_batch_set_engine(b, engine, 4)
        else:
            J.jacobi_batch_set_tile(b, 8, 4)
        A = [u.cuda() for u in us]
        B = [torch.full_like(x, float("nan")) for x in A]
        R = [(hg[g] * hg[g] * fs[g]).cuda() for g in range(2)] + [None]
        outs = J.jacobi_batch_run_rhs(b, A, B, R)
        torch.cuda.synchronize()
        for g in range(3):
            assert np.array_equal(outs[g].cpu().numpy(), exp[g]), (engine, g)
    b.close()


def test_engine_selection_and_errors():
    b = J.Batch([(8, 8, 8)], [torch.float64], [2])
    assert J.jacobi_batch_get_engine(b)["engine"] == J.BATCH_SWEEPS
    L = J.load()
    assert L.jacobi_batch_set_engine(b.ptr, 7, 0) == -1
    assert L.jacobi_batch_set_engine(b.ptr, J.BATCH_SWEEPS, -1) == -1
    assert L.jacobi_batch_debug_set_fault(b.ptr, 1, 50) == -9  # hook needs the persistent engine
    J.jacobi_batch_set_tile(b, 8, 8)
    assert J.jacobi_batch_get_engine(b)["engine"] == J.BATCH_PERSISTENT
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
    exp = [oracle.jacobi_result(h.numpy(), T) for h, T in zip(hosts, Ts)]
    assert J.jacobi_batch_get_engine(b)["engine"] == J.BATCH_SWEEPS
    _check(b, hosts, Ts, expected=exp)
    J.jacobi_batch_set_tile(b, 32, 8)  # the persistent engine, same results
    _check(b, hosts, Ts, tol_fp64=False, expected=exp)
    # FP32 grids in blocked passes beside either engine: bit-identical
    for d in (2, 3):
        J.jacobi_batch_set_fp32_depth(b, d)
        _check(b, hosts, Ts, tol_fp64=False, expected=exp)
    J.jacobi_batch_set_engine(b, J.BATCH_SWEEPS, 16)
    _check(b, hosts, Ts, tol_fp64=False, expected=exp)
    b.close()


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_small_mixed_batch_fp32_depth(depth):
    # odd and even row pitches (copy pieces of one and two cells), grids
    # smaller than one region and than the halo margin, T from 0 to 9 so that
    # both pass-count parities and remainder passes occur
    rng = np.random.default_rng(11 + depth)
    n = 19
    dims = [tuple(int(v) for v in rng.integers(1, 90, size=3)) for _ in range(n)]
    dims += [(1, 1, 1), (2, 1, 3), (130, 3, 2), (63, 61, 131)]
    f32 = [bool(v) for v in rng.integers(0, 2, size=n)] + [True] * 4
    Ts = [int(v) for v in rng.integers(0, 10, size=n)] + [3, 0, 5, 2 * depth + 1]
    hosts = _make(dims, f32, 90)
    b = J.Batch(dims, [torch.float32 if f else torch.float64 for f in f32], Ts)
    J.jacobi_batch_set_fp32_depth(b, depth)
    assert J.jacobi_batch_get_fp32_depth(b) == depth
    for engine in (J.BATCH_SWEEPS, J.BATCH_PERSISTENT):
        if engine == J.BATCH_PERSISTENT:
            J.jacobi_batch_set_tile(b, 32, 8)
        else:
            J.jacobi_batch_set_engine(b, engine, 8)
        _check(b, hosts, Ts)
    b.close()


def test_fp32_depth_all_fp32_batch_and_arguments():
    dims = [(33, 20, 17), (64, 64, 64), (5, 70, 9)]
    Ts = [7, 4, 1]
    hosts = _make(dims, [True] * 3, 120)
    b = J.Batch(dims, [torch.float32] * 3, Ts)
    L = J.load()
    assert L.jacobi_batch_set_fp32_depth(b.ptr, 0) == -1
    assert L.jacobi_batch_set_fp32_depth(b.ptr, 5) == -1
    J.jacobi_batch_set_fp32_depth(b, 3)  # no grid left for the engine
    _check(b, hosts, Ts)
    # no source term on the blocked FP32 passes; depth 1 takes it again
    A = [h.cuda() for h in hosts]
    B = [torch.empty_like(x) for x in A]
    R = [torch.zeros_like(x) for x in A]
    with pytest.raises(RuntimeError):
        J.jacobi_batch_run_rhs(b, A, B, R)
    J.jacobi_batch_run_rhs(b, A, B, [None] * 3)
    torch.cuda.synchronize()
    J.jacobi_batch_set_fp32_depth(b, 1)
    J.jacobi_batch_run_rhs(b, A, B, R)
    torch.cuda.synchronize()
    assert J.jacobi_batch_get_status(b) == 0
    b.close()
