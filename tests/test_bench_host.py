"""Host-side pieces of bench.py that need no GPU: the CPU-oracle baseline
(all cores and one core) on a small workload grid."""
import bench
import oracle


def test_cpu_baseline_reports_all_cores_and_single_thread():
    w = dict(bench.WORKLOADS["fp64_64"])
    r = bench.cpu_oracle_sample(w, 0.2)
    assert r["kind"] == "oracle" and r["unit"] == "GLUP/s" and r["value"] > 0
    assert r["cores"] == oracle.threads()
    assert r["single_thread"]["value"] > 0


def test_oracle_thread_count_does_not_change_results():
    import numpy as np
    from paper_1006_3148_gb300 import inputs
    a0 = inputs.uniform_grid(20, 17, 13, seed=3).numpy()
    n = oracle.threads()
    try:
        oracle.set_threads(1)
        r1 = oracle.jacobi_result(a0.copy(), 5)
        oracle.set_threads(max(2, n))
        r2 = oracle.jacobi_result(a0.copy(), 5)
    finally:
        oracle.set_threads(n)
    assert np.array_equal(r1, r2)
