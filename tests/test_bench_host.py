"""Host-side pieces of bench.py that need no GPU: the CPU-oracle baseline
(all cores and one core) on a small workload grid, the workloads' config
keys shared by both arms, and the reference arm's line."""
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


def test_every_workload_has_one_config_for_both_arms():
    # both arms build config with the same function of the workload, so the
    # driver's ratio compares like with like
    for key, w in bench.WORKLOADS.items():
        w = dict(w)
        if w["gen"] == "batch":
            c = bench.batch_config(w, 1)
        elif w["gen"] == "poisson":
            c = bench.poisson_config(w, 1)
        else:
            c = bench.grid_config(w, 1)
        assert c["workload"] == w["name"], key
        assert c["parallelism"] == "single"


def test_reference_arm_line_on_a_small_workload(capsys):
    import argparse
    import json
    args = argparse.Namespace(gpus=1, steps=2, warmup=1, impl="reference", workload="fp64_64", cpu_budget=1.0,
                              no_cpu_baseline=False)
    w = dict(bench.WORKLOADS["fp64_64"])
    line = bench.run_reference(args, w)
    assert line["impl"] == "reference" and line["unit"] == "GLUP/s" and line["higher_is_better"] is True
    assert line["config"] == bench.grid_config(w, 1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    json.dumps(line)
