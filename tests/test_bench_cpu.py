"""The benchmark's JSON contract, checked on the CPU: the reference arm (the
oracle on the host cores) on a small grid prints one JSON line with every
key the contract names, and the algorithmic-work helpers count what they
say on a hand-countable system."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--grid", "12", "--steps", "4",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 4 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["iters"] >= 1 and d["relres"] <= 1e-3 * (1 + 1e-6)
    assert "workload" in d["config"]


class _Info:
    def __init__(self, nb, nnzb, nl, nu):
        self.nb, self.nnzb, self.nnzb_lower, self.nnzb_upper = nb, nnzb, nl, nu


def test_work_counts_on_a_hand_counted_system():
    """Two cells joined both ways: 4 blocks, 1 lower, 1 upper."""
    b = _bench_module()
    info = _Info(2, 4, 1, 1)
    # application: 9 values x 8 B per block, 4 B per off-diagonal column,
    # two row-pointer arrays of n + 1, five 24-B vector passes, y written and
    # read back (2 x 3 values x 8 B) per row
    assert b.algorithmic_apply_bytes(info, False) == 4 * 72 + 4 * 2 + 2 * 4 * 3 + 5 * 24 * 2 + 2 * 3 * 8 * 2
    assert b.algorithmic_apply_bytes(info, True) == 4 * 36 + 4 * 2 + 2 * 4 * 3 + 5 * 24 * 2 + 2 * 3 * 4 * 2
    nbytes, fma = b.iteration_work(info, False)
    assert nbytes == 2 * (76 * 4 + 4 * 2) + 2 * (76 * 4 + 4 * 2) + 27 * 24 * 2
    assert fma == 18 * 4 + 18 * 4 + 36 * 2
    nbytes32, fma32 = b.iteration_work(info, True)
    assert nbytes32 < nbytes and fma32 == 18 * 4 + 36 * 2
    jb, jf = b.jacobi_apply_work(info, 1, False)
    assert jf == int(4.5 * 2 + 9 * 1 * 2 + 9 * 2 * 2) and jb > b.algorithmic_apply_bytes(info, False) // 2


def test_work_counts_with_the_product_reuse():
    """The same two cells with the reuse: row 0 has no block left of its
    diagonal (its product is p_0, no block walked), row 1 has no upper block
    (walks its 2 blocks); nothing is stored by the backward sweep."""
    b = _bench_module()
    info = _Info(2, 4, 1, 1)
    info.nnzb_product, info.rows_identity, info.rows_reuse, info.nupdates = 2, 1, 0, 0
    assert b.product_terms(info) == (2, 1, 0)
    # 2 walked blocks, A's row pointers, the walk lengths, one slice's row
    # classes, one added 3-vector
    assert b.product_bytes(info) == 2 * 76 + 4 * 3 + 4 * 2 + 8 + 24
    assert b.kernel_work(info, False)["spmv"] == (2 * 76 + 4 * 3 + 4 * 2 + 8 + 24 + 72 * 2, 9 * 2 + 6 * 2)
    plain = b.algorithmic_apply_bytes(_Info(2, 4, 1, 1), False)
    assert b.algorithmic_apply_bytes(info, False) == plain + 8
    nbytes, fma = b.iteration_work(info, False)
    assert nbytes == 2 * (2 * 76 + 4 * 2 + 4 * 2 + 8 + 24) + 2 * (76 * 4 + 4 * 2 + 8) + 27 * 24 * 2
    assert fma == 18 * 2 + 18 * 4 + 36 * 2
    # a reusing row stores its upper sum in each application
    info.rows_reuse = 1
    assert b.algorithmic_apply_bytes(info, False) == plain + 8 + 24
    # the textbook count of the same iteration: all of A in every product
    assert b.iteration_work(b.PlainInfo(info), False) == b.iteration_work(_Info(2, 4, 1, 1), False)


def test_fp64_fma_peak_is_the_documented_lane_rate():
    b = _bench_module()
    assert np.isclose(b.FP64_FMA_PEAK, 2 * 152 * 2.07e9)


def test_batched_cpu_baseline_runs_one_oracle_process_per_core():
    """The batched workload's oracle baseline on 8 systems and 2 spawned
    processes: every system converges, the line names the cores and the
    sample, and the rate is repeats x systems / the slowest process."""
    code = ("import bench, json; print(json.dumps(bench.cpu_baseline_batched(8, repeats=2, cores=2)))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["kind"] == "oracle" and d["cores"] == 2 and d["unit"] == "solves/s"
    assert d["status_ok"] == 8 and d["iters_mean"] >= 1 and d["value"] > 0
    assert "8 systems" in d["sample"] and "per core" in d["sample"]


def test_serving_cpu_baseline_solves_the_serving_streams_requests():
    """The serving workload's oracle baseline on the first 12 requests over 4
    patterns: every request converges, and the requests are the serving
    stream's (the same pattern draw as the serving leg)."""
    code = ("import bench, json; print(json.dumps(bench.cpu_baseline_serving(4, nreq=12, cores=2)))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["kind"] == "oracle" and d["cores"] == 2 and d["status_ok"] == 12 and d["value"] > 0
    b = _bench_module()
    pick = b.serving_picks(4, 12)
    assert pick.min() >= 0 and pick.max() < 4
    np.testing.assert_array_equal(pick, b.serving_picks(4, 40)[:12])  # a prefix of any longer stream
    assert f"over {len(set(pick.tolist()))} of 4 patterns" in d["sample"]


def test_small_configuration_leg_cases_and_oracle_half():
    """The C1 / C2 leg covers both configurations, both C2 tolerances and the
    library's default order beside the paper's; its oracle half solves C1 in
    natural order to the stopping rule."""
    b = _bench_module()
    cases = b.small_config_cases()
    assert {(c[0], c[2]) for c in cases} == {("C1", 1e-2), ("C2", 1e-2), ("C2", 1e-6)}
    assert {c[3] for c in cases if c[0] == "C2"} == {"colour", "auto"}
    q = cases[0][1]()
    t, res = b.oracle_small(q, 1e-2, "natural", repeats=3)
    assert t > 0 and res.status == 0 and res.iters >= 1 and res.relres <= 1e-2 * (1 + 1e-6)
