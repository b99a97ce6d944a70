"""The benchmark script's host side, without a GPU: the reference arm (the
oracle) prints one contract line, the roofline arithmetic matches its closed
form, and the traffic record is keyed to the current kernel sources."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "binary_1k", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"] == "binary_1k"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_roofline_closed_forms():
    """Nominal rates: the one-sided bound at the split where both pipes
    saturate, x = 8/11, is 16 / (2 - x/2) = 88/9 pairs/clk/SM; the symmetric
    bound, x = 2/11, is 2 x 16 / (2 - x/2) = 352/21 interactions/clk/SM."""
    bench = _bench()
    one, x1 = bench.pairs_per_sm_clk(False)
    sym, x2 = bench.pairs_per_sm_clk(True)
    assert one == pytest.approx(88.0 / 9.0, rel=2e-3) and x1 == pytest.approx(8 / 11, abs=2e-3)
    assert sym == pytest.approx(352.0 / 21.0, rel=2e-3) and x2 == pytest.approx(2 / 11, abs=2e-3)
    # halving the MUFU rate halves a MUFU-bound split's gain
    slow = {"fp32_lanes_per_clk_sm": 128.0, "mufu_sqrt_per_clk_sm": 8.0,
            "mufu_rcp_per_clk_sm": 8.0}
    assert bench.pairs_per_sm_clk(False, slow)[0] < one


def test_traffic_record_matches_sources():
    bench = _bench()
    with open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")) as f:
        rec = json.load(f)
    if rec["sources_sha256_16"] != bench.pair_sources_sha():
        pytest.skip("the pair kernels changed since the committed ncu launch list "
                    "(bench.py then reports traffic null)")
    cfg = dict(zip(bench.PAIR_CFG_KEYS, [int(v) for v in rec["pair_cfg"].split(",")]))
    assert bench._pair_traffic(rec["workload"], cfg) == rec["dram_bytes_per_launch"]


def test_reference_arm_runs_on_rank_zero_only():
    """Under a multi-rank launch only rank 0 times the oracle and prints; the
    other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "binary_1k", "--steps", "1", "--warmup", "0",
                          "--gpus", "2"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                         env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
