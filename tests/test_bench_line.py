"""Host-side pieces of bench.py's JSON line (no GPU): the summary each extra
workload contributes to the default run's line, the list of extra workloads,
and the roofline traffic lookup."""
import bench


def _line(**over):
    d = {"value": 1.0e9, "unit": "ant-steps/s", "ms_per_step": 12.5, "steps": 1, "warmup": 3,
         "instances_per_s": 4.0, "fallback_fraction": 0.03, "gpu_launches": 7,
         "config": {"workload": "x", "ants_per_warp": 2, "fused": 1, "cluster_log2": 1, "fallback_list": 32,
                    "warps_per_block": 0, "parts": 0, "description": "dropped"},
         "roofline": {"kernel": "k", "achieved": 10.0, "peak": 100.0, "unit": "GB/s", "frac": 0.1, "traffic": None},
         "e2e": {"value": 0.9e9, "unit": "ant-steps/s", "h2d_bytes_per_step": 5},
         "plain_gpu": {"value": 1.0e7, "unit": "ant-steps/s", "speedup_of_batched": 100.0, "sample": "dropped"},
         "latency_model": {"critical_share": 0.9, "note": "dropped"},
         "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9}}
    d.update(over)
    return d


def test_side_summary_keeps_the_figures_and_drops_the_prose():
    s = bench._side_summary(_line())
    assert s["value"] == 1.0e9 and s["ms_per_step"] == 12.5 and s["warmup"] == 3
    assert s["fallback_fraction"] == 0.03 and s["gpu_launches"] == 7
    assert s["layout"] == {"ants_per_warp": 2, "fused": 1, "cluster_log2": 1, "fallback_list": 32,
                           "warps_per_block": 0, "parts": 0}
    assert s["roofline"] == {"kernel": "k", "achieved": 10.0, "peak": 100.0, "unit": "GB/s", "frac": 0.1}
    assert s["e2e"] == {"value": 0.9e9, "unit": "ant-steps/s"}
    assert s["plain_gpu"] == {"value": 1.0e7, "unit": "ant-steps/s", "speedup_of_batched": 100.0}
    assert s["critical_share"] == 0.9
    assert s["clocks"] == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert "description" not in str(s) and "note" not in s


def test_side_summary_of_the_serving_line():
    serve = _line(latency_ms={"p50": 1.0, "p90": 2.0, "p99": 3.0, "mean": 1.5}, ant_steps_per_s=2.0e9,
                  config={"workload": "serve"}, latency_model=None, roofline=None)
    s = bench._side_summary(serve)
    assert s["latency_ms"] == {"p50": 1.0, "p90": 2.0, "p99": 3.0}
    assert s["ant_steps_per_s"] == 2.0e9 and "roofline" not in s and s["layout"] == {}


def test_extra_workloads_of_the_default_run():
    names = [n for n, _ in bench.SIDE_RUNS]
    assert names == ["tsp500", "atsp1000", "tsp10k_2opt", "serve", "paper_tsp500", "paper_tsp500_2opt",
                     "paper_tsp1k"]
    for name, extra in bench.SIDE_RUNS:
        assert name in bench.WORKLOAD_TEXT
        if name != "serve":
            assert "--no-cpu" in extra                                   # the oracle runs once, in the main line
            assert int(extra[extra.index("--warmup") + 1]) >= 3          # timing rule: at least 3 warm-up steps


def test_traffic_is_attached_only_to_the_captured_layout():
    assert ("batch128", 1, 0, 32, 0, 200) in bench.NCU_TRAFFIC
    assert bench.NCU_TRAFFIC.get(("batch128", 1, 2, 32, 1, 200)) is None
    t = bench.NCU_TRAFFIC[("batch128", 1, 0, 32, 0, 200)]
    assert 1e10 < t < 1.3e10     # DRAM bytes of one step's two fused launches, far below the algorithmic 342 GB
