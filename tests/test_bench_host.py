"""Host-side parts of bench.py (no GPU): the planning line and the oracle samples of the reference arm."""
import argparse

import pytest

import bench


def test_plan_search_line_small_grid():
    """The contraction-path search line on two Fig. 3.1 points: the JSON keys the contract asks for,
    no GPU launches, and both searches never worse than the greedy alone."""
    args = argparse.Namespace(workload="plan31")
    wl = dict(bench.WORKLOADS["plan31"], points=[(6, 4), (10, 6)])
    line = bench.plan_search_line(args, wl)
    for key in ("metric", "value", "unit", "higher_is_better", "gpu_launches", "config", "greedy", "search",
                "adaptive", "per_point"):
        assert key in line
    assert line["gpu_launches"] == 0 and line["higher_is_better"] is False
    for row in line["per_point"].values():
        assert row["search"]["cost_bytes"] <= row["greedy"]["cost_bytes"]
        assert row["adaptive"]["cost_bytes"] <= row["greedy"]["cost_bytes"]


@pytest.mark.parametrize("kind,n,depth,seed", [("q428", 16, 4, 1001), ("sweep_amps", 28, 14, 6000)])
def test_oracle_samples_of_new_workloads(kind, n, depth, seed):
    """The reference arm's oracle samples for the fixed-point and amplitude-sweep workloads run on
    the host and report a positive rate with its unit and what was sampled."""
    info, err = bench.run_oracle_sample(kind, n, depth, seed, 1.0)
    assert err is None, err
    assert info["value"] > 0 and info["unit"] == "amplitudes/s" and info["sample"]
