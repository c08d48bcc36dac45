"""The throughput metric of Eq. 13 against the paper's printed example."""
import json
import os

import pytest

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq13_throughput.json")


def test_eq13_matches_paper_example():
    g = json.load(open(GOLDEN))
    assert bench.mdes(g["width"], g["height"], g["d_max"], 1.0 / g["fps"]) == \
        pytest.approx(g["mdes"], abs=0.005)


def test_aggregation_flop_count():
    # one multiply and one add per tap of the (2 rho + 1)^2 window, per (u, v, d)
    assert bench.agg_flops_per_launch(1280, 720, 64, 5) == 242 * 1280 * 720 * 64
