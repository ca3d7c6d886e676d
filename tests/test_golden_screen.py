"""The feasibility screen of the 2000-bus workload (tests/golden/
screen_loading.py, run on the oracle): the configured loading and every
heavier rung fail on four network draws, and the benchmark's network
loading (0.4 (300/2000)^(1/4) = 0.249) lies between the largest rung that
passes and the next one, which fails."""
import json
import os

from paper_2310_13145_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bench_loading_is_the_largest_screened_feasible_one():
    d = json.load(open(os.path.join(HERE, "golden", "screen_c5_2000bus.json")))
    assert d["criterion"].startswith("Algorithm 1 stop")
    rungs = {e["loading"]: e for e in d["ladder"]}
    assert not rungs[1.0]["passed"] and len(rungs[1.0]["tries"]) >= 4
    for e in d["ladder"]:
        if e["passed"]:
            t = e["tries"][-1]
            assert t["passed"] and max(t["r_p"], t["r_d"], t["z_rms"]) <= 1e-4
        else:
            assert all(not t["passed"] for t in e["tries"])
    best = d["largest_passing_loading"]
    heavier = min(x for x in rungs if x > best)
    assert not rungs[heavier]["passed"]
    assert synth.network_loading(2000) <= best < heavier
