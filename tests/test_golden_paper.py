"""The only derived numbers the paper prints: Table 3's gaps follow from
Tables 1 and 2 with the definition of Sec. IV-E, (upper - lower)/upper."""
import json
import os

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def test_table3_gaps_follow_from_tables_1_and_2():
    d = json.load(open(GOLD))["cases"]
    for name, c in d.items():
        gap_admm = 100 * (c["admm_obj"] - c["juniper_lb"]) / c["admm_obj"]
        assert abs(gap_admm - c["gap_admm"]) < 0.011, name
        if c["juniper_ub"] is not None:
            gap_j = 100 * (c["juniper_ub"] - c["juniper_lb"]) / c["juniper_ub"]
            assert abs(gap_j - c["gap_juniper"]) < 0.011, name
