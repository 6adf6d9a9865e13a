"""The workload table's m0 values are the ones the oracle tuning script
recorded (tests/golden/workloads.json, written by tests/golden/tune_m0.py)."""
import json
import os

from paper_2004_08146_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workloads.json")


def test_m0_matches_oracle_tuning():
    data = json.load(open(GOLDEN))
    for name, rec in data.items():
        w = workloads.WORKLOADS[name]
        assert tuple(rec["dims"]) == tuple(w["dims"])
        assert rec["eps"] == w["eps"] and rec["csw"] == w["csw"] and rec["seed"] == w["seed"]
        assert rec["m0"] == w["m0"]
