"""The workload table: its m0 values are the ones the oracle tuning script
recorded (tests/golden/workloads.json, written by tests/golden/tune_m0.py and
tune_m0_dense.py), and bench.py passes each workload's solver shape on."""
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


def test_bench_parameters_follow_the_workload_table():
    """bench.py hands each workload's solver shape to the library unchanged
    (host logic only: the parameter block is filled, no GPU work)."""
    import bench
    from paper_2004_08146_gb300 import qcd
    w = workloads.get("c4_64x32c3")
    p = bench.workload_params(qcd, w)
    assert (p.levels, p.nv2, tuple(p.agg2)) == (3, 24, (2, 2, 2, 2))
    assert (p.block, p.m_min, p.m_max, p.update_every, p.sap_half) == (16, 30, 50, 20, 1)
    assert tuple(p.sap_block) == (2, 2, 2, 2) and p.use_mg == 1
    w3 = workloads.get("c3_32x16c3")
    p3 = bench.workload_params(qcd, w3)
    assert (p3.levels, p3.block, p3.m_min, p3.m_max, p3.sap_half) == (2, 16, 30, 50, 1)
    p2 = bench.workload_params(qcd, workloads.get("c2_16x8c3"))
    assert (p2.block, p2.levels, p2.guard, p2.coarse_maxiter) == (4, 2, 0, 12)
    # Table 2 defaults stay in place
    assert (p2.nu, p2.inner_maxiter, p2.inner_tol, p2.coarse_tol, p2.setup_iters) == (4, 5, 0.1, 0.5, 6)
