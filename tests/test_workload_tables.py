"""The query tables the benchmarks run are exactly the ones the committed
calibration scripts under tests/golden/ wrote (each search calls only the
oracle), so every bench query can be traced to a seeded oracle run."""
import json
import os

from paper_2206_09983_b300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)["queries"]


def test_rmat20_c3_table_is_the_calibration_output():
    cal = load("rmat20_c3_calibration.json")
    assert len(cal) == len(workloads.RMAT20_C3_QUERIES) == 32
    for row, c in zip(workloads.RMAT20_C3_QUERIES, cal):
        i, nv, edges, el, vl = row
        assert (i, nv, [list(e) for e in edges], el, vl) == \
            (c["index"], c["nv"], c["edges"], c["elabels"], c["vlabels"]), i


def test_flow_table_is_the_calibration_output():
    cal = load("flow_queries_calibration.json")
    assert len(cal) == len(workloads.FLOW_QUERIES) == 8
    for row, c in zip(workloads.FLOW_QUERIES, cal):
        i, nv, edges, el = row
        assert (i, nv, [list(e) for e in edges], el) == (c["index"], c["nv"], c["edges"], c["elabels"]), i
        assert 2**8 <= c["first_batch_new"] <= 2**16
