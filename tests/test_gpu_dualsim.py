"""Dual simulation through the C ABI (mn_dual_simulation) against the CPU
oracle (oracle/dualsim.py), word by word, over a sliding window with expiries
and explicit deletes, for paths, cycles (with a chord), stars, trees and a
query that cannot match."""
import numpy as np
import pytest

from oracle import dualsim, oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import vm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def _queries():
    cyc = gen.q_cycle(4, labels=[0, -1, 1, -1], vmask=vm(None, 0, None, None), iso=False)
    cyc["edges"].append((0, 2, 2, cyc["edges"][0][3], cyc["edges"][0][4], cyc["edges"][0][5],
                         cyc["edges"][0][6]))                      # a chord u0 -> u2
    return [gen.q_path(3, labels=[0, 1, 2], vmask=vm(1, None, None, 0), iso=True, temporal="chain"),
            cyc,
            gen.q_out_star(3, labels=[1, 1, -1], vmask=vm(None, 2, None, None), iso=False),
            gen.q_tree6(labels=[0, 1, 2, 3, 0], vmask=vm(None, None, 1, None, None, None), iso=False),
            gen.q_cycle(3, labels=[3, 3, 3], vmask=vm(5, 5, 5), iso=False)]   # labels absent


def test_dual_simulation_matches_oracle():
    s = gen.rmat_stream(10, 20000, 0.57, 0.19, 0.19, 4, 1.2, 3, 1000, seed=0xD5)
    n, W, B = len(s["src"]), 8000, 3000
    qs = _queries()
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=W, max_batch=W,
                max_queries=len(qs))
    try:
        g.insert(M.edges_from_stream(s, 0, W), count_only=True)
        for q in qs:
            g.register_query(q)
        checked = nonempty = 0
        for k, (lo, hi, hi_new, x) in enumerate(oracle.window_batches(n, B, W, W)):
            g.insert(M.edges_from_stream(s, hi, hi_new), count_only=True)
            if k not in (0, 2):
                continue
            lo_l, hi_l, _ = g.info()
            dead = np.arange(lo_l + 5, lo_l + 2000, 11, dtype=np.uint64) if k == 2 else None
            if dead is not None:
                g.delete(dead, count_only=True)
            alive = np.ones(hi_l - lo_l, dtype=np.uint8)
            if dead is not None:
                alive[(dead - lo_l).astype(np.int64)] = 0
            for qi, q in enumerate(qs):
                got = g.dual_simulation(qi)
                exp = dualsim.dual_simulation(s, lo_l, hi_l, q, alive=alive)
                bad = np.nonzero(got != exp)[0]
                assert len(bad) == 0, f"batch {k} query {qi}: vertex {bad[0]} gpu {got[bad[0]]:#x} oracle {exp[bad[0]]:#x}"
                checked += 1
                nonempty += int(exp.any())
        assert checked == 10 and nonempty >= 6
        assert not g.dual_simulation(len(qs) - 1).any()       # the query whose labels are absent
    finally:
        g.close()
