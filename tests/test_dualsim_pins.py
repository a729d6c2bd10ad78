"""Pins of the dual-simulation oracle (oracle/dualsim.py) against the
definition, not against itself:
  * brute force: on tiny graphs, the union of every relation that satisfies
    the definition (checked pair by pair) is the largest one, and the oracle
    returns exactly it (or nothing when a query vertex is left unmatched);
  * every homomorphic embedding's vertex pairs lie in the relation (each
    embedding is a dual simulation);
  * a one-edge query relates exactly the endpoints of its matching edges."""
import itertools

import numpy as np
import pytest

from oracle import dualsim, oracle
from paper_2206_09983_b300 import gen


def _rel(sim, nv):
    return {(u, v) for v in range(len(sim)) for u in range(nv) if (int(sim[v]) >> u) & 1}


def _tiny_queries():
    return [gen.q_path(1, labels=[0], iso=False),
            gen.q_path(2, labels=[0, -1], iso=False),
            gen.q_cycle(2, labels=[-1, 1], iso=False),
            gen.q_cycle(3, labels=[-1, -1, -1], vmask=[1, 0, 0], iso=False)]


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_largest_relation(seed):
    s = gen.uniform_stream(4, 9, 2, 2, seed=100 + seed)
    n = len(s["src"])
    for q in _tiny_queries():
        nv = q["nv"]
        cand = [(u, v) for u in range(nv) for v in range(s["num_vertices"])
                if (int(s["vmask"][v]) & q["vmask"][u]) == q["vmask"][u]]
        assert len(cand) <= 12
        best = set()
        for k in range(len(cand) + 1):
            for sub in itertools.combinations(cand, k):
                rel = set(sub)
                if rel <= best:
                    continue
                if dualsim.is_dual_simulation(s, 0, n, q, rel):
                    best |= rel
        assert dualsim.is_dual_simulation(s, 0, n, q, best)
        if {u for u, _ in best} != set(range(nv)):
            best = set()
        got = _rel(dualsim.dual_simulation(s, 0, n, q), nv)
        assert got == best, (seed, q["edges"])


@pytest.mark.parametrize("seed", range(4))
def test_homomorphic_embeddings_lie_in_the_relation(seed):
    s = gen.uniform_stream(30, 400, 2, 3, seed=200 + seed)
    n = len(s["src"])
    qs = [gen.q_path(2, labels=[0, 1], iso=False), gen.q_cycle(3, iso=False),
          gen.q_out_star(2, labels=[2, -1], vmask=[1, 0, 2], iso=False)]
    for q in qs:
        sim = dualsim.dual_simulation(s, 0, n, q)
        rows = oracle.list_static(s, 0, n, q)
        for r in rows:
            for u in range(q["nv"]):
                assert (int(sim[int(r[u])]) >> u) & 1
        if len(rows):
            assert sim.any()


def test_one_edge_query_closed_form():
    s = gen.uniform_stream(50, 300, 3, 3, seed=7)
    n = len(s["src"])
    q = gen.q_path(1, labels=[1], vmask=[1, 2], iso=False)
    words = oracle.debi_words(s, 0, n, q)
    exp = np.zeros(s["num_vertices"], dtype=np.uint32)
    for i in np.nonzero(words)[0]:
        exp[s["src"][i]] |= 1
        exp[s["dst"][i]] |= 2
    if not ((exp & 1).any() and (exp & 2).any()):
        exp[:] = 0
    assert np.array_equal(dualsim.dual_simulation(s, 0, n, q), exp)
    assert exp.any()


def test_deleted_edges_do_not_count():
    s = gen.uniform_stream(20, 200, 1, 2, seed=9)
    n = len(s["src"])
    q = gen.q_cycle(2, iso=False)
    alive = np.ones(n, dtype=np.uint8)
    alive[::2] = 0
    keep = np.nonzero(alive)[0]
    s2 = dict(s, src=s["src"][keep], dst=s["dst"][keep], label=s["label"][keep],
              attr=s["attr"][keep], ts=s["ts"][keep])
    assert np.array_equal(dualsim.dual_simulation(s, 0, n, q, alive=alive),
                          dualsim.dual_simulation(s2, 0, len(keep), q))
