"""Host spill of expired edges (mn_set_spill / mn_read_spill): every edge
that leaves the window is kept in a pinned host FIFO with its DEBI words as
they were at expiry; the records read back equal the stream's edges and the
words equal the oracle's edgeMatcher words, for a count window (with the
FIFO wrapping around) and a time window."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import make_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def check_spill(g, s, qs, lo, hi):
    e, w, held = g.read_spill(lo, hi, len(qs))
    for k in ("src", "dst", "label", "attr", "ts"):
        assert (e[k] == s[k][lo:hi]).all(), k
    for qi, q in enumerate(qs):
        assert (w[qi] == oracle.debi_words(s, lo, hi, q)).all(), f"query {qi} words"


def test_count_window_spill_wraps_around():
    s = gen.uniform_stream(200, 12000, 2, 3, seed=0x4D4E00C0, attr_range=50)
    qs = [gen.q_cycle(3, labels=[0, -1, 1], iso=True),
          gen.make_query(2, [(0, 1, 2, (5, 30))], vmask=[1, 0], iso=True)]
    with make_graph(s, window=3000, max_batch=1000) as g:
        for q in qs:
            g.register_query(q)
        g.set_spill(2500)
        for lo_b in range(0, 12000, 1000):
            g.insert(M.edges_from_stream(s, lo_b, lo_b + 1000))
            wlo, whi, _ = g.info()
            _, _, held = g.read_spill(0, 0, len(qs))
            assert held[1] == wlo                           # everything expired so far
            assert held[1] - held[0] == min(wlo, 2500)      # the FIFO keeps the most recent
            if held[1] > held[0]:
                check_spill(g, s, qs, held[0], held[1])
        with pytest.raises(M.MnError):
            g.read_spill(0, 10, len(qs))                     # overwritten long ago
        assert g.stats()["spill_bytes"] > 0


def test_time_window_spill():
    s = gen.uniform_stream(150, 8000, 2, 2, seed=0x4D4E00C1, attr_range=5)
    qs = [gen.q_path(2, labels=[0, 1], iso=True, temporal="chain")]
    span = int(s["ts"][2000] - s["ts"][0])
    with make_graph(s, max_batch=1000, capacity=8000) as g:
        g.register_query(qs[0])
        g.set_time_window(span)
        g.set_spill(10000)
        for lo_b in range(0, 8000, 1000):
            g.insert(M.edges_from_stream(s, lo_b, lo_b + 1000))
        wlo, whi, _ = g.info()
        assert wlo > 0
        check_spill(g, s, qs, 0, wlo)
