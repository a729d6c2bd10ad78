"""Pins of the CPU oracle against facts that do not come from the oracle.

* closed forms: homomorphism counts of directed cycles, paths and out-stars
  are matrix products over the (label/attribute/timestamp-filtered)
  multiplicity matrix of the live edges (textbook walk counting), computed
  here with numpy integer matmuls;
* an inclusion-exclusion closed form for injective 2-paths, and iso = homo
  for a directed triangle on a self-loop-free graph;
* a sort-based count of time-respecting 2-paths (chain temporal order);
* brute force over all vertex maps versus the seed DFS;
* the incremental identities of Sec. II-B: dS = S(G + dG) minus S(G) as
  sets, |S(G2)| = |S(G)| + |dS+| - |dS-|, and batch-size invariance of the
  union of dS+ over an insert-only stream.
"""

import numpy as np
import pytest

from paper_2206_09983_b300 import gen

I32 = (gen.INT32_MIN, gen.INT32_MAX)
I64 = (gen.INT64_MIN, gen.INT64_MAX)


def tiny_stream(seed, n=7, m=30, vl=2, el=3, loops=True):
    return gen.uniform_stream(n, m, vl, el, seed=seed, attr_range=4, self_loops=loops)


def mult_matrix(s, label=-1, attr=I32, ts=I64, live=None):
    """A[v, w] = number of live edges v->w passing the edge filters."""
    n = s["num_vertices"]
    A = np.zeros((n, n), dtype=np.int64)
    ok = np.ones(len(s["src"]), dtype=bool)
    if live is not None:
        ok &= live
    if label >= 0:
        ok &= s["label"] == label
    ok &= (s["attr"] >= attr[0]) & (s["attr"] < attr[1])
    ok &= (s["ts"] >= ts[0]) & (s["ts"] < ts[1])
    np.add.at(A, (s["src"][ok].astype(np.int64), s["dst"][ok].astype(np.int64)), 1)
    return A


def diag(s, qmask):
    return np.diag(((s["vmask"] & np.uint32(qmask)) == np.uint32(qmask)).astype(np.int64))


def walk_count_cycle(s, q):
    k = q["nv"]
    M = np.eye(s["num_vertices"], dtype=np.int64)
    for i in range(k):
        _, _, lab, alo, ahi, tlo, thi = q["edges"][i]
        M = M @ diag(s, q["vmask"][i]) @ mult_matrix(s, lab, (alo, ahi), (tlo, thi))
    return int(np.trace(M))


def walk_count_path(s, q):
    k = len(q["edges"])
    M = np.eye(s["num_vertices"], dtype=np.int64)
    for i in range(k):
        _, _, lab, alo, ahi, tlo, thi = q["edges"][i]
        M = M @ diag(s, q["vmask"][i]) @ mult_matrix(s, lab, (alo, ahi), (tlo, thi))
    M = M @ diag(s, q["vmask"][k])
    return int(M.sum())


def star_count(s, q):
    """Out-star homomorphisms: sum_v [D0]_v prod_leaves (A_l D_leaf 1)_v."""
    n = s["num_vertices"]
    acc = np.diag(diag(s, q["vmask"][0])).copy()
    for i, (_, leaf, lab, alo, ahi, tlo, thi) in enumerate(q["edges"]):
        acc = acc * (mult_matrix(s, lab, (alo, ahi), (tlo, thi)) @ np.diag(diag(s, q["vmask"][leaf])))
    assert acc.shape == (n,)
    return int(acc.sum())


def all_count(oracle, s, q):
    n = len(s["src"])
    return oracle.count_static(s, 0, n, q)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [2, 3, 4])
def test_homo_cycle_closed_form(oracle_lib, seed, k):
    s = tiny_stream(100 + seed)
    rng = np.random.default_rng(seed)
    labels = [int(rng.integers(-1, 3)) for _ in range(k)]
    vm = [int(rng.integers(0, 4)) for _ in range(k)]
    q = gen.q_cycle(k, labels=labels, vmask=vm, iso=False)
    expect = walk_count_cycle(s, q)
    assert all_count(oracle_lib, s, q) == expect
    if k <= 3:
        assert len(oracle_lib.brute_force(s, 0, len(s["src"]), q)) == expect


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_homo_path_closed_form(oracle_lib, seed, k):
    s = tiny_stream(200 + seed)
    rng = np.random.default_rng(seed)
    labels = [int(rng.integers(-1, 3)) for _ in range(k)]
    vm = [int(rng.integers(0, 4)) for _ in range(k + 1)]
    q = gen.q_path(k, labels=labels, vmask=vm, iso=False)
    q["edges"][0] = q["edges"][0][:3] + (1, 3) + q["edges"][0][5:]   # attribute window on e0
    expect = walk_count_path(s, q)
    assert all_count(oracle_lib, s, q) == expect
    assert len(oracle_lib.brute_force(s, 0, len(s["src"]), q)) == expect


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("leaves", [2, 3])
def test_homo_out_star_closed_form(oracle_lib, seed, leaves):
    s = tiny_stream(300 + seed)
    rng = np.random.default_rng(seed)
    labels = [int(rng.integers(-1, 3)) for _ in range(leaves)]
    vm = [int(rng.integers(0, 4)) for _ in range(leaves + 1)]
    q = gen.q_out_star(leaves, labels=labels, vmask=vm, iso=False)
    ts_mid = int(s["ts"][len(s["ts"]) // 2])
    q["edges"][-1] = q["edges"][-1][:5] + (ts_mid, gen.INT64_MAX)   # timestamp window
    assert all_count(oracle_lib, s, q) == star_count(s, q)


@pytest.mark.parametrize("seed", range(8))
def test_iso_two_path_inclusion_exclusion(oracle_lib, seed):
    """Injective 2-paths = walks minus the three coincidence sets (+2 T)."""
    s = tiny_stream(400 + seed, n=6, m=40)
    A = mult_matrix(s)
    out_d, in_d, loops = A.sum(1), A.sum(0), np.diag(A)
    H = int((A @ A).sum())
    S01 = int((loops * out_d).sum())          # v0 = v1
    S12 = int((in_d * loops).sum())           # v1 = v2
    S02 = int(np.trace(A @ A))                # v0 = v2
    T = int((loops * loops).sum())            # all three equal
    expect = H - (S01 + S12 + S02 - 2 * T)
    q = gen.q_path(2, iso=True)
    assert all_count(oracle_lib, s, q) == expect
    assert len(oracle_lib.brute_force(s, 0, len(s["src"]), q)) == expect


@pytest.mark.parametrize("seed", range(6))
def test_iso_triangle_equals_homo_without_loops(oracle_lib, seed):
    s = tiny_stream(500 + seed, n=8, m=60, loops=False)
    qi = gen.q_cycle(3, iso=True)
    qh = gen.q_cycle(3, iso=False)
    assert all_count(oracle_lib, s, qi) == all_count(oracle_lib, s, qh) == walk_count_cycle(s, qh)


@pytest.mark.parametrize("seed", range(6))
def test_temporal_chain_two_path_sort_count(oracle_lib, seed):
    """Homomorphic 2-paths e0 = (a->b), e1 = (b->c) with ts(e0) < ts(e1):
    for each e1, the number of edges into src(e1) with a smaller timestamp."""
    s = tiny_stream(600 + seed, n=6, m=50)
    n = s["num_vertices"]
    expect = 0
    for v in range(n):
        into = np.sort(s["ts"][s["dst"] == v])
        outs = s["ts"][s["src"] == v]
        expect += int(np.searchsorted(into, outs, side="left").sum())
    q = gen.q_path(2, iso=False, temporal="chain")
    assert all_count(oracle_lib, s, q) == expect
    # reversed order (pairs): ts(e1) < ts(e0)
    qr = gen.q_path(2, iso=False, temporal="pairs", prec=[(1, 0)])
    expect_r = 0
    for v in range(n):
        outs = np.sort(s["ts"][s["src"] == v])
        into = s["ts"][s["dst"] == v]
        expect_r += int(np.searchsorted(outs, into, side="left").sum())
    assert all_count(oracle_lib, s, qr) == expect_r


# ---------------------------------------------------------------- brute force vs seed DFS

def random_tiny_query(rng, nv_max=4):
    nv = int(rng.integers(2, nv_max + 1))
    kind = "tree" if rng.random() < 0.5 else "cycle"
    chords = int(rng.integers(0, 2)) if kind == "cycle" and nv >= 4 else 0
    if kind == "cycle" and nv == 2:
        kind = "tree"
    q = gen.random_query(rng, nv, kind, 3, 2, chords=chords)
    q["vmask"] = [m if rng.random() < 0.5 else 0 for m in q["vmask"]]
    q["edges"] = [e if rng.random() < 0.6 else e[:2] + (-1,) + e[3:] for e in q["edges"]]
    q["iso"] = bool(rng.random() < 0.5)
    t = rng.random()
    q["temporal"] = "chain" if t < 0.3 else ("pairs" if t < 0.5 else "none")
    k = len(q["edges"])
    if k < 2:
        q["temporal"] = "none"
    if q["temporal"] == "pairs":
        q["prec"] = [tuple(map(int, rng.choice(k, 2, replace=False)))]
    if rng.random() < 0.3:
        e = q["edges"][0]
        q["edges"][0] = e[:3] + (1, 3) + e[5:]
    return q


@pytest.mark.parametrize("seed", range(30))
def test_brute_force_equals_seed_oracle(oracle_lib, seed):
    rng = np.random.default_rng(1000 + seed)
    s = tiny_stream(700 + seed, n=int(rng.integers(4, 7)), m=int(rng.integers(10, 26)))
    q = random_tiny_query(rng)
    n = len(s["src"])
    bf = oracle_lib.brute_force(s, 0, n, q)
    st = oracle_lib.list_static(s, 0, n, q)
    assert bf.shape == st.shape and (bf == st).all()
    assert oracle_lib.count_static(s, 0, n, q) == len(bf)
    # iso embeddings are a subset of the homomorphisms
    qh = dict(q, iso=False)
    homo = {tuple(r) for r in oracle_lib.brute_force(s, 0, n, qh)}
    assert {tuple(r) for r in bf} <= homo


def as_set(rows):
    return {tuple(r) for r in rows}


@pytest.mark.parametrize("seed", range(20))
def test_delta_is_set_difference(oracle_lib, seed):
    """dS+ = S(G + ins) \\ S(G) and dS- = S(G1) \\ S(G1 - del), by brute force."""
    rng = np.random.default_rng(2000 + seed)
    s = tiny_stream(800 + seed, n=5, m=24)
    q = random_tiny_query(rng)
    lo, hi, hi_new = 3, 12, 19
    pos = oracle_lib.delta(s, lo, hi_new, hi, hi_new, q)
    before = as_set(oracle_lib.brute_force(s, lo, hi, q))
    after = as_set(oracle_lib.brute_force(s, lo, hi_new, q))
    assert as_set(pos) == after - before and len(pos) == len(after - before)
    assert oracle_lib.delta_count_first_edge(s, lo, hi_new, hi, hi_new, q) == len(pos)
    # expiry of [lo, lo + 4) on G1
    neg = oracle_lib.delta(s, lo, hi_new, lo, lo + 4, q)
    after_del = as_set(oracle_lib.brute_force(s, lo + 4, hi_new, q))
    assert as_set(neg) == after - after_del
    # the counting identity |S(G2)| = |S(G)| + |dS+| - |dS-|
    assert len(after_del) == len(after) - len(neg)
    assert len(after) == len(before) + len(pos)


@pytest.mark.parametrize("seed", range(4))
def test_window_stream_count_invariant(oracle_lib, seed):
    s = gen.uniform_stream(40, 600, 2, 3, seed=900 + seed, attr_range=3)
    q = gen.q_cycle(3, labels=[-1, 0, -1], iso=bool(seed % 2), temporal="none")
    W, B = 250, 37
    prev = 0
    for lo, hi, hi_new, x in oracle_lib.window_batches(len(s["src"]), B, W):
        pos = oracle_lib.delta(s, lo, hi_new, hi, hi_new, q)
        neg = oracle_lib.delta(s, lo, hi_new, lo, lo + x, q)
        now = oracle_lib.count_static(s, lo + x, hi_new, q)
        assert now == prev + len(pos) - len(neg)
        prev = now


@pytest.mark.parametrize("seed", range(3))
def test_batch_partition_invariance(oracle_lib, seed):
    s = gen.uniform_stream(30, 300, 2, 2, seed=950 + seed)
    q = gen.q_path(2, labels=[0, -1], iso=True, temporal="chain" if seed == 1 else "none")
    n = len(s["src"])
    full = oracle_lib.list_static(s, 0, n, q)
    for B in (1, 7, 64, n):
        rows = []
        for lo, hi, hi_new, x in oracle_lib.window_batches(n, B, 0):
            rows.append(oracle_lib.delta(s, lo, hi_new, hi, hi_new, q))
        allr = np.concatenate(rows)
        assert len(allr) == len(full)
        assert as_set(allr) == as_set(full)


@pytest.mark.parametrize("seed", range(4))
def test_debi_word_is_single_edge_embedding(oracle_lib, seed):
    """Bit e of an edge's DEBI word is set iff that edge embeds the one-edge
    query made of e and its endpoint labels."""
    rng = np.random.default_rng(3000 + seed)
    s = tiny_stream(1100 + seed, n=6, m=30)
    q = random_tiny_query(rng)
    n = len(s["src"])
    words = oracle_lib.debi_words(s, 0, n, q)
    for e, (a, b, *rest) in enumerate(q["edges"]):
        one = gen.make_query(2, [(0, 1) + tuple(rest[0:1]) + (tuple(rest[1:3]), tuple(rest[3:5]))],
                             vmask=[q["vmask"][a], q["vmask"][b]], iso=False)
        hits = set(int(r[2]) for r in oracle_lib.brute_force(s, 0, n, one))
        for i in range(n):
            assert bool(words[i] >> e & 1) == (i in hits)


def test_parallel_edges_multiply(oracle_lib):
    """Parallel edges are distinct edge instances: a 2-cycle over k parallel
    a->b and l parallel b->a edges has k*l embeddings per rotation."""
    s = {
        "src": np.array([0, 0, 0, 1, 1], dtype=np.uint32),
        "dst": np.array([1, 1, 1, 0, 0], dtype=np.uint32),
        "label": np.zeros(5, dtype=np.uint8),
        "attr": np.zeros(5, dtype=np.int32),
        "ts": np.arange(1, 6, dtype=np.int64),
        "vmask": np.array([1, 1], dtype=np.uint32),
        "num_vertices": 2, "num_edge_labels": 1,
    }
    q = gen.q_cycle(2, iso=True)
    assert oracle_lib.count_static(s, 0, 5, q) == 2 * 3 * 2
    qt = gen.q_cycle(2, iso=True, temporal="chain")
    # ts(e0) < ts(e1): u0->u1 at t in {1,2,3} then u1->u0 at t in {4,5}: 3*2;
    # u0 = 1: edge 1->0 (t 4,5) then 0->1 (t 1..3) later: none
    assert oracle_lib.count_static(s, 0, 5, qt) == 6


# ---------------------------------------------------------------- multi-label vertices

def multi_stream(seed, n=7, m=36, vl=3, el=2):
    return gen.uniform_stream(n, m, vl, el, seed=seed, attr_range=2, multi_label_p=0.45)


def test_multi_label_generator_gives_proper_supersets():
    s = multi_stream(1)
    pop = np.array([bin(int(x)).count("1") for x in s["vmask"]])
    assert (pop >= 1).all() and (pop >= 2).any()


def test_subset_test_hand_fixture(oracle_lib):
    """L_Q(u) subset-of L(f(u)) with several labels per data vertex (Sec. II-B):
    vertex masks 0b011, 0b001, 0b110, 0b111; a one-edge query whose source
    mask is 0b011 only starts at vertices 0 and 3 (both hold labels 0 and 1),
    and a destination mask 0b100 only ends at vertices 2 and 3."""
    s = {
        "src": np.array([0, 0, 1, 2, 3, 3, 1, 0], dtype=np.uint32),
        "dst": np.array([1, 2, 2, 3, 0, 2, 3, 3], dtype=np.uint32),
        "label": np.zeros(8, dtype=np.uint8),
        "attr": np.zeros(8, dtype=np.int32),
        "ts": np.arange(1, 9, dtype=np.int64),
        "vmask": np.array([0b011, 0b001, 0b110, 0b111], dtype=np.uint32),
        "num_vertices": 4, "num_edge_labels": 1,
    }
    # sources with both labels 0 and 1: vertices 0 (edges 0, 1, 7) and 3 (edges 4, 5)
    q = gen.make_query(2, [(0, 1)], vmask=[0b011, 0], iso=True)
    rows = oracle_lib.list_static(s, 0, 8, q)
    assert sorted(int(r[2]) for r in rows) == [0, 1, 4, 5, 7]
    # and destinations holding label 2: vertices 2, 3 -> edges 1 (0->2), 5 (3->2), 7 (0->3)
    q2 = gen.make_query(2, [(0, 1)], vmask=[0b011, 0b100], iso=True)
    assert sorted(int(r[2]) for r in oracle_lib.list_static(s, 0, 8, q2)) == [1, 5, 7]
    # a mask no vertex holds completely matches nothing
    q3 = gen.make_query(2, [(0, 1)], vmask=[0b1000, 0], iso=True)
    assert oracle_lib.count_static(s, 0, 8, q3) == 0


@pytest.mark.parametrize("seed", range(6))
def test_multi_label_closed_forms(oracle_lib, seed):
    """Homomorphism walk counts with multi-bit data and query masks: the
    diagonal D_u = [qmask(u) subset-of vmask(v)] carries the subset test."""
    s = multi_stream(1200 + seed)
    rng = np.random.default_rng(seed)
    masks = [0, 1, 2, 3, 4, 5, 6]
    vm = [int(rng.choice(masks)) for _ in range(4)]
    qc = gen.q_cycle(3, vmask=vm[:3], iso=False)
    assert all_count(oracle_lib, s, qc) == walk_count_cycle(s, qc)
    qp = gen.q_path(3, vmask=vm, iso=False)
    assert all_count(oracle_lib, s, qp) == walk_count_path(s, qp)
    assert len(oracle_lib.brute_force(s, 0, len(s["src"]), qc)) == walk_count_cycle(s, qc)
    qs = gen.q_out_star(3, vmask=vm, iso=False)
    assert all_count(oracle_lib, s, qs) == star_count(s, qs)


@pytest.mark.parametrize("seed", range(10))
def test_multi_label_brute_force_equals_seed_oracle(oracle_lib, seed):
    rng = np.random.default_rng(4000 + seed)
    s = multi_stream(1300 + seed, n=int(rng.integers(4, 7)), m=int(rng.integers(12, 26)))
    q = random_tiny_query(rng)
    q["vmask"] = [int(rng.integers(0, 8)) for _ in range(q["nv"])]
    n = len(s["src"])
    bf = oracle_lib.brute_force(s, 0, n, q)
    st = oracle_lib.list_static(s, 0, n, q)
    assert bf.shape == st.shape and (bf == st).all()


# ---------------------------------------------------------------- budgeted delta count

@pytest.mark.parametrize("seed", range(10))
def test_delta_count_budget_unlimited_is_exact(oracle_lib, seed):
    """With no node budget (0) the count is |S(G + ins) \\ S(G)| by brute
    force, reported complete."""
    rng = np.random.default_rng(5000 + seed)
    s = tiny_stream(1400 + seed, n=5, m=24)
    q = random_tiny_query(rng)
    lo, hi, hi_new = 2, 13, 20
    before = as_set(oracle_lib.brute_force(s, lo, hi, q))
    after = as_set(oracle_lib.brute_force(s, lo, hi_new, q))
    mask = np.zeros(hi_new - lo, dtype=np.uint8)
    mask[hi - lo:] = 1
    cnt, complete = oracle_lib.delta_count_budget(s, lo, hi_new, q, mask, 0)
    assert complete and cnt == len(after - before)
    big, complete = oracle_lib.delta_count_budget(s, lo, hi_new, q, mask, 10**9)
    assert complete and big == cnt


def test_delta_count_budget_partial_is_flagged_and_bounded(oracle_lib):
    """A budget that runs out is reported incomplete, and the partial count
    never exceeds the exact one and grows with the budget."""
    s = gen.uniform_stream(12, 200, 1, 1, seed=77)
    q = gen.q_path(3, iso=False)
    lo, hi, hi_new = 0, 150, 200
    exact = len(as_set(oracle_lib.brute_force(s, lo, hi_new, q)) -
                as_set(oracle_lib.brute_force(s, lo, hi, q)))
    assert exact > 100
    mask = np.zeros(hi_new - lo, dtype=np.uint8)
    mask[hi - lo:] = 1
    prev = -1
    saw_partial = False
    for budget in (1, 10, 100, 1000, 10**4, 10**5, 10**7):
        cnt, complete = oracle_lib.delta_count_budget(s, lo, hi_new, q, mask, budget)
        assert cnt <= exact and cnt >= prev
        if not complete:
            saw_partial = True
        else:
            assert cnt == exact
        prev = cnt
    assert saw_partial and prev == exact
    cnt, complete = oracle_lib.delta_count_budget(s, lo, hi_new, q, mask, 1)
    assert not complete


# ---------------------------------------------------------------- parallel (timing) oracle

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_parallel_delta_count_is_the_set_difference(oracle_lib, seed, threads):
    """The OpenMP count over seeds (the CPU baseline's timing oracle) gives
    |S(G + ins) minus S(G)| by brute force, for any thread count."""
    rng = np.random.default_rng(6000 + seed)
    s = tiny_stream(1500 + seed, n=5, m=26)
    q = random_tiny_query(rng)
    lo, hi, hi_new = 1, 12, 22
    before = as_set(oracle_lib.brute_force(s, lo, hi, q))
    after = as_set(oracle_lib.brute_force(s, lo, hi_new, q))
    mask = np.zeros(hi_new - lo, dtype=np.uint8)
    mask[hi - lo:] = 1
    assert oracle_lib.delta_count_parallel(s, lo, hi_new, q, mask, threads) == len(after - before)


def test_parallel_delta_count_on_a_larger_stream(oracle_lib):
    s = gen.rmat_stream(9, 6000, 0.57, 0.19, 0.19, 2, 1.2, 2, 10, seed=3)
    q = gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain")
    mask = np.zeros(6000, dtype=np.uint8)
    mask[4000:] = 1
    want = len(oracle_lib.delta(s, 0, 6000, 4000, 6000, q))
    assert want > 100
    for t in (1, 2, 0):
        assert oracle_lib.delta_count_parallel(s, 0, 6000, q, mask, t) == want
