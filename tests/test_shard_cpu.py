"""Host side of seed sharding, on CPU: two gloo ranks each hold a disjoint
part of a batch's result (the oracle's dS+ of a small stream, split by row);
the gather on rank 0 gives back the whole result, counts and sorted rows."""
import os
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _full_result():
    sys.path.insert(0, ROOT)
    from oracle import oracle
    from paper_2206_09983_b300 import gen

    s = gen.uniform_stream(40, 600, 2, 2, seed=3)
    qs = [gen.q_path(2, labels=[0, 1], iso=True), gen.q_cycle(3, iso=False)]
    return [oracle.delta(s, 0, 600, 500, 600, q) for q in qs]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2206_09983_b300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = _full_result()
        # this rank's part: a disjoint split of every list (rows i % world == rank)
        rows = {(q, +1): full[q][rank::world] for q in range(len(full))}
        cpos = [len(rows[(q, +1)]) for q in range(len(full))]
        res = shard.gather_batch(cpos, [0] * len(full), rows)
        if rank == 0:
            mpos, mneg, mrows = res
            ok = mpos == [len(r) for r in full] and mneg == [0] * len(full)
            for q in range(len(full)):
                ok = ok and np.array_equal(mrows[(q, +1)], full[q])
            out.put(bool(ok))
        else:
            out.put(res is None)
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_rebuilds_the_whole_result():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, 29571, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs)
    assert [out.get(timeout=5), out.get(timeout=5)] == [True, True]


def test_merge_helpers():
    from paper_2206_09983_b300 import shard

    a = np.array([[3, 1], [1, 2]], dtype=np.uint64)
    b = np.array([[2, 9]], dtype=np.uint64)
    m = shard.merge_rows([a, b, np.empty((0, 2), dtype=np.uint64)])
    assert m.tolist() == [[1, 2], [2, 9], [3, 1]]
    assert shard.merge_counts([[1, 2], [3, 4], [0, 5]]) == [4, 11]
