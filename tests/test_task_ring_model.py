"""Model check of the enumerator's lapped task ring (the protocol of
k_enumerate's task hand-off, re-stated step by step in Python, not the CUDA
code itself): warps as coroutines that yield at every atomic step, run under
many random interleavings with a tiny ring so that laps wrap, tickets get
skipped and slots get abandoned.  Every task must be run exactly once -- by
the warp that took it from the ring, or by its donor when the hand-off
failed -- and every taken task must carry the data its publisher wrote.

Slot state (64 bits, only grows): key(lap) + phase, key(lap) = lap * 4 (the
launch's epoch is constant here), phases RESERVED 0, PUBLISHED 1, ABANDONED 2,
CONSUMED 3; a slot is free when it holds no live task (abandoned, consumed,
or never used in this launch)."""
import random

import pytest

RES, PUB, ABD, CON = 0, 1, 2, 3


class Ring:
    def __init__(self, cap):
        self.cap = cap
        self.state = [-4] * cap          # "earlier launch": below every key, free
        self.data = [None] * cap
        self.head = 0                    # tickets drawn
        self.tail = 0                    # slots handed to publishers
        self.busy = 0
        self.idle = 0

    def key(self, t):
        return (t // self.cap) * 4

    @staticmethod
    def free(v):
        return v < 0 or v % 4 >= ABD


def publisher(ring, task, log):
    """Hand `task` to the ring; returns via log whether it was handed off."""
    yield
    if ring.tail - ring.head >= ring.cap // 2:
        log.append(("kept", task))
        return
    slot = ring.tail
    ring.tail += 1
    yield
    s, key = slot % ring.cap, ring.key(slot)
    v = ring.state[s]
    reserved = False
    for _ in range(8):
        if not (v < key and ring.free(v)):
            break
        yield                                            # the CAS
        if ring.state[s] == v:
            ring.state[s] = key + RES
            reserved = True
            break
        v = ring.state[s]
    if not reserved:
        log.append(("kept", task))
        return
    yield
    ring.data[s] = task                                  # write the task
    yield
    ring.state[s] = key + PUB                            # publish
    log.append(("handed", task))


def waiter(ring, spins, out):
    """Draw tickets until a task is taken (out = [task]) or the warp leaves."""
    ring.idle += 1
    for _ in range(64):
        yield
        t = ring.head
        ring.head += 1
        s, key = t % ring.cap, ring.key(t)
        quiet = 0
        for it in range(10 ** 6):
            yield
            v = ring.state[s]
            if v == key + PUB:
                yield
                task = ring.data[s]                      # read the task
                yield
                assert ring.state[s] == key + PUB, "published slot changed before it was consumed"
                ring.state[s] = key + CON
                ring.idle -= 1
                out.append(task)
                return
            if v >= key + 4:
                break                                    # skipped by a later lap: draw again
            if v != key + RES and ring.free(v) and (quiet >= 4 or it >= spins):
                yield                                    # the CAS
                if ring.state[s] == v:
                    ring.state[s] = key + ABD
                    ring.idle -= 1
                    return
                continue
            quiet = quiet + 1 if ring.busy == 0 else 0
        else:
            raise AssertionError("waiter spun without end")
    ring.idle -= 1


def worker(ring, rng, first_task, spawn, done, spins):
    """A warp: run a task (possibly donating sub-tasks), then wait for more."""
    task = first_task
    while task is not None:
        done.append(task)
        kids = spawn(task)
        for kid in kids:                                 # donate while others idle (or not)
            log = []
            yield from publisher(ring, kid, log)
            if log[-1][0] == "kept":                     # run it here
                done.append(kid)
                for g in spawn(kid):                     # its own sub-tasks run here too
                    done.append(g)
        yield
        ring.busy -= 1
        out = []
        yield from waiter(ring, spins, out)
        if not out:
            return
        ring.busy += 1
        task = out[0]


@pytest.mark.parametrize("seed", range(200))
def test_every_task_runs_exactly_once(seed):
    rng = random.Random(seed)
    cap = rng.choice([2, 4, 8])
    nwarps = rng.choice([2, 3, 5, 8])
    ring = Ring(cap)
    ids = iter(range(10 ** 9))
    created = []

    def spawn(task):
        depth = task[1]
        kids = [(next(ids), depth + 1) for _ in range(rng.randint(0, 3 if depth < 3 else 0))]
        created.extend(kids)
        return kids

    roots = [(next(ids), 0) for _ in range(nwarps)]
    created.extend(roots)
    done = []
    ring.busy = nwarps
    warps = [worker(ring, rng, r, spawn, done, spins=rng.choice([3, 50, 10 ** 5])) for r in roots]
    live = list(warps)
    steps = 0
    while live:
        w = rng.choice(live)
        try:
            next(w)
        except StopIteration:
            live.remove(w)
        steps += 1
        assert steps < 2_000_000, "the warps did not finish"
    assert sorted(done) == sorted(created), "a task was lost or run twice"
    assert ring.busy == 0 and ring.idle == 0
