"""CPU model of the dataflow schedule (csrc/plan.cu tables, csrc/ntt.cu `k_dataflow_ntt2`),
checked without a GPU.

The plan numbers gates level-major and keeps, per gate, the number of its inputs that
are gates (pending) and the list of its consumers (a gate reading the same gate twice
appears twice).  The initial queue holds the gates that read only primary inputs.  Each
block takes tickets in order; ticket t waits until slot t of the queue holds a gate (or
t >= G: the block stops); a finished gate decrements its consumers' pending counts and
appends every consumer that reaches zero.  The model runs that protocol as an event
simulation with random gate durations and checks what the kernel relies on: every gate
is evaluated exactly once, only after all of its gate inputs finished, every ticket below
G is eventually served (no block waits forever), and every block stops.
"""
import heapq

import numpy as np
import pytest


def random_dag(rng, num_inputs, G, window):
    """Gate g reads two wires among the primaries and the `window` previous gates."""
    idx = np.zeros((G, 2), np.int64)
    for g in range(G):
        lo = max(0, num_inputs + g - window)
        idx[g] = rng.integers(lo, num_inputs + g, 2) if num_inputs + g > 0 else (0, 0)
    return idx


def plan_tables(num_inputs, idx):
    """pending counts, consumer lists (CSR) and the initial queue, as the plan builds them."""
    G = len(idx)
    pend = np.zeros(G, np.int64)
    cnt = np.zeros(G + 1, np.int64)
    for q in range(G):
        for w in idx[q]:
            if w >= num_inputs:
                cnt[w - num_inputs + 1] += 1
                pend[q] += 1
    off = np.cumsum(cnt)
    cons = np.zeros(max(off[-1], 1), np.int64)
    fill = off[:-1].copy()
    for q in range(G):
        for w in idx[q]:
            if w >= num_inputs:
                cons[fill[w - num_inputs]] = q
                fill[w - num_inputs] += 1
    queue0 = [q for q in range(G) if pend[q] == 0]
    return pend, off, cons, queue0


def simulate(num_inputs, idx, blocks, rng):
    G = len(idx)
    pend, off, cons, queue0 = plan_tables(num_inputs, idx)
    queue = queue0 + [None] * (G - len(queue0))
    pushed = len(queue0)
    next_ticket = 0
    waiting = {}          # ticket -> block waiting for that slot
    events = []           # (time, seq, block, gate)
    seq = 0
    start, finish = {}, {}
    stopped = set()
    now = 0.0

    def take(b):
        nonlocal next_ticket, seq
        t = next_ticket
        next_ticket += 1
        if t >= G:
            stopped.add(b)
            return
        if queue[t] is None:
            waiting[t] = b
            return
        begin(b, queue[t])

    def begin(b, g):
        nonlocal seq
        assert g not in start, "gate evaluated twice"
        for w in idx[g]:
            if w >= num_inputs:
                assert (w - num_inputs) in finish and finish[w - num_inputs] <= now, "input not ready"
        start[g] = now
        heapq.heappush(events, (now + rng.uniform(0.5, 1.5), seq, b, g))
        seq += 1

    for b in range(blocks):
        take(b)
    while events:
        now, _, b, g = heapq.heappop(events)
        finish[g] = now
        for e in range(off[g], off[g + 1]):
            c = cons[e]
            pend[c] -= 1
            assert pend[c] >= 0
            if pend[c] == 0:
                slot = pushed
                pushed += 1
                queue[slot] = c
                if slot in waiting:
                    begin(waiting.pop(slot), c)
        take(b)
    return start, finish, pushed, stopped, waiting


@pytest.mark.parametrize("seed,num_inputs,G,window,blocks", [
    (1, 8, 200, 10, 7), (2, 4, 300, 3, 16), (3, 16, 500, 50, 296), (4, 2, 120, 1, 5),
    (5, 1, 60, 2, 64), (6, 32, 1000, 200, 37)])
def test_every_gate_once_after_its_inputs_and_all_blocks_stop(seed, num_inputs, G, window, blocks):
    rng = np.random.default_rng(seed)
    idx = random_dag(rng, num_inputs, G, window)
    start, finish, pushed, stopped, waiting = simulate(num_inputs, idx, blocks, rng)
    assert len(start) == G and len(finish) == G
    assert pushed == G
    assert not waiting
    assert stopped == set(range(blocks))


def test_chain_and_repeated_input():
    """A chain (one ready gate at a time) and a gate reading the same gate twice: its
    consumer list holds it twice and its pending count is 2."""
    ni = 2
    idx = np.array([[0, 1], [2, 0], [3, 3], [4, 2], [0, 0]])
    pend, off, cons, queue0 = plan_tables(ni, idx)
    assert list(pend) == [0, 1, 2, 2, 0]
    assert list(cons[off[1]:off[2]]) == [2, 2]
    assert queue0 == [0, 4]
    start, finish, pushed, stopped, waiting = simulate(ni, idx, 3, np.random.default_rng(0))
    assert pushed == 5 and len(finish) == 5 and not waiting
    assert start[1] >= finish[0] and start[2] >= finish[1] and start[3] >= finish[2]
