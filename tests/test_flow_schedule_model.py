"""A CPU model of the dataflow layer launch's schedule (sz_flow_c128).

The launch numbers its work items (layer s, matrix c, chain slot) in that order and
hands them out from one atomic counter.  An item waits for the done flags of the s
chains it reads (its predecessors in layer s - 1) and for every chain of layer s - 2.
Three layer regions rotate: layer s writes region s mod 3, which held layer s - 3.

The model replays that scheme with a pool of persistent workers (the CTAs) and
random chain durations, and checks what the kernel relies on:
  * every item a wait names has a smaller number, so it was taken by a running worker;
  * no layer overwrites a region slot while a chain of the layer that region held
    might still read it;
  * the pool never deadlocks, whatever the number of workers.
The predecessor slots use the colex rank of H minus one column, the formula the
kernels use, checked here against ranks listed by brute force."""
import heapq
import itertools
import math
import random

import pytest


def colex_subsets(t, s):
    """All s-subsets of {0..t-1} in colex order (rank = position)."""
    subs = [tuple(c) for c in itertools.combinations(range(t), s)]
    return sorted(subs, key=lambda c: tuple(reversed(c)))


def rank_without(h, p):
    """Colex rank of the sorted set h minus its p-th element."""
    return (sum(math.comb(b, q + 1) for q, b in enumerate(h) if q < p)
            + sum(math.comb(b, q) for q, b in enumerate(h) if q > p))


def items(t, count):
    """Item list in launch order: (s, c, slot, H, predecessor slots)."""
    out = []
    for s in range(t + 1):
        subs = colex_subsets(t, s)
        for c in range(count):
            for slot, h in enumerate(subs):
                out.append((s, c, slot, h, [rank_without(h, p) for p in range(s)]))
    return out


@pytest.mark.parametrize("t", [1, 3, 5, 8])
def test_predecessor_slots_are_colex_ranks(t):
    for s in range(1, t + 1):
        index = {h: r for r, h in enumerate(colex_subsets(t, s - 1))}
        for h in colex_subsets(t, s):
            for p in range(s):
                assert rank_without(h, p) == index[tuple(b for q, b in enumerate(h) if q != p)]


@pytest.mark.parametrize("t,count", [(3, 1), (5, 2), (7, 4), (8, 1)])
def test_waits_name_earlier_items(t, count):
    its = items(t, count)
    number = {(s, c, slot): i for i, (s, c, slot, _, _) in enumerate(its)}
    for i, (s, c, slot, h, preds) in enumerate(its):
        for ps in preds:
            assert number[(s - 1, c, ps)] < i
        if s >= 2:
            last_of_layer = max(number[(s - 2, cc, x)] for cc in range(count)
                                for x in range(math.comb(t, s - 2)))
            assert last_of_layer < i


def simulate(t, count, workers, rng, regions=3, wait_two_back=True, dur=(0.5, 2.0)):
    """Event simulation: each worker takes the next item number, waits for its
    dependencies, then runs for a random time.  Over its whole run a chain reads its
    predecessors' slots of region (s - 1) mod 3 and writes its own slot of region
    s mod 3.  Afterwards, every use of a region slot must be disjoint in time from
    every use of the same slot by another layer.  Returns the end time.  `regions` and
    `wait_two_back` exist to plant mistakes: fewer regions, or no wait for layer s - 2."""
    its = items(t, count)
    done = {}                                  # (s, c, slot) -> end time
    layer_end = [0.0] * (t + 1)                # time the last chain of a layer ended
    uses = {}                                  # (c, region, slot) -> [(layer, start, end)]
    free = [(0.0, w) for w in range(workers)]  # (time free, worker): persistent workers
    heapq.heapify(free)
    for s, c, slot, h, preds in its:           # items are handed out in number order
        tfree, w = heapq.heappop(free)
        deps = [done[(s - 1, c, ps)] for ps in preds]
        if s >= 2 and wait_two_back:
            deps.append(layer_end[s - 2])      # every chain of layer s - 2, all matrices
        start = max([tfree] + deps)
        end = start + rng.uniform(*dur)
        for ps in preds:
            uses.setdefault((c, (s - 1) % regions, ps), []).append((s - 1, start, end))
        uses.setdefault((c, s % regions, slot), []).append((s, start, end))
        done[(s, c, slot)] = end
        layer_end[s] = max(layer_end[s], end)
        heapq.heappush(free, (end, w))
    for key, iv in uses.items():
        for (l1, a1, b1), (l2, a2, b2) in itertools.combinations(iv, 2):
            if l1 != l2:
                assert b1 <= a2 or b2 <= a1, ("slot used by two layers at once", key, l1, l2)
    return max(layer_end)


@pytest.mark.parametrize("t,count", [(4, 1), (6, 3), (8, 1), (8, 4)])
@pytest.mark.parametrize("workers", [1, 3, 17, 456])
def test_random_schedules_complete_safely(t, count, workers):
    rng = random.Random(1000 * t + 10 * count + workers)
    for dur in ((0.5, 2.0), (0.1, 5.0)):
        for _ in range(3):
            simulate(t, count, workers, rng, dur=dur)


@pytest.mark.parametrize("regions,wait_two_back", [(2, True), (3, False)])
def test_planted_schedule_mistakes_are_caught(regions, wait_two_back):
    """Two rotating regions, or three without the wait for layer s - 2, let a layer
    overwrite a slot that another layer still uses: the model must report it."""
    rng = random.Random(77)
    caught = 0
    for _ in range(20):
        try:
            simulate(8, 2, 456, rng, regions=regions, wait_two_back=wait_two_back, dur=(0.1, 5.0))
        except AssertionError:
            caught += 1
    assert caught > 0
