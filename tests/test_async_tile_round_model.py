"""Model check of a dependency-driven round over TMA-staged tiles
(batch_euler_kernel<..., ASYNC = true> in batch_kernels.cuh), on the CPU.

Each CTA has one producer thread and W consumer warps joined by a ring of NS
slots (full / empty barriers).  The producer takes the round's tasks from one
counter, `chunk` at a time, waits until the task's problem has published
n x tiles x W consumer-warp completions (round step n > 0; skipped when the
previous task had the same problem and step), waits for the slot to be
released by all W consumer warps and stages the tile (the copy lands at any
later time); when the counter runs dry it writes an end marker.  Consumer
warps wait for the slot, meet at a barrier of the CTA's consumers, update
their part of the tile and release the slot.  They publish completions late
and in runs: the completed tiles of one problem accumulate and are published
(1) after the faces of a tile of another problem or after `run` tiles, (2)
before the warp blocks on a slot whose tile has not landed, and (3) at the
end.

Checked over random interleavings: the round ends (no deadlock); every task
is staged once and updated by every consumer warp once; a tile of step n is
staged only after every tile of its problem's step n - 1 has been updated by
all warps (its dt and halo come from that step); no slot is restaged while a
warp still reads it.

Planted faults that the model must catch: a dependency threshold one step
short, and consumer warps that do not publish before blocking (a producer
then waits for completions its own CTA's consumers hold back).
"""
import random

import pytest

from tests.test_async_round_model import round_tables

END = "end"


class TileRound:
    def __init__(self, problems, ctas, warps, ns, chunk, run, seed, fault=None):
        self.problems = problems
        _, self.table, _, self.cum, self.K = round_tables(problems)
        self.total = self.cum[-1]
        self.ctas, self.W, self.NS, self.chunk, self.run_len = ctas, warps, ns, chunk, run
        self.fault = fault
        self.rnd = random.Random(seed)
        self.next = 0
        self.done = [0] * len(problems)   # published consumer-warp completions per problem
        self.updated = {}                 # (problem, step) -> consumer-warp tile updates
        self.staged = [0] * self.total
        self.inflight = []                # (cta, slot) copies issued, not landed
        # per CTA: completed phases of full / empty per slot, pending empty
        # arrivals, slot headers, consumer barrier arrivals per ring sequence
        self.full = [[0] * ns for _ in range(ctas)]
        self.empty = [[0] * ns for _ in range(ctas)]
        self.empty_arr = [[0] * ns for _ in range(ctas)]
        self.hdr = [[None] * ns for _ in range(ctas)]
        self.bar = [{} for _ in range(ctas)]

    def step_of(self, k):
        lo, hi = 0, self.K
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if self.cum[mid] <= k:
                lo = mid
            else:
                hi = mid
        return lo

    def producer(self, c):
        seq = 0
        c_lo = c_hi = 0
        dep = None
        while True:
            have = False
            if c_lo == c_hi:
                lo = self.next
                self.next += self.chunk
                yield None
                c_lo, c_hi = lo, min(lo + self.chunk, self.total)
            if c_lo < c_hi:
                k = c_lo
                c_lo += 1
                n = self.step_of(k)
                p = self.table[k - self.cum[n]]
                if n > 0 and dep != (p, n):
                    need = (n - (1 if self.fault == "short_wait" else 0)) * self.problems[p][0] * self.W
                    yield lambda p=p, need=need: self.done[p] >= need
                    dep = (p, n)
                have = True
            s = seq % self.NS
            if seq >= self.NS:
                yield lambda s=s, ph=seq // self.NS: self.empty[c][s] >= ph
            if not have:
                self.hdr[c][s] = END
                self.full[c][s] += 1
                return
            if n > 0:
                assert self.updated.get((p, n - 1), 0) == self.problems[p][0] * self.W, \
                    f"problem {p}: a tile of step {n} staged before step {n - 1} was complete"
            self.staged[k] += 1
            self.hdr[c][s] = (k, p, n)
            self.inflight.append((c, s))
            seq += 1
            yield None

    def consumer(self, c, w):
        seq = 0
        pend, npend = None, 0

        def publish():
            nonlocal pend, npend
            self.done[pend] += npend
            pend, npend = None, 0

        while True:
            s, ph = seq % self.NS, seq // self.NS
            if pend is not None and self.full[c][s] < ph + 1 and self.fault != "no_publish_before_block":
                publish()
            yield lambda s=s, ph=ph: self.full[c][s] >= ph + 1
            h = self.hdr[c][s]
            bar = self.bar[c]
            bar[seq] = bar.get(seq, 0) + 1
            yield lambda seq=seq: self.bar[c][seq] == self.W
            if h == END:
                break
            k, p, n = h
            if pend is not None and (pend != p or npend >= self.run_len):
                publish()
            assert self.hdr[c][s] == h, "slot restaged while a warp reads it"
            self.updated[(p, n)] = self.updated.get((p, n), 0) + 1
            yield None
            pend = p
            npend += 1
            self.empty_arr[c][s] += 1
            if self.empty_arr[c][s] == self.W:
                self.empty_arr[c][s] = 0
                self.empty[c][s] += 1
            seq += 1
        if pend is not None:
            publish()

    def run(self):
        gens = [self.producer(c) for c in range(self.ctas)]
        gens += [self.consumer(c, w) for c in range(self.ctas) for w in range(self.W)]
        cond = [None] * len(gens)
        live = list(range(len(gens)))
        for _ in range(2_000_000):
            if not live:
                break
            if self.inflight and self.rnd.random() < 0.3:
                c, s = self.inflight.pop(self.rnd.randrange(len(self.inflight)))
                self.full[c][s] += 1
                continue
            ready = [i for i in live if cond[i] is None or cond[i]()]
            if not ready:
                if self.inflight:
                    continue
                raise AssertionError("deadlock: every producer and consumer waits")
            i = self.rnd.choice(ready)
            try:
                cond[i] = next(gens[i])
            except StopIteration:
                live.remove(i)
        assert not live, "model did not finish"
        assert all(x == 1 for x in self.staged), "a task was staged twice or never"
        for p, (tiles, steps) in enumerate(self.problems):
            for n in range(steps):
                assert self.updated.get((p, n), 0) == tiles * self.W


@pytest.mark.parametrize("seed", range(25))
def test_random_tile_rounds(seed):
    rnd = random.Random(2000 + seed)
    problems = [(rnd.randint(1, 6), rnd.randint(1, 5)) for _ in range(rnd.randint(1, 5))]
    ctas = rnd.randint(1, 3)
    for chunk in (1, 2, 3):
        for run in (1, 2, 16):
            for s in range(6):
                TileRound(problems, ctas, warps=2, ns=rnd.choice([2, 3, 4]), chunk=chunk, run=run, seed=s).run()


def test_one_tile_problem_on_one_cta():
    # consecutive steps of a one-tile problem follow each other in one chunk:
    # the producer waits for completions held by its own CTA's consumers
    for chunk in (1, 2, 4):
        for s in range(40):
            TileRound([(1, 8), (2, 3)], ctas=1, warps=2, ns=4, chunk=chunk, run=16, seed=s).run()


def test_catches_a_short_dependency_wait():
    with pytest.raises(AssertionError):
        for s in range(300):
            TileRound([(3, 5), (2, 4)], ctas=2, warps=2, ns=3, chunk=1, run=1, seed=s, fault="short_wait").run()


def test_catches_consumers_that_hold_completions_while_blocked():
    with pytest.raises(AssertionError, match="deadlock"):
        for s in range(300):
            TileRound([(1, 6)], ctas=1, warps=2, ns=4, chunk=2, run=16, seed=s,
                      fault="no_publish_before_block").run()
