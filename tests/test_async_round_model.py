"""Model check of a dependency-driven round over walk units
(batch_euler_walk_async_kernel in euler_solo2d.cuh, launch_round_async in
batch.cu), on the CPU.

The host orders the round's Euler problems by remaining steps (most first),
so the problems still stepping at round step n are a prefix of the table, and
forms cum[n + 1] = cum[n] + the units of that prefix.  On the device every
warp takes tasks k = 0, 1, ... (step-major) from one counter, `chunk` at a
time; task k of round step n (cum[n] <= k < cum[n + 1]) is table entry
t = k - cum[n].  Before a unit of step n > 0 runs, its warp waits until the
problem's completion counter has reached n x (units of the problem); after
the unit it publishes one completion.

Checked over random interleavings of the warps (any warp may be slow at any
point, and a warp's unit and its publication are separate events):

- the round ends (no deadlock) with every task run exactly once;
- a unit of step n runs only after every unit of the problem's step n - 1
  has run (its dt and every cell it reads come from that step);
- every problem runs exactly its own number of steps.

Planted faults that the model must catch: a wait threshold one step short,
a publication before the unit's work, and completions published only at the
end of a chunk (a chunk holding two consecutive steps of a one-unit problem
then waits for itself).
"""
import random

import pytest


def round_tables(problems):
    """problems: list of (units, steps).  Returns the table (problem index per
    entry), cum and K as the host builds them."""
    order = sorted(range(len(problems)), key=lambda i: -problems[i][1])  # stable: most remaining steps first
    table = []
    for i in order:
        table += [i] * problems[i][0]
    begin = {}
    pos = 0
    for i in order:
        begin[i] = pos
        pos += problems[i][0]
    K = max(s for _, s in problems)
    cum = [0]
    for n in range(K):
        cum.append(cum[-1] + sum(problems[i][0] for i in order if problems[i][1] > n))
    return order, table, begin, cum, K


class Round:
    def __init__(self, problems, warps, chunk, seed, fault=None):
        self.problems = problems
        self.order, self.table, self.begin, self.cum, self.K = round_tables(problems)
        self.total = self.cum[-1]
        self.warps, self.chunk, self.fault = warps, chunk, fault
        self.rnd = random.Random(seed)
        self.next = 0
        self.done = [0] * len(problems)            # published completions per problem
        self.ran = {}                              # (problem, step) -> units run
        self.task_runs = [0] * self.total

    def step_of(self, k):
        lo, hi = 0, self.K
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if self.cum[mid] <= k:
                lo = mid
            else:
                hi = mid
        return lo

    def run_unit(self, k, n, p):
        if n > 0:
            assert self.ran.get((p, n - 1), 0) == self.problems[p][0], \
                f"problem {p}: a unit of step {n} ran before step {n - 1} was complete"
        self.ran[(p, n)] = self.ran.get((p, n), 0) + 1
        self.task_runs[k] += 1

    def warp(self):
        c_lo = c_hi = 0
        s_lo = s_hi = s_n = 0
        unpublished = []
        while True:
            if c_lo == c_hi:
                if self.fault == "publish_at_chunk_end":
                    for p in unpublished:
                        self.done[p] += 1
                    unpublished = []
                lo = self.next
                self.next += self.chunk  # one atomic add
                yield None
                if lo >= self.total:
                    return
                c_lo, c_hi = lo, min(lo + self.chunk, self.total)
            k = c_lo
            c_lo += 1
            if not (s_lo <= k < s_hi):
                s_n = self.step_of(k)
                s_lo, s_hi = self.cum[s_n], self.cum[s_n + 1]
            p = self.table[k - s_lo]
            if s_n > 0:
                need = (s_n - (1 if self.fault == "short_wait" else 0)) * self.problems[p][0]
                yield lambda p=p, need=need: self.done[p] >= need
            if self.fault == "publish_first":
                self.done[p] += 1
                yield None
                self.run_unit(k, s_n, p)
            else:
                self.run_unit(k, s_n, p)
                yield None  # the unit's stores, then the release add, as separate events
                if self.fault == "publish_at_chunk_end":
                    unpublished.append(p)
                else:
                    self.done[p] += 1

    def run(self):
        gens = [self.warp() for _ in range(self.warps)]
        cond = [None] * len(gens)
        live = list(range(len(gens)))
        for _ in range(1_000_000):
            if not live:
                break
            ready = [i for i in live if cond[i] is None or cond[i]()]
            assert ready, "deadlock: every warp waits"
            i = self.rnd.choice(ready)
            try:
                cond[i] = next(gens[i])
            except StopIteration:
                live.remove(i)
        assert not live, "model did not finish"
        assert all(c == 1 for c in self.task_runs), "a task ran twice or never"
        for p, (units, steps) in enumerate(self.problems):
            for n in range(steps):
                assert self.ran.get((p, n), 0) == units
            assert (p, steps) not in self.ran


def host_chunk(cum, workers, max_chunk=8):
    """The host's chunk: as many tasks as every worker gets per step, 1 .. 8."""
    return max(1, min(max_chunk, cum[1] // max(1, workers)))


@pytest.mark.parametrize("seed", range(30))
def test_random_rounds(seed):
    rnd = random.Random(1000 + seed)
    problems = [(rnd.randint(1, 7), rnd.randint(1, 6)) for _ in range(rnd.randint(1, 6))]
    warps = rnd.randint(1, 5)
    _, _, _, cum, _ = round_tables(problems)
    for chunk in sorted({1, 2, 3, host_chunk(cum, warps)}):
        for s in range(20):
            Round(problems, warps, chunk, seed=s).run()


def test_single_unit_problems_many_steps():
    # one-unit problems: consecutive steps of one problem are adjacent tasks
    problems = [(1, 9), (1, 4), (2, 7)]
    for chunk in (1, 2, 4, 8):
        for s in range(50):
            Round(problems, warps=3, chunk=chunk, seed=s).run()


def test_catches_a_short_wait():
    with pytest.raises(AssertionError):
        for s in range(200):
            Round([(3, 5), (2, 4)], warps=4, chunk=1, seed=s, fault="short_wait").run()


def test_catches_publication_before_the_work():
    with pytest.raises(AssertionError):
        for s in range(200):
            Round([(3, 5), (2, 4)], warps=4, chunk=1, seed=s, fault="publish_first").run()


def test_catches_publication_deferred_to_the_chunk_end():
    with pytest.raises(AssertionError, match="deadlock"):
        for s in range(200):
            Round([(1, 6)], warps=2, chunk=2, seed=s, fault="publish_at_chunk_end").run()
