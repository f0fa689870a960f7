"""The synchronisation protocol of the row sweep (euler_sweep_row3.cuh), checked
on a model before any GPU run and on every change since.

Actors: lane 0 of warp 0 (halo row below, also the TMA producer), the other
lanes of warp 0, the row warps 1..TY and warp TY+1 (halo row above); each runs
the kernel's sequence of waits, shared-memory reads and writes and arrivals for
a list of work items of zn planes.  A TMA copy lands at a random later time.
Warp 0 writes its outputs of plane iteration i (tile-edge x data and the y
state of the row below the tile) to buffer i mod 4 with its own mbarrier, after
every thread has released plane z - 4.

Modelled exactly as the hardware does them:
  * an mbarrier completes a phase when its arrival count is reached; a parity
    wait for phase k succeeds when the completed-phase count c has c & 1 !=
    k & 1.  A wait is "lapped" if it looks at the barrier when c > k + 1 (it
    would then wait for the wrong phase): the model asserts c <= k + 1 at every
    look, and success only at c == k + 1;
Checked for random interleavings: every actor finishes (no deadlock), no wait
is lapped, and every read sees the version of the data written for its own
plane (ring slots, the y-state rows, the y-face rows, warp 0's buffers).
"""
import random

import pytest

NS = 7  # ring slots


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.c = count, count, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.c += 1
            self.pending = self.count


class Model:
    def __init__(self, TY, items, seed):
        self.TY, self.items = TY, items
        self.rnd = random.Random(seed)
        NW = TY + 2
        self.NW = NW
        self.n_actors = 1 + 1 + TY + 1  # lane 0 of warp 0, other lanes of warp 0, row warps, warp TY+1
        self.full = [Bar(1) for _ in range(NS)]
        self.empty = [Bar(self.n_actors) for _ in range(NS)]
        self.rb = [Bar(1) for _ in range(NW)]
        self.fb = [Bar(1) for _ in range(NW)]
        self.NE = 4
        self.eb = [Bar(2) for _ in range(self.NE)]  # both actors of warp 0 arrive
        self.slot_ver = [None] * NS   # plane sequence number held by each slot
        self.ry_ver = [None] * (TY + 1)  # index w: y state of row w - 1 (written by row warp w)
        self.fy_ver = [None] * (TY + 1)
        self.edge_ver = {}            # buffer k -> iteration written by warp 0
        self.inflight = []            # (seq) copies issued, not landed
        self.issued = 0
        self.total_planes = sum(zn + 4 for zn in items)

    # ---- blocking conditions -------------------------------------------------
    def bar_ready(self, bar, k):
        assert bar.c <= k + 1, f"lapped wait: phase {k}, barrier at {bar.c}"
        return bar.c == k + 1

    # ---- actor programs (generators yield a condition to wait for) ------------
    def wait_full(self, st, seq):
        while st["waited"] <= seq:
            s = st["waited"]
            b = self.full[s % NS]
            yield lambda b=b, k=s // NS: self.bar_ready(b, k)
            st["waited"] += 1

    def read_plane(self, seq):
        assert self.slot_ver[seq % NS] == seq, f"slot holds plane {self.slot_ver[seq % NS]}, read wants {seq}"

    def release(self, seq):
        self.empty[seq % NS].arrive()

    def issue_until(self, limit):
        while self.issued < self.total_planes and self.issued < limit:
            p = self.issued
            if p >= NS:
                b = self.empty[p % NS]
                yield lambda b=b, k=p // NS - 1: self.bar_ready(b, k)
            self.inflight.append(p)
            self.issued += 1

    def program(self, role, w):
        st = {"waited": 0}
        seq_base = 0
        it = 0
        row = role == "row"
        for zn in self.items:
            if role == "w0lane0":
                yield from self.issue_until(seq_base + 5)
            yield from self.wait_full(st, seq_base + (3 if row else 1))
            if row:
                for j in range(4):
                    self.read_plane(seq_base + j)
            self.release(seq_base)
            self.release(seq_base + 1)
            for zl in range(zn):
                sz = seq_base + 2 + zl
                kb = it % self.NE
                if role in ("w0lane0", "w0rest"):
                    if sz >= 4:
                        sp = sz - 4
                        b = self.empty[sp % NS]
                        yield lambda b=b, k=sp // NS: self.bar_ready(b, k)
                    if role == "w0lane0":
                        yield from self.issue_until(sz + 4)
                yield from self.wait_full(st, sz + 2 if row else sz)
                if role in ("w0lane0", "w0rest"):
                    self.read_plane(sz)
                    self.edge_ver[kb] = it
                    self.eb[kb].arrive()
                elif role == "top":
                    self.read_plane(sz)
                    b = self.rb[self.TY]
                    yield lambda b=b, k=it: self.bar_ready(b, k)
                    assert self.ry_ver[self.TY] == it
                    self.fy_ver[self.TY] = it
                    self.fb[self.NW - 1].arrive()
                else:
                    for j in range(3):
                        self.read_plane(sz + j)
                    self.ry_ver[w] = it
                    self.rb[w].arrive()
                    if w == 1:
                        b = self.eb[kb]
                        yield lambda b=b, k=it // self.NE: self.bar_ready(b, k)
                        assert self.edge_ver[kb] == it
                    else:
                        b = self.rb[w - 1]
                        yield lambda b=b, k=it: self.bar_ready(b, k)
                        assert self.ry_ver[w - 1] == it, (w, it, self.ry_ver[w - 1])
                    self.fy_ver[w - 1] = it
                    self.fb[w].arrive()
                    b = self.eb[kb]
                    yield lambda b=b, k=it // self.NE: self.bar_ready(b, k)
                    assert self.edge_ver[kb] == it
                    b = self.fb[w + 1]
                    yield lambda b=b, k=it: self.bar_ready(b, k)
                    assert self.fy_ver[w] == it, (w, it, self.fy_ver[w])
                self.release(sz)
                it += 1
            yield from self.wait_full(st, seq_base + zn + 3)
            self.release(seq_base + zn + 2)
            self.release(seq_base + zn + 3)
            seq_base += zn + 4

    def run(self):
        TY = self.TY
        roles = [("w0lane0", 0), ("w0rest", 0)] + [("row", w) for w in range(1, TY + 1)] + [("top", TY + 1)]
        gens = [self.program(r, w) for r, w in roles]
        cond = [None] * len(gens)
        done = [False] * len(gens)
        for _ in range(10_000_000):
            # a copy in flight may land at any time
            if self.inflight and self.rnd.random() < 0.3:
                p = self.inflight.pop(self.rnd.randrange(len(self.inflight)))
                assert self.slot_ver[p % NS] is None or self.slot_ver[p % NS] == p - NS
                # every actor released the slot's previous plane (empty phase complete)
                self.slot_ver[p % NS] = p
                self.full[p % NS].arrive()
                continue
            ready = [i for i in range(len(gens)) if not done[i] and (cond[i] is None or cond[i]())]
            if not ready:
                if self.inflight:
                    continue
                assert all(done), "deadlock"
                return
            i = self.rnd.choice(ready)
            try:
                cond[i] = next(gens[i])
            except StopIteration:
                done[i] = True
                cond[i] = None
        raise AssertionError("model did not finish")


@pytest.mark.parametrize("items", [[1], [2, 3], [5, 1, 4], [32, 6], [3, 3, 3, 3]])
def test_row_sweep_protocol(items):
    for seed in range(40):
        Model(TY=4, items=items, seed=seed).run()


def test_row_sweep_protocol_full_tile():
    for seed in range(6):
        Model(TY=14, items=[6, 2], seed=seed).run()


def test_model_catches_a_shallow_gate():
    """A planted fault: warp 0 gated on plane z - 5 instead of z - 4 overwrites
    a buffer (or laps its barrier) before the row warps are done with it."""

    class Loose(Model):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            self.NE = 3
            self.eb = [Bar(2) for _ in range(3)]

    with pytest.raises(AssertionError):
        for seed in range(300):
            Loose(TY=3, items=[9, 5], seed=seed).run()


def test_model_catches_a_producer_without_slot_waits():
    """A planted fault: a producer that refills a ring slot without waiting for
    every thread to release the slot's previous plane overwrites a plane that
    a warp still reads."""

    class Eager(Model):
        def issue_until(self, limit):
            while self.issued < self.total_planes and self.issued < limit + 3:
                self.inflight.append(self.issued)
                self.issued += 1
            yield None

    with pytest.raises(AssertionError):
        for seed in range(200):
            Eager(TY=3, items=[8, 4], seed=seed).run()
