"""Model check of the per-warp copy ring of the split FORCE walk sweeps
(euler_force_walk.cuh), on the CPU.

Each thread stages chunks (x sweep) or rows (y sweep) into NS shared-memory
slots with asynchronous copies, commits one copy group per staged chunk or
row, and waits with cp.async.wait_group (all but the N most recent groups of
the thread complete) before reading.  The model replays the kernel's order of
stage / commit / wait / read for one thread over several consecutive walks
and checks that

- every read of a slot finds the copy of the chunk or row it expects there,
  and that copy's group complete;
- no copy into a slot is issued while a chunk or row staged there earlier is
  still to be read (a refill only takes a slot whose contents were read);
- at the end of every walk all staged copies have been read.

Copies land at any time between their issue and their group's completion,
so "complete" is the only point at which a read may rely on them.  The
cross-lane part (SoA copies span two lanes' pairs) is covered by the warp
barrier that sits between every wait and read and before every refill, so
one thread's order is the whole protocol.
"""
import pytest


class Ring:
    def __init__(self, ns):
        self.ns = ns
        self.groups = []     # list of lists of (slot, tag) copies, in commit order
        self.pending = []    # copies issued since the last commit
        self.complete = 0    # groups [0, complete) are complete
        self.slot = [None] * ns        # tag of the last copy issued into each slot
        self.slot_group = [None] * ns  # group index of that copy
        self.unread = set()  # tags staged but not yet read

    def stage(self, slot, tag):
        assert self.slot[slot] not in self.unread, f"refill of slot {slot} before {self.slot[slot]} was read"
        self.pending.append((slot, tag))
        self.slot[slot] = tag
        self.slot_group[slot] = len(self.groups)  # the group the next commit forms
        self.unread.add(tag)

    def commit(self):
        self.groups.append(self.pending)
        self.pending = []

    def wait(self, n):
        self.complete = max(self.complete, len(self.groups) - n)

    def read(self, slot, tag):
        assert self.slot[slot] == tag, f"slot {slot} holds {self.slot[slot]}, expected {tag}"
        assert self.slot_group[slot] < self.complete, f"{tag} read before its copy group completed"
        self.unread.discard(tag)


def x_walk(r, ns, walk, nch):
    """The x sweep: chunk k in slot k % NS, NS - 1 chunks ahead, wait<NS - 1>."""
    for k in range(ns - 1):
        if k < nch:
            r.stage(k, (walk, k))
        r.commit()
    slot = 0
    for k in range(nch):
        kn = k + ns - 1
        if kn < nch:
            r.stage(ns - 1 if slot == 0 else slot - 1, (walk, kn))
        r.commit()
        r.wait(ns - 1)
        r.read(slot, (walk, k))
        slot = 0 if slot == ns - 1 else slot + 1


def y_walk(r, ns, walk, nrows_interior):
    """The y sweep: row i (ys - 1 + i) in slot i % NS, NS - 2 rows ahead, wait<NS - 3>;
    rows i and i + 1 are read for interior row i (i >= 1), rows 0 and 1 first."""
    nrows = nrows_interior + 2
    for i in range(ns - 1):
        if i < nrows:
            r.stage(i, (walk, i))
        r.commit()
    r.wait(ns - 3)
    r.read(0, (walk, 0))
    r.read(1, (walk, 1))
    slot = 1
    for y in range(nrows_interior):
        i = y + 1
        ir = i + ns - 2
        sr = slot - 2 if slot >= 2 else slot + ns - 2
        if ir < nrows:
            r.stage(sr, (walk, ir))
        r.commit()
        r.wait(ns - 3)
        sn = 0 if slot == ns - 1 else slot + 1
        r.read(slot, (walk, i))
        r.read(sn, (walk, i + 1))
        slot = sn


@pytest.mark.parametrize("ns", [3, 4, 5, 6, 8])
def test_x_walk_ring(ns):
    for lengths in ([1], [2, 1], [5, 5, 5], [1, 7, 2, 26], list(range(1, 12))):
        r = Ring(ns)
        for w, nch in enumerate(lengths):
            x_walk(r, ns, w, nch)
            assert not r.unread, f"walk {w}: staged and never read {sorted(r.unread)}"


@pytest.mark.parametrize("ns", [3, 4, 5, 6, 8])
def test_y_walk_ring(ns):
    for lengths in ([1], [2, 1], [16, 16, 12], [1, 3, 26, 2], list(range(1, 20))):
        r = Ring(ns)
        for w, n in enumerate(lengths):
            y_walk(r, ns, w, n)
            assert not r.unread, f"walk {w}: staged and never read {sorted(r.unread)}"


def test_model_catches_a_short_wait():
    """The model is not vacuous: waiting for one group too few fails."""
    r = Ring(6)
    r_wait = r.wait
    r.wait = lambda n: r_wait(n + 1)
    with pytest.raises(AssertionError, match="before its copy group completed"):
        x_walk(r, 6, 0, 8)


def test_model_catches_an_early_refill():
    """Refilling the slot about to be read (instead of the one read last) fails."""
    r = Ring(6)
    with pytest.raises(AssertionError):
        r.stage(0, ("w", 0))
        r.commit()
        r.stage(0, ("w", 6))
