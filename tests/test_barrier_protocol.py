"""The named-barrier protocol of the split-barrier 3D sweep (euler_sweep_pair3.cuh),
checked on a model: for each tile of zn planes the pair warps (4) and the other
warps (4) issue, per plane zl,

  pair:  [zl+1 < zn] arrive PD[(zl+1) & 1];  sync FD;  [zl+1 < zn] arrive UD
  other: [zl > 0] sync PD[zl & 1], sync UD;  arrive FD

between full CTA barriers at each tile start and end.  A hardware barrier of
count 256 completes a phase once 8 warps arrived (arrive or sync); a sync
waits for its phase.  Every phase must consist of arrivals meant for the same
plane (no warp laps a barrier), and every interleaving must finish."""
import random

import pytest


def _program(role, zn, tiles, pd_ids=2):
    ops = []
    for t in range(tiles):
        ops.append(("full", None, (t, "start")))
        for zl in range(zn):
            if role == "pair":
                if zl + 1 < zn:
                    ops.append(("arrive", ("PD", (zl + 1) % pd_ids), (t, zl + 1)))
                ops.append(("sync", ("FD",), (t, zl)))
                if zl + 1 < zn:
                    ops.append(("arrive", ("UD",), (t, zl)))
            else:
                if zl > 0:
                    ops.append(("sync", ("PD", zl % pd_ids), (t, zl)))
                    ops.append(("sync", ("UD",), (t, zl - 1)))
                ops.append(("arrive", ("FD",), (t, zl)))
        ops.append(("full", None, (t, "end")))
    return ops


def _simulate(zn, tiles, seed, pd_ids=2):
    rnd = random.Random(seed)
    progs = [_program("pair" if w < 4 else "other", zn, tiles, pd_ids) for w in range(8)]
    pc = [0] * 8
    waiting = [None] * 8
    phases = {}
    while True:
        ready = [w for w in range(8) if pc[w] < len(progs[w]) and waiting[w] is None]
        if not ready:
            assert all(pc[w] == len(progs[w]) for w in range(8)), f"deadlock at {pc}"
            break
        w = rnd.choice(ready)
        op, bar, tag = progs[w][pc[w]]
        pc[w] += 1
        key = "full" if op == "full" else bar
        st = phases.setdefault(key, [0, []])
        st[1].append(tag)
        if op in ("sync", "full"):
            waiting[w] = (key, st[0])
        if len(st[1]) == 8:
            assert len(set(st[1])) == 1, f"barrier {key} mixes phases {sorted(set(st[1]))}"
            for v in range(8):
                if waiting[v] == (key, st[0]):
                    waiting[v] = None
            st[0] += 1
            st[1] = []
    assert all(not st[1] for st in phases.values()), "a barrier phase never completed"


@pytest.mark.parametrize("zn", [1, 2, 3, 4, 7, 32])
def test_split_barrier_protocol(zn):
    for seed in range(200):
        _simulate(zn, tiles=3, seed=seed)


def test_one_predicted_state_barrier_would_lap():
    # the pair warps run one plane ahead on the predicted-state hand-off: with a
    # single barrier instead of two alternating ones, some interleaving mixes planes
    with pytest.raises(AssertionError, match="mixes phases"):
        for seed in range(200):
            _simulate(6, tiles=2, seed=seed, pd_ids=1)
