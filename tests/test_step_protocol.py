"""Model check of the ring protocol of the TMA-staged FP32 recursion step.

The kernel keeps lattice rows y-1..y+1 of V_m in a 5-slot ring and the 2h~
entries of row y in a 3-slot ring, each slot completing on its own mbarrier
(one arrival with the expected byte count, then the copy's bytes), and has no
block barrier: every warp arrives on a row-done mbarrier (ring of three,
count = warps) when it has finished a row, and the issuing thread waits for
row y-1 to be done before it refills the window slot of row y-2 (with row
y+3) and the coefficient slot of row y-1 (with row y+2).  Waits test only the
parity of a phase, so the protocol must never let a barrier run two phases
ahead of a waiter, must never re-arm a slot whose copy is in flight, and must
never overwrite a slot a warp still reads.  This test replays the protocol
under random interleavings of warps and copy completions (a model of the
schedule, not the kernel) and checks exactly that, for short and long bands
and 1 to 16 warps.
"""
import random

import pytest


class _Bar:
    def __init__(self, count):
        self.phase = 0          # completed phases
        self.count = count
        self.pending = count
        self.armed = False

    def done(self, parity):     # mbarrier.try_wait.parity
        return (self.phase & 1) != parity


def _run(nrow, warps, seed):
    rng = random.Random(seed)
    fv = [_Bar(1) for _ in range(5)]
    fc = [_Bar(1) for _ in range(3)]
    dn = [_Bar(warps) for _ in range(3)]
    vslot = [None] * 5
    cslot = [None] * 3
    flight = []

    def issue(bars, slots, ring, kind, idx):
        b = bars[idx % ring]
        assert not b.armed, f"{kind} slot re-armed while its copy is in flight"
        b.armed = True
        b.pending = 0                       # arrive.expect_tx
        slots[idx % ring] = ("in flight", idx)
        flight.append((b, slots, idx % ring, idx))

    for w in range(0, min(3, nrow + 1) + 1):
        issue(fv, vslot, 5, "window", w)
    for c in range(0, min(1, nrow - 1) + 1):
        issue(fc, cslot, 3, "coefficient", c)
    state = [[0, "wait"] for _ in range(warps)]
    for _ in range(10 ** 6):
        live = [i for i, (q, _) in enumerate(state) if q < nrow]
        if not live and not flight:
            return
        moves = [("warp", i) for i in live] + ([("land", None)] if flight else [])
        kind, i = rng.choice(moves)
        if kind == "land":
            b, slots, s, idx = flight.pop(rng.randrange(len(flight)))
            slots[s] = ("ok", idx)
            b.phase += 1
            b.armed = False
            b.pending = 1
            continue
        q, st = state[i]
        if st == "wait":
            ok = q > 0 or (fv[0].done(0) and fv[1].done(0))
            ok = ok and fv[(q + 2) % 5].done(((q + 2) // 5) & 1) and fc[q % 3].done((q // 3) & 1)
            if ok:
                state[i][1] = "issue" if i == 0 else "compute"
        elif st == "issue":
            if q >= 1 and not dn[(q - 1) % 3].done(((q - 1) // 3) & 1):
                continue
            if q + 4 <= nrow + 1:
                issue(fv, vslot, 5, "window", q + 4)
            if q + 2 < nrow:
                issue(fc, cslot, 3, "coefficient", q + 2)
            state[i][1] = "compute"
        elif st == "compute":
            for w in (q, q + 1, q + 2):
                assert vslot[w % 5] == ("ok", w), (q, w, vslot[w % 5])
            assert cslot[q % 3] == ("ok", q)
            state[i][1] = "arrive"
        else:  # the reads of the row are over only now: nothing may have replaced them
            for w in (q, q + 1, q + 2):
                assert vslot[w % 5] == ("ok", w), ("overwritten", q, w)
            assert cslot[q % 3] == ("ok", q)
            b = dn[q % 3]
            b.pending -= 1
            if b.pending == 0:
                b.phase += 1
                b.pending = warps
            state[i] = [q + 1, "wait"]
    raise AssertionError("no progress: the protocol deadlocks")


@pytest.mark.parametrize("nrow", [1, 2, 3, 5, 7, 34])
@pytest.mark.parametrize("warps", [1, 2, 16])
def test_ring_protocol_random_schedules(nrow, warps):
    for seed in range(12):
        _run(nrow, warps, seed)
