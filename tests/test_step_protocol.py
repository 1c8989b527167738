"""Model check of the ring protocol of the TMA-staged FP32 recursion step.

The kernel keeps lattice rows y-1..y+1 of V_m (and the next rows in flight)
in a ring of VR slots and the 2h~ entries of row y in a ring of CR slots, each
slot completing on its own mbarrier (one arrival with the expected byte
count, then the copy's bytes), and has no block barrier: every warp arrives
on a row-done mbarrier (ring of DR, count = warps) when it has finished a
row, and the issuing thread waits for row y-1 to be done before it refills
the window slot of row y-2 (with row y+VR-3) and the coefficient slot of row
y-1 (with row y+CR-2).  The kernel uses VR, CR, DR = 5, 3, 3; a deeper
window ring (6, 3, 4) is checked too.  Waits test only the
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


def _run(nrow, warps, seed, VR=5, CR=3, DR=3):
    rng = random.Random(seed)
    fv = [_Bar(1) for _ in range(VR)]
    fc = [_Bar(1) for _ in range(CR)]
    dn = [_Bar(warps) for _ in range(DR)]
    vslot = [None] * VR
    cslot = [None] * CR
    flight = []

    def issue(bars, slots, ring, kind, idx):
        b = bars[idx % ring]
        assert not b.armed, f"{kind} slot re-armed while its copy is in flight"
        b.armed = True
        b.pending = 0                       # arrive.expect_tx
        slots[idx % ring] = ("in flight", idx)
        flight.append((b, slots, idx % ring, idx))

    for w in range(0, min(VR - 2, nrow + 1) + 1):
        issue(fv, vslot, VR, "window", w)
    for c in range(0, min(CR - 2, nrow - 1) + 1):
        issue(fc, cslot, CR, "coefficient", c)
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
            ok = ok and fv[(q + 2) % VR].done(((q + 2) // VR) & 1) and fc[q % CR].done((q // CR) & 1)
            if ok:
                state[i][1] = "issue" if i == 0 else "compute"
        elif st == "issue":
            if q >= 1 and not dn[(q - 1) % DR].done(((q - 1) // DR) & 1):
                continue
            if q + VR - 1 <= nrow + 1:
                issue(fv, vslot, VR, "window", q + VR - 1)
            if q + CR - 1 < nrow:
                issue(fc, cslot, CR, "coefficient", q + CR - 1)
            state[i][1] = "compute"
        elif st == "compute":
            for w in (q, q + 1, q + 2):
                assert vslot[w % VR] == ("ok", w), (q, w, vslot[w % VR])
            assert cslot[q % CR] == ("ok", q)
            state[i][1] = "arrive"
        else:  # the reads of the row are over only now: nothing may have replaced them
            for w in (q, q + 1, q + 2):
                assert vslot[w % VR] == ("ok", w), ("overwritten", q, w)
            assert cslot[q % CR] == ("ok", q)
            b = dn[q % DR]
            b.pending -= 1
            if b.pending == 0:
                b.phase += 1
                b.pending = warps
            state[i] = [q + 1, "wait"]
    raise AssertionError("no progress: the protocol deadlocks")


@pytest.mark.parametrize("rings", [(5, 3, 3), (6, 3, 4)])
@pytest.mark.parametrize("nrow", [1, 2, 3, 5, 7, 34])
@pytest.mark.parametrize("warps", [1, 2, 16])
def test_ring_protocol_random_schedules(rings, nrow, warps):
    for seed in range(12):
        _run(nrow, warps, seed, *rings)


def test_too_short_done_ring_is_caught():
    # warps may run CR - 1 rows apart: a row-done ring of CR - 1 phases aliases
    with pytest.raises(AssertionError):
        for seed in range(50):
            _run(34, 4, seed, 5, 3, 2)
