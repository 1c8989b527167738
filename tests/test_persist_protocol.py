"""Model check of the halo exchange of the persistent batched recursion.

A cluster of K CTAs runs one work item (one column chunk of one cell) for
all M moments: CTA `rank` holds band rank (R = ceil(ny / K) lattice rows,
rows [y0, y1)) of V_m in shared memory.  Its two halo rows, lattice rows
y0 - 1 and y1 (periodic), are the last row of band ra and the first row of
band rb.  They come through exchange slots in global memory: slot (k, h, p)
holds the first (h = 0) or last (h = 1) row of band k at parity p.  Before
the first step every CTA writes the parity-0 slots of V_0; step m reads the
parity m & 1 slots of bands ra and rb, computes V_{m+1} and writes its own
boundary rows to the parity (m + 1) & 1 slots; a cluster barrier ends every
step; after the last step the CTA reads the parity (M - 1) & 1 slots once
more for the last moment's sums, and a final barrier ends the item before
the next item's V_0 goes into the parity-0 slots.

Between two barriers the CTAs run in any order, so the protocol is correct
when, in every such interval, no slot is both written and read (or written
twice), and every read sees the row of the moment it needs.  This test
replays the kernel's index arithmetic (the same formulas for R, y0, y1, ra,
rb) for every lattice height up to 40, clusters of 8 (and 2, 4, 16), orders
M = 1 .. 6 and several items in a row, and checks both properties and that
the halo rows are the lattice neighbours of the band.
"""
import pytest


def _wrap(v, n):
    return v % n


def _bands(ny, K):
    R = -(-ny // K)
    out = []
    for rank in range(K):
        y0 = min(ny, rank * R)
        y1 = min(ny, y0 + R)
        ra = _wrap(y0 - 1, ny) // R
        rb = _wrap(y1, ny) // R
        out.append((y0, y1, ra, rb))
    return R, out


def _replay(ny, K, M, items=3):
    R, bands = _bands(ny, K)
    # slot contents: (item, moment, band, side) of the row it holds
    slots = {}
    intervals = []  # per barrier interval: list of (op, slot, value)

    def new_interval():
        intervals.append([])

    for item in range(items):
        # initial rows of V_0 (parity 0), then the item's first barrier
        new_interval()
        for k, (y0, y1, ra, rb) in enumerate(bands):
            if y1 > y0:
                for h in (0, 1):
                    intervals[-1].append(("w", (k, h, 0), (item, 0, k, h)))
        for m in range(M - 1):
            new_interval()
            p, q = m & 1, (m + 1) & 1
            for k, (y0, y1, ra, rb) in enumerate(bands):
                if y1 <= y0:
                    continue
                intervals[-1].append(("r", (ra, 1, p), (item, m, ra, 1)))
                intervals[-1].append(("r", (rb, 0, p), (item, m, rb, 0)))
                for h in (0, 1):
                    intervals[-1].append(("w", (k, h, q), (item, m + 1, k, h)))
        # the last moment's sums read the halo of V_{M-1}, then the item ends
        if M >= 2:
            new_interval()
            p = (M - 1) & 1
            for k, (y0, y1, ra, rb) in enumerate(bands):
                if y1 > y0:
                    intervals[-1].append(("r", (ra, 1, p), (item, M - 1, ra, 1)))
                    intervals[-1].append(("r", (rb, 0, p), (item, M - 1, rb, 0)))

    for ops in intervals:
        written = {}
        read = set()
        for op, slot, val in ops:
            if op == "w":
                assert slot not in written, f"slot {slot} written twice between barriers"
                written[slot] = val
            else:
                read.add(slot)
        assert not (read & set(written)), f"slots {sorted(read & set(written))} read and written between barriers"
        for op, slot, val in ops:
            if op == "r":
                assert slots.get(slot) == val, f"slot {slot} holds {slots.get(slot)}, needed {val}"
        slots.update(written)
    return R, bands


@pytest.mark.parametrize("K", [8, 2, 4, 16])
def test_exchange_is_race_free_and_current(K):
    for ny in range(2, 41):
        for M in range(1, 7):
            _replay(ny, K, M)


@pytest.mark.parametrize("K", [8, 2, 4, 16])
def test_halo_rows_are_the_lattice_neighbours(K):
    for ny in range(2, 41):
        R, bands = _bands(ny, K)
        rows = set()
        for k, (y0, y1, ra, rb) in enumerate(bands):
            if y1 <= y0:
                continue
            rows.update(range(y0, y1))
            a0, a1 = bands[ra][0], bands[ra][1]
            b0, b1 = bands[rb][0], bands[rb][1]
            assert a1 > a0 and b1 > b0, "a halo comes from an empty band"
            assert a1 - 1 == _wrap(y0 - 1, ny), "row y0 - 1 is not the last row of band ra"
            assert b0 == _wrap(y1, ny), "row y1 is not the first row of band rb"
        assert rows == set(range(ny)), "the bands do not cover the lattice"
