"""CPU check of the shared-memory schedule of the stream sweep kernels.

The x and y/z stream kernels pass edge values and face fluxes between
neighbouring cells through rings in shared memory indexed by the cell (y/z:
c mod (rows per chunk + 1); x: slot mod (slots per chunk + 1)) and hold the
y/z primitive rows in a ring of twice the rows per chunk.  Each chunk has two
barriers: after the edge values are written (phase A) and after the fluxes
are written (phase B); the finish of the chunk (phase C) runs in the same
barrier interval as the next chunk's phase A.  This test replays that schedule
for the chunk sizes in the kernel source and checks that every read of a ring
slot sees the write of the cell it wants, with no other write to that slot
ordered in between or unordered against either access.  It models the index
arithmetic and the barrier placement, not the kernel: the kernels' results
are checked against the oracle on the GPU."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), os.pardir, "paper_2305_09163_gb300", "csrc",
                   "mfc_sweeps.cuh")


def _constant(name):
    with open(SRC) as f:
        m = re.search(r"constexpr int %s = (\d+);" % name, f.read())
    assert m, name
    return int(m.group(1))


def _interval(chunk, phase):
    """Barrier interval of a phase: A_k -> 2k, B_k -> 2k+1, C_k -> 2k+2 (the
    interval of A_{k+1}: no barrier between a chunk's finish and the next chunk)."""
    return 2 * chunk + {"A": 0, "B": 1, "C": 2}[phase]


def _hazards(writes, reads):
    """writes: list of (interval, key, slot); reads: list of (interval, key, slot).
    A read is safe if its key's write comes in an earlier interval and no write of
    another key to the same slot falls in [write interval, read interval]."""
    by_key = {}
    for t, key, slot in writes:
        assert key not in by_key, key
        by_key[key] = (t, slot)
    by_slot = {}
    for t, key, slot in writes:
        by_slot.setdefault(slot, []).append((t, key))
    bad = []
    for tr, key, slot in reads:
        tw, ws = by_key[key]
        assert ws == slot
        if not tw < tr:
            bad.append(("read before write", key, tw, tr))
            continue
        for tx, other in by_slot[slot]:
            if other != key and tw <= tx <= tr:
                bad.append(("overwritten", key, other, tw, tx, tr))
    return bad


def _edge_and_flux_schedule(cells_per_chunk, ring, first, chunks):
    """Edge values and fluxes of the stream kernels: chunk k covers cells
    first + k*R .. first + k*R + R - 1; the edge value of cell c is written in
    A and read by cell c+1 in B, its flux written in B and read by cell c+1's
    finish in C."""
    R = cells_per_chunk
    chunk_of = lambda c: (c - first) // R
    ew, er, fw, fr = [], [], [], []
    last = first + chunks * R - 1
    for c in range(first, last + 1):
        k = chunk_of(c)
        ew.append((_interval(k, "A"), c, c % ring))
        fw.append((_interval(k, "B"), c, c % ring))
        if c + 1 <= last:
            k1 = chunk_of(c + 1)
            er.append((_interval(k1, "B"), c, c % ring))
            fr.append((_interval(k1, "C"), c, c % ring))
    return _hazards(ew, er) + _hazards(fw, fr)


def _primitive_row_schedule(rows_per_chunk, s0, chunks):
    """Primitive rows of the y/z kernel: a ring of 2R rows; the prologue loads
    rows s0-3 .. s0+4 before the first barrier, chunk k (base = s0-1+kR) reads
    rows base-2 .. base+R+1 in A and writes the prefetched rows base+2R-2 ..
    base+3R-3 in B, after the first barrier."""
    R = rows_per_chunk
    ring = 2 * R
    writes, reads = [], []
    for h in range(2):
        for row in range(R):
            i = s0 - 3 + row + R * h
            writes.append((-1, i, i % ring))
    for k in range(chunks):
        base = s0 - 1 + k * R
        for i in range(base - 2, base + R + 2):
            reads.append((_interval(k, "A"), i, i % ring))
        for row in range(R):
            i = base + ring - 2 + row
            writes.append((_interval(k, "B"), i, i % ring))
    return _hazards(writes, reads)


@pytest.mark.parametrize("first", [-1, 0, 5, 130])
def test_yz_edge_and_flux_rings_are_race_free(first):
    R = _constant("kRowsPerChunk")
    assert _edge_and_flux_schedule(R, R + 1, first, 12) == []


@pytest.mark.parametrize("first", [-2, 0, 126, 2046])
def test_x_edge_and_flux_rings_are_race_free(first):
    T = _constant("kStreamThreads")
    assert _edge_and_flux_schedule(T, T + 1, first, 6) == []


@pytest.mark.parametrize("s0", [0, 7, 64])
def test_yz_primitive_ring_is_race_free(s0):
    assert _primitive_row_schedule(_constant("kRowsPerChunk"), s0, 12) == []


def test_the_check_finds_a_ring_one_row_short():
    """A ring of R rows (no room for the previous chunk's last cell) or a
    primitive ring of 2R-1 rows must fail: the check can see a race."""
    R = _constant("kRowsPerChunk")
    assert _edge_and_flux_schedule(R, R, 0, 6)
    T = _constant("kStreamThreads")
    assert _edge_and_flux_schedule(T, T, 0, 4)

    def short_ring(rows_per_chunk, s0, chunks):
        ring = 2 * rows_per_chunk - 1
        writes, reads = [], []
        for i in range(s0 - 3, s0 + 5):
            writes.append((-1, i, i % ring))
        for k in range(chunks):
            base = s0 - 1 + k * rows_per_chunk
            for i in range(base - 2, base + rows_per_chunk + 2):
                reads.append((_interval(k, "A"), i, i % ring))
            for row in range(rows_per_chunk):
                i = base + 2 * rows_per_chunk - 2 + row
                writes.append((_interval(k, "B"), i, i % ring))
        return _hazards(writes, reads)

    assert short_ring(R, 0, 6)
