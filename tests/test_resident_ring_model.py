"""Host model of the resident-slab form's schedule ring (no GPU needed).

The resident path of the stream kernel copies the schedule blob in fixed
chunks into a ring of `nst` shared-memory stages; a producer refills a stage
only after every consumer warp has released the chunk it held, a warp releases
the chunks before an item when it prepares that item, waits for the chunks the
item covers, reads this thread's first op of it, and meets the other warps at a
barrier where a level ends.  This model runs the same protocol step by step,
with the warps and the producer interleaved at random, over item lists laid out
the way the planner lays out a blob (windows of level-ordered tiles, padding
between windows, local records without ops).  It checks that every read finds
its chunk in its stage and that no interleaving deadlocks, for 2, 4 and 8
stages.
"""
import random

import pytest

CH = 16  # 8-byte units per chunk (the kernel uses 2,048; small chunks make crossings frequent)
TILE = 14  # ops per tile at most (the kernel: 2,046, one stage minus two units)


def blob_items(rng, windows):
    """Items (offset, count, level_end, local) in blob order, as the planner
    concatenates its windows: a local record is one item; a global window is a
    run of level-ordered tiles, its op region padded to an even length."""
    items, off = [], 0
    for _ in range(windows):
        if rng.random() < 0.2:
            n8 = 2 * rng.randint(1, CH // 2)  # whole 16-byte units, never more than one stage
            items.append((off, n8, False, True))
            off += n8
            continue
        nops = 0
        for _ in range(rng.randint(1, 6)):
            level = rng.randint(1, 3 * TILE)
            q = 0
            while q < level:
                c = min(TILE, level - q)
                items.append((off + nops + q, c, q + c == level, False))
                q += c
            nops += level
        off += (nops + 1) & ~1
    return items, off


class Ring:
    def __init__(self, items, blob8, nst, warps):
        self.items, self.nst, self.W = items, nst, warps
        self.nchunks = (blob8 + CH - 1) // CH
        self.stage = [None] * nst  # chunk each stage holds
        self.filled = 0  # chunks copied so far (in order)
        self.released = [0] * warps  # chunks each warp has released
        self.waited = [0] * warps  # chunks each warp has seen land
        # per warp: next action index into a flat program
        self.pc = [0] * warps
        self.prog = self.program()
        self.at_barrier = [False] * warps

    def program(self):
        """The consumer's action sequence: prepare item 0, then for every item
        apply it, prepare the next, and meet at the barrier of a level end."""
        prog = [("prepare", 0)]
        for i, (_, _, level_end, _) in enumerate(self.items):
            prog.append(("apply", i))
            if i + 1 < len(self.items):
                prog.append(("prepare", i + 1))
                if level_end:
                    prog.append(("barrier", i))
        return prog

    def chunks_of(self, i):
        off, count, _, _ = self.items[i]
        return off // CH, (off + count - 1) // CH

    def read(self, i, w):
        """A warp reads item i's ops (or header): every chunk must sit in its stage."""
        c0, c1 = self.chunks_of(i)
        for c in range(c0, c1 + 1):
            assert c < self.waited[w], "read before the chunk was waited for"
            assert self.stage[c % self.nst] == c, "stage was refilled while still in use"

    def producer_can(self):
        c = self.filled
        if c >= self.nchunks:
            return False
        return c < self.nst or min(self.released) > c - self.nst

    def producer_step(self):
        c = self.filled
        self.stage[c % self.nst] = c
        self.filled += 1

    def warp_step(self, w):
        """One action of warp w if it can make progress; returns False if blocked."""
        if self.pc[w] >= len(self.prog):
            return False
        kind, i = self.prog[self.pc[w]]
        if kind == "prepare":
            c0, c1 = self.chunks_of(i)
            if self.released[w] < c0:  # release first (never blocks)
                self.released[w] = c0
                return True
            if self.waited[w] <= c1:
                if self.filled <= self.waited[w]:
                    return False  # the chunk has not landed
                self.waited[w] += 1
                return True
            self.read(i, w)  # this thread's first op of the item
        elif kind == "apply":
            if not self.items[i][3]:
                self.read(i, w)
        else:  # barrier
            if not self.at_barrier[w]:
                self.at_barrier[w] = True
                return True
            if not all(self.at_barrier[x] and self.prog[self.pc[x]] == ("barrier", i) for x in range(self.W)):
                return False
            # the last warp to see everyone there releases the barrier for all
            for x in range(self.W):
                self.at_barrier[x] = False
                self.pc[x] += 1
            return True
        self.pc[w] += 1
        return True

    def run(self, rng):
        steps = 0
        while any(pc < len(self.prog) for pc in self.pc) or self.producer_can():
            agents = [-1] + list(range(self.W))
            rng.shuffle(agents)
            moved = False
            for a in agents:
                if a < 0:
                    if self.producer_can():
                        self.producer_step()
                        moved = True
                        break
                elif self.warp_step(a):
                    moved = True
                    break
            assert moved, "deadlock: no warp and no copy can make progress"
            steps += 1
        return steps


@pytest.mark.parametrize("nst", [2, 4, 8])
@pytest.mark.parametrize("seed", range(25))
def test_ring_protocol_never_reads_a_refilled_stage_nor_deadlocks(nst, seed):
    rng = random.Random(1000 * nst + seed)
    items, blob8 = blob_items(rng, rng.randint(1, 40))
    ring = Ring(items, blob8, nst, warps=rng.choice([1, 2, 4, 8]))
    ring.run(rng)
    assert ring.filled == ring.nchunks
    assert all(pc == len(ring.prog) for pc in ring.pc)


def test_blob_layout_covers_every_chunk():
    """Items cover the blob with gaps of at most one unit (a window's padding
    after an odd number of ops, so at an odd offset, never at a chunk start):
    every chunk holds part of some item, and the producer never copies a chunk
    that no warp waits for and releases."""
    rng = random.Random(7)
    for _ in range(200):
        items, blob8 = blob_items(rng, rng.randint(1, 30))
        covered = set()
        for off, count, _, _ in items:
            covered.update(range(off // CH, (off + count - 1) // CH + 1))
        assert covered == set(range((blob8 + CH - 1) // CH))
        ends = [o + c for o, c, _, _ in items]
        for (o, _, _, _), e in zip(items[1:], ends):
            assert 0 <= o - e <= 1
            if o - e == 1:
                assert e % 2 == 1  # the padding unit sits at an odd offset
        assert 0 <= blob8 - ends[-1] <= 1
