"""CPU model of the bulk-copy ring's refill rule (tile_points_ring in
round_kernels.cuh), run over random interleavings of the CTA's warps.

Rule modelled: a tile of nch chunks streams through NST stages (chunk g of
the CTA's running count in stage g mod NST).  At a tile's start one thread
issues chunks 0 .. min(nch, NST) - 1.  Each warp consumes the chunks in
order: it waits until its chunk has landed, reads it, and adds 1 to its
stage's release counter (the counters persist across tiles); the warp whose
add makes the counter a multiple of the warp count refills the stage with
the chunk NST ahead, when the tile has one.  Checked: no warp waits for a
chunk that is never issued, every chunk is issued once, and a stage is
refilled only after every warp has released the chunk it held.
"""
import random

NST, WARPS = 4, 8


def run_tiles(tiles, rng):
    rel = [0] * NST                 # per-stage release counters (shared memory)
    seq = 0
    stage_holds = {}                # stage -> chunk currently in it
    released = {}                   # chunk -> warps that released it
    issued = set()

    def issue(g):
        s = g % NST
        assert g not in issued, f"chunk {g} issued twice"
        if s in stage_holds:
            prev = stage_holds[s]
            assert released.get(prev, 0) == WARPS, f"stage {s} refilled while chunk {prev} is still read"
        stage_holds[s] = g
        issued.add(g)

    for nch in tiles:
        for c in range(min(nch, NST)):
            issue(seq + c)
        pos = [0] * WARPS           # next chunk (within the tile) of each warp
        steps = 0
        while min(pos) < nch:
            steps += 1
            assert steps < 100000, "no progress: a warp waits for a chunk nobody issues"
            w = rng.randrange(WARPS)
            c = pos[w]
            if c >= nch:
                continue
            g = seq + c
            if g not in issued:     # still waiting for its chunk to be issued / to land
                continue
            released[g] = released.get(g, 0) + 1
            s = g % NST
            old = rel[s]
            rel[s] += 1
            if (old + 1) % WARPS == 0 and c + NST < nch:
                issue(g + NST)
            pos[w] += 1
        seq += nch
    assert issued == set(range(seq))
    assert all(released[g] == WARPS for g in range(seq))


def test_refill_rule_random_interleavings():
    rng = random.Random(11)
    for _ in range(400):
        tiles = [rng.choice([1, 2, 3, 4, 5, 9, rng.randint(1, 24)]) for _ in range(rng.randint(1, 6))]
        run_tiles(tiles, rng)
