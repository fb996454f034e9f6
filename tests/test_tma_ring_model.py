"""CPU model of the TMA staging pipeline of the FP32 variable-coefficient CG
(csrc/hs_cg32v.cu).

One producer thread issues the plane copies of a block's work items, in
order, into NSLOT shared-memory slots.  Slot s has a "full" barrier (the
producer's arrival plus the copied bytes) and an "empty" barrier (one arrival
per compute warp).  Stream position q (counted over every pass of the launch)
uses slot q mod NSLOT for the (q div NSLOT)-th time: a compute warp waits for
the full barrier's phase of parity (q div NSLOT) mod 2, and the producer
waits for the empty barrier's previous phase before re-arming the slot.  A
compute warp at step z of an item reads planes z-1, z, z+1, and releases
plane z-1 after the step (planes z1-1 and z1 at the end of the item).

The model transcribes that index arithmetic and runs the producer and the
warps under random interleavings (as on the GPU, warps run at their own
pace: no block barrier inside a pass), checking that
  * no thread waits forever (the model makes progress until every pass ends);
  * a warp reads a slot only after the copy it waits for has landed, and the
    slot then holds exactly the (item, plane) the warp expects;
  * the producer re-arms a slot only after every warp released its previous
    plane, and the parities of both barriers match the phase counts;
  * at the end of a pass nothing is in flight.
It fails when a warp forgets one release (control below).
"""
import random

import pytest


def item_planes(item, tl, nz):
    tiles_x, tiles_y, lz = tl
    c = item // (tiles_x * tiles_y)
    z0 = c * lz
    z1 = min(nz, z0 + lz)
    return z0, z1, max(z0 - 1, 0), min(z1, nz - 1)


class Barrier:
    """An mbarrier: phases complete after `count` arrivals (and, for full
    barriers, the landing of the copy)."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0            # number of completed phases

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        # try_wait.parity: true once the phase with that parity completed
        # (the current, incomplete phase has parity self.phase % 2)
        return (self.phase % 2) != parity


def run(tl, nz, nwarps, nslot, ranks, size, passes, seed, skip_release=None):
    rnd = random.Random(seed)
    nitems = tl[0] * tl[1] * ((nz + tl[2] - 1) // tl[2])
    for rank in ranks:
        full = [Barrier(1) for _ in range(nslot)]
        empty = [Barrier(nwarps) for _ in range(nslot)]
        content = [None] * nslot
        cnt = 0
        for _ in range(passes):
            seq = [(item, z) for item in range(rank, nitems, size)
                   for z in range(item_planes(item, tl, nz)[2], item_planes(item, tl, nz)[3] + 1)]
            # producer: a generator that yields while it waits
            def producer():
                for q, (item, z) in enumerate(seq):
                    qa = cnt + q
                    slot, use = qa % nslot, qa // nslot
                    if use > 0:
                        while not empty[slot].done((use - 1) % 2):
                            yield
                        assert empty[slot].phase == use, "slot re-armed before every warp released it"
                    content[slot] = ("copying", qa, item, z)
                    yield                      # the copy is in flight
                    content[slot] = ("landed", qa, item, z)
                    full[slot].arrive()

            def warp(w):
                base = cnt
                for item in range(rank, nitems, size):
                    z0, z1, qlo, qhi = item_planes(item, tl, nz)

                    def wait_read(z):
                        qa = base + (z - qlo)
                        slot = qa % nslot
                        while not full[slot].done((qa // nslot) % 2):
                            yield
                        assert full[slot].phase == qa // nslot + 1
                        assert content[slot] == ("landed", qa, item, z), (content[slot], qa, item, z)

                    def release(z):
                        qa = base + (z - qlo)
                        if skip_release == (w, qa):
                            return
                        empty[qa % nslot].arrive()

                    if z0 - 1 >= 0:
                        yield from wait_read(z0 - 1)
                    yield from wait_read(z0)
                    for z in range(z0, z1):
                        if z + 1 <= nz - 1:
                            yield from wait_read(z + 1)
                        # the step reads planes z - 1, z, z + 1 again
                        if z > 0:
                            yield from wait_read(z - 1)
                        yield from wait_read(z)
                        yield
                        if z - 1 >= qlo:
                            release(z - 1)
                    release(z1 - 1)
                    if z1 <= qhi:
                        release(z1)
                    base += qhi - qlo + 1

            threads = [producer()] + [warp(w) for w in range(nwarps)]
            live = list(range(len(threads)))
            steps = 0
            while live:
                k = rnd.choice(live)
                try:
                    next(threads[k])
                except StopIteration:
                    live.remove(k)
                steps += 1
                if steps > 200000:
                    raise AssertionError("no progress: a wait never ends")
            for slot in range(nslot):
                assert content[slot] is None or content[slot][0] == "landed"
            cnt += len(seq)


TILINGS = [((2, 3, 5), 17), ((1, 1, 4), 9), ((4, 2, 7), 30), ((1, 2, 1), 6), ((3, 1, 3), 3), ((2, 2, 33), 33)]


@pytest.mark.parametrize("nslot", [4, 6, 8])
@pytest.mark.parametrize("tl,nz", TILINGS)
def test_pipeline_protocol_under_random_interleavings(nslot, tl, nz):
    nitems = tl[0] * tl[1] * ((nz + tl[2] - 1) // tl[2])
    for size in (1, 3, nitems, nitems + 2):
        ranks = range(min(size, nitems + 1))
        for seed in range(3):
            run(tl, nz, nwarps=3, nslot=nslot, ranks=ranks, size=size, passes=3, seed=seed)


def test_model_catches_a_missing_release():
    with pytest.raises(AssertionError):
        run(((2, 1, 9), 9)[0], 9, nwarps=3, nslot=4, ranks=[0], size=1, passes=2, seed=0, skip_release=(1, 2))
