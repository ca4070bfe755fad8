"""The retransform GEMM's A ring (k_tc_retransform): RA = 8 k-block slots,
fill warp f filling k-blocks f, f + 8, ... of every tile into slot
(tile * KB + kb) % RA, and waiting on that slot's `afree` barrier with the
parity of the previous lap.  A parity wait can only be trusted if the
waiting warp's consecutive uses of a slot are exactly one lap apart and no
other warp fills the slot in between; this checks that ownership rule for
every K-block count the kernel meets (BF16: 64-element k-blocks, split:
32-element, Nt = 32 .. 256), with the kernel's own index formulas.  Then the
tensor-memory accumulator hand-off between the MMA role and the epilogue
warps (one slot, or two alternating slots), on a model of the mbarrier's
parity waits under random interleavings."""
import pytest

RA = 8           # A slots = fill warps
FILL_WARPS = 8


@pytest.mark.parametrize("KB", [1, 2, 4, 8, 16])
def test_each_slot_has_one_owner_one_lap_apart(KB):
    uses = {}  # slot -> list of (n, warp)
    for tile in range(64):
        for f in range(FILL_WARPS):
            for kb in range(f, KB, FILL_WARPS):
                n = tile * KB + kb
                uses.setdefault(n % RA, []).append((n, f))
    assert sorted(uses) == list(range(min(RA, 64 * KB)))
    for slot, seq in uses.items():
        seq.sort()
        owners = {w for _, w in seq}
        assert len(owners) == 1, (KB, slot, owners)
        ns = [n for n, _ in seq]
        assert all(b - a == RA for a, b in zip(ns, ns[1:])), (KB, slot, ns[:6])


def test_every_k_block_of_every_tile_is_filled_once():
    for KB in (1, 2, 4, 8, 16):
        filled = [(tile, kb) for tile in range(4) for f in range(FILL_WARPS)
                  for kb in range(f, KB, FILL_WARPS)]
        assert sorted(filled) == [(t, k) for t in range(4) for k in range(KB)]


class Barrier:
    """An mbarrier as the kernels use it: a phase completes when its arrival
    count is reached, and a parity wait for P passes once the phase with
    parity P has completed, i.e. while the current phase number has the
    other parity (so a waiter two phases behind or ahead is not told apart)."""

    def __init__(self, count):
        self.count, self.arrived, self.phase = count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived, self.phase = 0, self.phase + 1

    def ready(self, parity):
        return (self.phase & 1) != parity


@pytest.mark.parametrize("AS", [1, 2])
@pytest.mark.parametrize("seed", range(20))
def test_alternating_accumulators_are_never_overwritten_or_read_early(AS, seed):
    """The accumulator hand-off of the tensor-memory GEMMs with AS slots
    (AS = 2: the column-split FP8 stage-1 GEMM and the retransform GEMM,
    AS = 1: the other GEMMs): the MMA role fills use u into slot u % AS
    after waiting on that slot's acc_empty with parity ((u / AS) - 1) & 1
    (from u >= AS on) and commits acc_full; the epilogue waits on acc_full
    with parity (u / AS) & 1, reads, and arrives on acc_empty.  Under random
    interleavings (several epilogue warps arriving one by one), no use is
    started over a slot whose last use has not been drained, no epilogue
    warp reads a use before it is complete, and the MMA role's final waits
    on the last AS uses end only once every warp has drained them."""
    import random
    rnd = random.Random(seed)
    U, WARPS = 23, 3
    full = [Barrier(1) for _ in range(AS)]
    empty = [Barrier(WARPS) for _ in range(AS)]
    slot_use = [None] * AS              # use held by each slot (None: free)
    drained = [set() for _ in range(U)]  # epilogue warps done with use u
    mma = {"u": 0, "writing": None, "final": 0}
    epi = [0] * WARPS                   # next use of each epilogue warp
    steps = 0
    while True:
        steps += 1
        assert steps < 100000, "no progress"
        actors = []
        if mma["u"] < U or mma["writing"] is not None or mma["final"] < min(AS, U):
            actors.append("mma")
        actors += [w for w in range(WARPS) if epi[w] < U]
        if not actors:
            break
        a = rnd.choice(actors)
        if a == "mma":
            if mma["writing"] is not None:          # commit the use being filled
                u = mma["writing"]
                full[u % AS].arrive()
                mma["writing"] = None
                mma["u"] += 1
            elif mma["u"] < U:
                u = mma["u"]
                s = u % AS
                if u >= AS and not empty[s].ready(((u // AS) - 1) & 1):
                    continue
                prev = slot_use[s]
                assert prev is None or len(drained[prev]) == WARPS, (u, prev)
                slot_use[s] = u
                mma["writing"] = u
            else:                                   # the final waits on the last AS uses
                k = U - min(AS, U) + mma["final"]
                if empty[k % AS].ready((k // AS) & 1):
                    assert len(drained[k]) == WARPS, k
                    mma["final"] += 1
        else:
            w = a
            u = epi[w]
            s = u % AS
            if not full[s].ready((u // AS) & 1):
                continue
            assert slot_use[s] == u and mma["writing"] != u, (w, u, slot_use[s])
            drained[u].add(w)
            empty[s].arrive()
            epi[w] += 1
    assert all(len(d) == WARPS for d in drained)


@pytest.mark.parametrize("S", [2, 4])
@pytest.mark.parametrize("seed", range(20))
def test_converter_stage_ring(S, seed):
    """The K-block ring of the GEMMs whose stages are completed in shared
    memory (FP8 A widened to FP16; B's second half built from its first):
    the producer waits on empty[s] with parity ((n / S) - 1) & 1 from n >= S
    on and issues the TMA (which completes full[s]); each of 4 converter
    warps waits on full[s] with parity (n / S) & 1, writes its part and
    arrives on aready[s]; the MMA role waits on aready[s] with parity
    (n / S) & 1, reads, and commits empty[s].  Under random interleavings no
    TMA lands in a stage still being converted or read, no converter works
    on a stage before its TMA or while the MMAs read it, and the MMAs read
    only fully converted stages."""
    import random
    rnd = random.Random(1000 + seed)
    NK, CONV = 29, 4
    full = [Barrier(1) for _ in range(S)]
    aready = [Barrier(CONV) for _ in range(S)]
    empty = [Barrier(1) for _ in range(S)]
    state = [None] * S                 # (use n, 'loaded' | 'converting' | 'converted' | 'read')
    converted = [set() for _ in range(NK)]
    prod, mma = 0, 0
    conv = [0] * CONV
    steps = 0
    while prod < NK or mma < NK or min(conv) < NK:
        steps += 1
        assert steps < 200000, "no progress"
        a = rnd.choice(["prod", "mma"] + list(range(CONV)))
        if a == "prod" and prod < NK:
            s = prod % S
            if prod >= S and not empty[s].ready(((prod // S) - 1) & 1):
                continue
            assert state[s] is None or state[s][1] == "read", (prod, state[s])
            state[s] = (prod, "loaded")
            full[s].arrive()
            prod += 1
        elif a == "mma" and mma < NK:
            s = mma % S
            if not aready[s].ready((mma // S) & 1):
                continue
            assert state[s] == (mma, "converted") and len(converted[mma]) == CONV, (mma, state[s])
            state[s] = (mma, "read")
            empty[s].arrive()
            mma += 1
        elif isinstance(a, int) and conv[a] < NK:
            n = conv[a]
            s = n % S
            if not full[s].ready((n // S) & 1):
                continue
            assert state[s] is not None and state[s][0] == n and state[s][1] in ("loaded", "converting"), (a, n, state[s])
            converted[n].add(a)
            state[s] = (n, "converted" if len(converted[n]) == CONV else "converting")
            aready[s].arrive()
            conv[a] += 1
