"""The retransform GEMM's A ring (k_tc_retransform): RA = 8 k-block slots,
fill warp f filling k-blocks f, f + 8, ... of every tile into slot
(tile * KB + kb) % RA, and waiting on that slot's `afree` barrier with the
parity of the previous lap.  A parity wait can only be trusted if the
waiting warp's consecutive uses of a slot are exactly one lap apart and no
other warp fills the slot in between; this checks that ownership rule for
every K-block count the kernel meets (BF16: 64-element k-blocks, split:
32-element, Nt = 32 .. 256), with the kernel's own index formulas."""
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
