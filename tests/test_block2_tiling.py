"""CPU check of the tile enumeration of the temporally blocked first iteration (BPS_VARIANT_BLOCK2,
sweep_u8_block2_kernel in csrc/bp.cu): the same index arithmetic, restated here, must give every
pixel of each colour to exactly one tile, and every even pixel that sends to a tile's odd pixels
must be computed by that tile (its own even pixels or the ring around it).  The GPU parity tests
check the kernel's results against the oracle; this checks the enumeration at shapes and edges the
GPU cases do not all reach (tiles cut by the image border, one-pixel images)."""
import pytest

TW, TH = 32, 16          # BLK_TW, BLK_TH
HALF = TW // 2
OWN = TH * HALF
RING = 2 * HALF + TH


def own(c, x0, y0, tw, th):
    for k in range(OWN):
        row, i = divmod(k, HALF)
        y = y0 + row
        x = x0 + ((c + y) & 1) + 2 * i
        if row < th and x < x0 + tw:
            yield x, y


def ring(x0, y0, tw, th, W, H):
    for r in range(RING):
        if r < 2 * HALF:
            y = y0 - 1 if r < HALF else y0 + th
            x = x0 + (y & 1) + 2 * (r % HALF)
            if x >= x0 + tw:
                continue
        elif r < 2 * HALF + TH // 2:
            x, y = x0 - 1, y0 + 1 + 2 * (r - 2 * HALF)
        else:
            x = x0 + tw
            y = y0 + (x & 1) + 2 * (r - 2 * HALF - TH // 2)
        if 0 <= x < W and 0 <= y < H and (r < 2 * HALF or y < y0 + th):
            yield x, y


@pytest.mark.parametrize("W,H", [(150, 110), (96, 72), (33, 17), (64, 16), (1, 1), (1, 40), (45, 1), (31, 15), (65, 33)])
def test_block2_tiles_cover_every_pixel_once_and_every_sender(W, H):
    owners = {}
    for ty in range((H + TH - 1) // TH):
        for tx in range((W + TW - 1) // TW):
            x0, y0 = tx * TW, ty * TH
            tw, th = min(TW, W - x0), min(TH, H - y0)
            evens = set(own(0, x0, y0, tw, th))
            odds = set(own(1, x0, y0, tw, th))
            rng = set(ring(x0, y0, tw, th, W, H))
            assert all((x + y) % 2 == 0 for x, y in evens | rng)
            assert all((x + y) % 2 == 1 for x, y in odds)
            assert not (evens & rng)
            for p in evens | odds:
                assert x0 <= p[0] < x0 + tw and y0 <= p[1] < y0 + th
                owners[p] = owners.get(p, 0) + 1
            computed = evens | rng
            for x, y in odds:  # every existing neighbour of an odd pixel is even and computed here
                for q in ((x, y - 1), (x, y + 1), (x - 1, y), (x + 1, y)):
                    if 0 <= q[0] < W and 0 <= q[1] < H:
                        assert q in computed, (W, H, (x, y), q)
            # the ring holds only pixels that send to one of the tile's odd pixels
            for x, y in rng:
                assert any(q in odds for q in ((x, y - 1), (x, y + 1), (x - 1, y), (x + 1, y)))
    assert len(owners) == W * H and set(owners.values()) == {1}
