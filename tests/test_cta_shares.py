"""The TMA particle kernel's split of a species' slots over its CTAs, written out as the
kernel forms it: CTA k of K takes slots [r0, r1) with r0 = floor(n k / K) rounded down to
a multiple of 4 and r1 the next CTA's r0 (n for the last), walked in tiles of 1,984 slots
from r0, the last one partial.  Checked for many counts and grid sizes: the ranges cover
[0, n) once, every share is within 4 slots of n / K, and every tile meets the bulk copies'
rules (16-byte start and size for the particles; the cells copied in whole groups of 4
from a 16-byte boundary, the rest of the tile's cells read one by one)."""
import numpy as np
import pytest

TILE = 1984  # particles per tile: 992 consumer threads x 2


def shares(n, K):
    out = []
    for k in range(K):
        r0 = (n * k // K) & ~3
        r1 = n if k + 1 == K else (n * (k + 1) // K) & ~3
        out.append((r0, r1))
    return out


def tiles(r0, r1):
    i0 = r0
    while i0 < r1:
        cnt = min(TILE, r1 - i0)
        yield i0, cnt
        i0 += TILE


@pytest.mark.parametrize("K", [1, 2, 7, 151, 152, 304])
def test_shares_cover_every_slot_once_and_are_even(K):
    rng = np.random.default_rng(K)
    counts = [0, 1, 3, 4, 5, 603, 604, 605, K * 4 - 1, K * TILE, K * TILE + 1, 4_096_000,
              4_070_123] + [int(x) for x in rng.integers(0, 9_000_000, 40)]
    for n in counts:
        sh = shares(n, K)
        seen = 0
        prev = 0
        for r0, r1 in sh:
            assert r0 == prev and r1 >= r0
            prev = r1
            assert r0 % 4 == 0
            assert abs((r1 - r0) - n / K) <= 4 + 1e-9
            covered = 0
            for i0, cnt in tiles(r0, r1):
                assert 0 < cnt <= TILE and i0 + cnt <= r1
                assert (i0 * 16) % 16 == 0 and (cnt * 16) % 16 == 0  # particles: 16 B each
                cb = cnt & ~3  # cells by bulk copy
                assert (i0 * 4) % 16 == 0 and (cb * 4) % 16 == 0
                assert cnt - cb < 4
                covered += cnt
            assert covered == r1 - r0
            seen += r1 - r0
        assert prev == n and seen == n


def test_whole_tile_shares_left_some_ctas_a_tile_more():
    """The split it replaced: whole tiles per CTA.  For a species of the headline sheath
    (3.8M to 4.1M particles over 151 CTAs, 12.8 to 13.7 tiles a CTA) the fraction of CTAs
    with a tile more than the rest is the fractional part of tiles / CTAs, here 0.59 to
    0.81: the launch lasts as long as those CTAs, a tile (7 to 8%) longer than the others.
    The slot shares differ by at most 4."""
    K = 151
    for n in (3_838_000, 4_070_000, 4_096_000):
        nt = (n + TILE - 1) // TILE
        per_cta = np.array([nt * (k + 1) // K - nt * k // K for k in range(K)])
        assert per_cta.max() - per_cta.min() == 1
        frac = nt / K - nt // K
        assert np.mean(per_cta == per_cta.max()) == pytest.approx(frac, abs=1.0 / K)
        assert 0.5 < frac < 0.9
        sizes = [r1 - r0 for r0, r1 in shares(n, K)]
        assert max(sizes) - min(sizes) <= 4
