"""The default z chunk of 3D launches (jf_auto_zchunk, host logic in
libjf.so, no GPU): the one-wave rule for grids that fit one wave of 32-plane
CTAs, and for larger grids the chunk length whose greedy schedule of CTAs
(in launch order, over the resident CTA slots) finishes first.  The schedule
is written out here from its definition and searched by brute force."""
import heapq
import math
import os

import pytest

from paper_2203_13760_gb300 import jf

if not os.path.exists(jf.LIB_PATH):  # pragma: no cover
    pytest.skip("libjf.so not built", allow_module_level=True)

SMS = 152


def schedule_end(tiles, nz, z, slots, prologue=0.5):
    """Finish time of `tiles` CTAs per chunk, chunk after chunk, each taking
    the next free slot: a list schedule simulated CTA by CTA."""
    free = [0.0] * slots
    end = 0.0
    for z0 in range(0, nz, z):
        cost = min(z, nz - z0) + prologue
        for _ in range(tiles):
            t = heapq.heappop(free) + cost
            heapq.heappush(free, t)
            end = max(end, t)
    return end


def expected(n, tile=(32, 7), cps=2, sms=SMS):
    tiles = math.ceil(n[0] / tile[0]) * math.ceil(n[1] / tile[1])
    slots = sms * cps
    z = max(1, math.ceil(n[2] * tiles / slots))
    if z <= 32:
        return z
    ends = {c: schedule_end(tiles, n[2], c, slots) for c in range(20, 41)}
    best = min(ends.values())
    return max(c for c, e in ends.items() if e <= best + 1e-9)


@pytest.mark.parametrize("n", [(32, 32, 32), (64, 64, 64), (128, 128, 128), (100, 90, 70)])
def test_one_wave_rule(n):
    """Grids that fit one wave of 32-plane CTAs take ceil(nz tiles / slots)."""
    tiles = math.ceil(n[0] / 32) * math.ceil(n[1] / 7)
    assert jf.auto_zchunk(n) == max(1, math.ceil(n[2] * tiles / (2 * SMS)))
    assert jf.auto_zchunk(n) <= 32


@pytest.mark.parametrize("n", [(192, 192, 192), (256, 256, 256), (384, 384, 384), (256, 200, 300)])
def test_schedule_rule_matches_brute_force(n):
    assert jf.auto_zchunk(n) == expected(n)


def test_bench_grid_choice():
    """TGV 256^3 with the 32 x 7 tile at two CTAs per SM: 36 planes (eight
    chunks, the last one 4 planes), whose schedule beats 32 planes."""
    z = jf.auto_zchunk((256, 256, 256))
    assert z == 36
    tiles, slots = 8 * 37, 2 * SMS
    assert schedule_end(tiles, 256, z, slots) < schedule_end(tiles, 256, 32, slots)


def test_other_tiles_and_occupancy():
    # 32 x 6 tile at one CTA per SM (the FP64 default): tiles = 8 x 43 per plane;
    # 32 x 4 (8 x 64)
    assert jf.auto_zchunk((256, 256, 256), tile=(32, 6), ctas_per_sm=1) == expected((256, 256, 256), (32, 6), 1)
    assert jf.auto_zchunk((256, 256, 256), tile=(32, 4), ctas_per_sm=1) == expected((256, 256, 256), (32, 4), 1)
    # a tiny grid never goes below one plane
    assert jf.auto_zchunk((8, 8, 1)) == 1


def test_invalid_arguments():
    assert jf.auto_zchunk((0, 10, 10)) == 0
    assert jf.auto_zchunk((10, 10, 10), tile=(32, 0)) == 0
    assert jf.auto_zchunk((10, 10, 10), ctas_per_sm=0) == 0
    assert jf.auto_zchunk((10, 10, 10), sms=0) == 0
