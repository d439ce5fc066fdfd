"""Pins of the oracle's octree tables (Sec. 2.1.1: boxes of 8^3 cells, 2^3
children at half the spacing, proper nesting) against brute force."""
import itertools

import numpy as np
import pytest

import oracle
import synth

DIRS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
        if (dx, dy, dz) != (0, 0, 0)]


def brute_force_check(t, nb_levels_uniform):
    """Every table entry recomputed from box coordinates with Python dicts."""
    n = len(t["level"])
    where = {(int(t["level"][b]), *map(int, t["ijk"][b])): b for b in range(n)}
    assert len(where) == n, "duplicate boxes"
    off = t["level_offset"]
    for l in range(len(off) - 1):
        keys = t["morton"][off[l]:off[l + 1]]
        assert np.all(np.diff(keys.astype(np.float64)) > 0), "level %d not Morton sorted" % l
        assert np.all(t["level"][off[l]:off[l + 1]] == l)
    for b in range(n):
        l = int(t["level"][b])
        i, j, k = map(int, t["ijk"][b])
        assert int(t["morton"][b]) == synth.morton3(i, j, k)
        side = 1 << l
        for d, (dx, dy, dz) in enumerate(DIRS):
            q = (i + dx, j + dy, k + dz)
            if min(q) < 0 or max(q) >= side:
                want = -1
            else:
                want = where.get((l, *q), -2)
            assert t["nbr"][b, d] == want, (b, d)
        # parent / children
        if l == 0:
            assert t["parent"][b] == -1
        else:
            p = t["parent"][b]
            assert where[(l - 1, i // 2, j // 2, k // 2)] == p
            c = (i & 1) + 2 * (j & 1) + 4 * (k & 1)
            assert t["child"][p, c] == b
        ch = t["child"][b]
        assert np.all(ch >= 0) or np.all(ch < 0), "children come in eights"
        if ch[0] >= 0:
            for c in range(8):
                ci = (2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2))
                assert where[(l + 1, *ci)] == ch[c]
    # proper nesting: every neighbour position of a box at level l >= 1 is
    # inside a box of level l or l-1 (or outside the domain)
    for b in range(n):
        l = int(t["level"][b])
        if l == 0:
            continue
        i, j, k = map(int, t["ijk"][b])
        side = 1 << l
        for dx, dy, dz in DIRS:
            q = (i + dx, j + dy, k + dz)
            if min(q) < 0 or max(q) >= side:
                continue
            assert (l, *q) in where or (l - 1, q[0] // 2, q[1] // 2, q[2] // 2) in where


def test_uniform_levels_bruteforce():
    dom = synth.domain_uniform_cube(64)
    o = oracle.Oracle(dom)
    t = o.tables()
    assert list(t["level_offset"]) == [0, 1, 9, 73, 585]
    brute_force_check(t, 4)


def test_streamer_small_bruteforce():
    dom, st = synth.workload("streamer_small")
    o = oracle.build_mesh(dom, st)
    t = o.tables()
    assert o.n_levels == dom.lbase + dom.max_level + 1
    assert o.n_boxes > 100
    brute_force_check(t, dom.lbase + 1)


def test_neighbour_involution():
    dom, st = synth.workload("streamer_small")
    t = oracle.build_mesh(dom, st).tables()
    for b in range(len(t["level"])):
        for d, (dx, dy, dz) in enumerate(DIRS):
            nb = t["nbr"][b, d]
            if nb >= 0:
                back = DIRS.index((-dx, -dy, -dz))
                assert t["nbr"][nb, back] == b


def test_nesting_drop_rule():
    """A request whose 26-neighbourhood is not all present is dropped."""
    dom = synth.Domain(length=1.0, nb=2, max_level=3)
    o = oracle.Oracle(dom)
    flags = np.zeros(8, np.int8)
    flags[0] = 1                                   # refine box (0,0,0) of level 1
    assert o.refine_level(1, flags) == 8 and o.dropped == 0
    lo, hi = o.level_range(2)
    ijk2 = o.level_ijk(2)
    flags2 = np.zeros(hi - lo, np.int8)
    # box (1,1,1) of level 2 touches level-2 positions owned by unrefined
    # level-1 boxes -> must be dropped; box (0,0,0) touches only its
    # siblings and the outside -> allowed
    want_refined = []
    for b, q in enumerate(map(tuple, ijk2)):
        if q in ((1, 1, 1), (0, 0, 0)):
            flags2[b] = 1
    o.refine_level(2, flags2)
    assert o.dropped == 1
    t = o.tables()
    lv2 = {tuple(t["ijk"][b]): b for b in range(lo, hi)}
    assert t["child"][lv2[(0, 0, 0)], 0] >= 0
    assert t["child"][lv2[(1, 1, 1)], 0] < 0
