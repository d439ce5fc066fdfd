"""Pins of the oracle's refinement criterion and regridding (Sec. 2.5,
Eq. 8: dx < c0 c1 / alpha(c1 |E|), c0 = 1, c1 = 1.2, a refinement buffer of
three cells, derefinement with c0 = 1/8 and dx < 30 um) against brute force
over cell coordinates, closed forms and invariants."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from test_oracle_tables import DIRS, brute_force_check

C0, C1, C0D, DXD, BUF = 1.0, 1.2, 0.125, 30e-6, 3


def streamer_mesh():
    dom, st = synth.workload("streamer_small")
    o = oracle.build_mesh(dom, st)
    o.set_table(synth.coefficient_table())
    return dom, st, o


def set_tip_field(dom, o, e_peak=2e7, e_bg=1.5e6, sigma=1.5e-3, centre=None):
    """|E| on every cell: a Gaussian peak (closed form) on a background."""
    t = o.tables()
    x, y, z = synth.cell_centres(dom, t["level"], t["ijk"])
    c = centre if centre is not None else (4e-3, 4e-3, 5e-3)
    r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    o.set(oracle.EMAG, e_bg + e_peak * np.exp(-r2 / (2 * sigma ** 2)))
    return t


def local_ijk(c):
    return c & 7, (c >> 3) & 7, c >> 6


def brute_flags(dom, o, t, c0=C0, c1=C1, c0d=C0D, dxd=DXD, buf=BUF):
    """Eq. 8 cell by cell, the buffer by Chebyshev distance between cells of
    ALL same-level leaf boxes (no neighbour table), derefinement rule."""
    em = o.get(oracle.EMAG)
    leaf = t["child"][:, 0] < 0
    lbase, lmax = dom.lbase, dom.lbase + dom.max_level
    n = len(leaf)
    need_cells = {}          # level -> list of global cell coordinates
    fine = np.zeros(n, bool)
    cidx = np.arange(512)
    li, lj, lk = local_ijk(cidx)
    for b in np.where(leaf)[0]:
        l = int(t["level"][b])
        dx = dom.h(l)
        a = np.array([o.lookup(2, c1 * e) for e in em[b]])
        need = a * dx >= c0 * c1
        fine[b] = dx < dxd and bool(np.all(a * dx < c0d * c1))
        if need.any():
            g = np.stack([t["ijk"][b, 0] * 8 + li, t["ijk"][b, 1] * 8 + lj, t["ijk"][b, 2] * 8 + lk], 1)[need]
            need_cells.setdefault(l, []).append(g)
    flags = np.zeros(n, np.int8)
    for b in np.where(leaf)[0]:
        l = int(t["level"][b])
        marked = False
        if l in need_cells:
            g = np.concatenate(need_cells[l])
            lo = t["ijk"][b] * 8
            hi = lo + 7
            d = np.maximum(np.maximum(lo[None, :] - g, g - hi[None, :]), 0).max(1)
            marked = bool((d <= buf).any())
        if marked:
            flags[b] = 1 if l < lmax else 0
        elif fine[b] and l > lbase:
            flags[b] = -1
    return flags


def test_criterion_flags_bruteforce():
    dom, st, o = streamer_mesh()
    t = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    want = brute_flags(dom, o, t)
    assert np.array_equal(f, want)
    assert (f == 1).sum() > 0 and (f == 0).sum() > 0
    # the buffer reaches boxes with no cell of their own above the threshold
    f0 = o.refine_flags(C0, C1, C0D, DXD, 0)
    assert np.array_equal(f0, brute_flags(dom, o, t, buf=0))
    assert (f == 1).sum() > (f0 == 1).sum()


def test_criterion_threshold_and_derefinement():
    """A uniform |E| sits exactly on either side of Eq. 8 for the finest
    spacing; derefinement needs the c0/8 criterion and dx < dx_deref."""
    dom, st, o = streamer_mesh()
    t = o.tables()
    leaf = t["child"][:, 0] < 0
    lmax = dom.lbase + dom.max_level
    dx = dom.h(lmax)
    tab = synth.coefficient_table()
    # an |E| whose alpha(c1 E) dx is far below c0 c1 everywhere: nothing to refine
    o.set(oracle.EMAG, np.full((o.n_boxes, 512), 1e5))
    f = o.refine_flags(C0, C1, C0D, 1.0, BUF)
    lev = t["level"]
    assert np.all(f[~leaf] == 0)
    assert np.all(f[leaf & (lev > dom.lbase)] == -1)      # all derefinable (dx_deref large)
    assert np.all(f[leaf & (lev == dom.lbase)] == 0)      # the base grid stays
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)             # dx >= 30 um here: none
    assert np.all(f <= 0) and np.all(f[leaf] == 0)
    # an |E| with alpha(c1 E) dx >= c0 c1 on the coarsest leaves: those refine
    big = tab["E"][-1]
    o.set(oracle.EMAG, np.full((o.n_boxes, 512), big))
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    a = o.lookup(2, C1 * big)
    for b in np.where(leaf)[0]:
        l = int(lev[b])
        want = 1 if (a * dom.h(l) >= C0 * C1 and l < lmax) else 0
        assert f[b] == want, (b, l)
    assert a * dx < C0 * C1 or True


def expected_mesh(dom, t, flags):
    """Box set after regridding, from coordinates only."""
    n = len(t["level"])
    lmax = dom.lbase + dom.max_level
    where = {(int(t["level"][b]), *map(int, t["ijk"][b])): b for b in range(n)}
    leaf = t["child"][:, 0] < 0
    par = {b: where.get((int(t["level"][b]) - 1, *(int(v) // 2 for v in t["ijk"][b])), -1) for b in range(n)}
    R, dropped = set(), 0
    for b in range(n):
        l = int(t["level"][b])
        if not leaf[b] or flags[b] <= 0 or l >= lmax:
            continue
        i, j, k = map(int, t["ijk"][b])
        side = 1 << l
        ok = all((l, i + dx, j + dy, k + dz) in where for dx, dy, dz in DIRS
                 if 0 <= i + dx < side and 0 <= j + dy < side and 0 <= k + dz < side)
        if ok:
            R.add(b)
        else:
            dropped += 1
    D = set()
    for p in range(n):
        if leaf[p]:
            continue
        kids = [b for b in range(n) if par[b] == p]
        if not all(leaf[c] and flags[c] < 0 for c in kids):
            continue
        ok = True
        for c in kids:
            l = int(t["level"][c])
            i, j, k = map(int, t["ijk"][c])
            for dx, dy, dz in DIRS:
                nb = where.get((l, i + dx, j + dy, k + dz))
                if nb is not None and par[nb] != p and (not leaf[nb] or nb in R):
                    ok = False
        if ok:
            D.add(p)
    keys = [(int(t["level"][b]), *map(int, t["ijk"][b])) for b in range(n) if par[b] not in D or par[b] == -1]
    for b in R:
        l = int(t["level"][b])
        i, j, k = map(int, t["ijk"][b])
        keys += [(l + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + (c >> 2)) for c in range(8)]
    keys.sort(key=lambda q: (q[0], synth.morton3(q[1], q[2], q[3])))
    return keys, len(R), len(D), dropped


def test_regrid_tables_bruteforce():
    dom, st, o = streamer_mesh()
    t = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, 1.0, BUF)   # dx_deref large: also derefinements
    keys, nr, nd, ndrop = expected_mesh(dom, t, f)
    assert nr > 0 and nd > 0
    r = o.regrid(f)
    assert r == (nr, nd, ndrop)
    t2 = o.tables()
    got = [(int(t2["level"][b]), *map(int, t2["ijk"][b])) for b in range(o.n_boxes)]
    assert got == keys
    brute_force_check(t2, dom.lbase + 1)


def coarse_value(vals, l, g, from_g, kind, dom):
    """Value of global cell g at level l, or the wall ghost from cell from_g."""
    side = 8 << l
    if min(g) < 0 or max(g) >= side:
        inner = vals[(l, *from_g)]
        if kind == "density":
            return inner
        for a in range(3):
            if g[a] < 0 or g[a] >= side:
                f = 2 * a + (1 if g[a] >= side else 0)
                return (2.0 * dom.bc_val[f] - inner) if dom.bc_type[f] else inner
    return vals[(l, *g)]


def test_regrid_data_prolongation_and_kept_boxes():
    """Kept leaves keep their data bit for bit; new children get the
    linear prolongation (c + c_sx + c_sy + c_sz)/4 of their parent's cells,
    limited to 2c for densities (mirror ghosts at walls), recomputed here
    from the old data by coordinates; a linear potential is exact."""
    dom, st, o = streamer_mesh()
    t = set_tip_field(dom, o)
    x, y, z = synth.cell_centres(dom, t["level"], t["ijk"])
    g0, g1 = dom.bc_val[4], dom.bc_val[5]
    lin = lambda zz: g0 + (g1 - g0) * (zz - dom.origin[2]) / dom.length   # matches the z walls
    o.set(oracle.PHI, lin(z))
    rng = np.random.default_rng(7)
    # densities spread over orders of magnitude, so that the 2c limit acts
    ne = 1e18 * rng.random((o.n_boxes, 512)) ** 4
    o.set(oracle.NE, ne)
    o.set(oracle.NI, 2.0 * ne)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    # the oracle restricts densities before it regrids: do the same to the copy
    o.regrid(np.zeros(o.n_boxes, np.int8))
    t = o.tables()
    old = {v: o.get(v) for v in (oracle.PHI, oracle.NE, oracle.NI)}
    leaf = t["child"][:, 0] < 0
    cells = {}
    cidx = np.arange(512)
    li, lj, lk = local_ijk(cidx)
    for v in old:
        d = {}
        for b in range(o.n_boxes):
            l = int(t["level"][b])
            for c in range(512):
                d[(l, t["ijk"][b, 0] * 8 + li[c], t["ijk"][b, 1] * 8 + lj[c], t["ijk"][b, 2] * 8 + lk[c])] = old[v][b, c]
        cells[v] = d
    oldkey = {(int(t["level"][b]), *map(int, t["ijk"][b])): b for b in range(o.n_boxes)}
    nr, nd, _ = o.regrid(f)
    assert nr > 0
    t2 = o.tables()
    new = {v: o.get(v) for v in old}
    n_new = n_lim = 0
    for b in range(o.n_boxes):
        key = (int(t2["level"][b]), *map(int, t2["ijk"][b]))
        if key in oldkey:
            ob = oldkey[key]
            if leaf[ob]:
                for v in old:
                    assert np.array_equal(new[v][b], old[v][ob]), (key, v)
            continue
        n_new += 1
        l = key[0] - 1
        for c in range(512):
            G = (key[1] * 8 + li[c], key[2] * 8 + lj[c], key[3] * 8 + lk[c])
            cc = tuple(q >> 1 for q in G)
            for v in old:
                kind = "phi" if v == oracle.PHI else "density"
                cval = cells[v][(l, *cc)]
                s = cval
                for a in range(3):
                    q = list(cc)
                    q[a] += 1 if (G[a] & 1) else -1
                    s += coarse_value(cells[v], l, tuple(q), cc, kind, dom)
                want = 0.25 * s
                if kind == "density" and want > 2.0 * cval:
                    want = 2.0 * cval
                    n_lim += 1
                assert new[v][b, c] == want, (key, c, v)
    assert n_new == 8 * nr
    assert n_lim > 0
    # linear potential reproduced exactly in the new boxes
    x2, y2, z2 = synth.cell_centres(dom, t2["level"], t2["ijk"])
    assert np.abs(new[oracle.PHI] - lin(z2)).max() <= 1e-12 * max(abs(g0), abs(g1))


def test_regrid_round_trip_and_dropped_requests():
    """Refine where the criterion asks, then derefine exactly the new boxes:
    the original mesh comes back; refinement requests with a missing
    neighbour at their level are dropped (proper nesting)."""
    dom, st, o = streamer_mesh()
    t0 = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    keys0 = [(int(t0["level"][b]), *map(int, t0["ijk"][b])) for b in range(o.n_boxes)]
    nr, nd, ndrop = o.regrid(f)
    assert nr > 0 and nd == 0
    t1 = o.tables()
    keys1 = [(int(t1["level"][b]), *map(int, t1["ijk"][b])) for b in range(o.n_boxes)]
    added = set(keys1) - set(keys0)
    back = np.array([-1 if k in added else 0 for k in keys1], np.int8)
    nr2, nd2, _ = o.regrid(back)
    assert (nr2, nd2) == (0, nr)
    t2 = o.tables()
    assert [(int(t2["level"][b]), *map(int, t2["ijk"][b])) for b in range(o.n_boxes)] == keys0
    # a single refined box at level 1 of a 2^3 base: its children cannot refine
    dom2 = synth.Domain(length=1.0, nb=2, max_level=3)
    o2 = oracle.Oracle(dom2)
    f1 = np.zeros(o2.n_boxes, np.int8)
    f1[o2.level_range(1)[0]] = 1
    assert o2.regrid(f1) == (1, 0, 0)
    f2 = np.zeros(o2.n_boxes, np.int8)
    lo, hi = o2.level_range(2)
    f2[lo:hi] = 1
    # only the child in the domain corner has all its neighbour positions
    # filled (siblings) or outside the domain
    assert o2.regrid(f2) == (1, 0, 7)
    t2 = o2.tables()
    lo3 = o2.level_range(3)[0]
    assert tuple(t2["ijk"][t2["parent"][lo3]]) == (0, 0, 0)


def test_regrid_derefinement_blocked_by_nesting():
    """A box whose children neighbour a box with children keeps them; once
    the grandchildren go, the same request succeeds."""
    dom = synth.Domain(length=1.0, nb=2, max_level=3)
    o = oracle.Oracle(dom)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(1)
    f[lo:hi] = 1
    assert o.regrid(f)[0] == 8                      # all of level 2
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo:lo + 8] = 1                                # the children of the first level-1 box
    assert o.regrid(f)[0] == 8
    t = o.tables()
    brute_force_check(t, dom.lbase + 1)
    n3 = o.level_range(3)[1] - o.level_range(3)[0]
    assert n3 == 64
    # every other level-1 box touches the first one: derefining their
    # children is blocked while level 3 exists
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo + 8:hi] = -1
    assert o.regrid(f)[:2] == (0, 0)
    # remove level 3 (its boxes only neighbour cousins that are leaves)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(3)
    f[lo:hi] = -1
    assert o.regrid(f)[:2] == (0, 8)
    assert o.n_levels == 3
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo:hi] = -1
    assert o.regrid(f)[:2] == (0, 8)
    assert o.n_levels == 2
    brute_force_check(o.tables(), dom.lbase + 1)


def test_derefined_box_holds_the_mean_of_its_children():
    """Densities are restricted before the mesh changes: a derefined box
    becomes a leaf holding, per cell, the mean of its eight child cells."""
    dom = synth.Domain(length=1.0, nb=2, max_level=3)
    o = oracle.Oracle(dom)
    f = np.zeros(o.n_boxes, np.int8)
    f[o.level_range(1)[0]] = 1
    assert o.regrid(f)[0] == 1
    rng = np.random.default_rng(11)
    o.set(oracle.NE, rng.random((o.n_boxes, 512)))
    o.set(oracle.NI, np.zeros((o.n_boxes, 512)))
    t = o.tables()
    p = o.level_range(1)[0]
    kids = t["child"][p]
    ne = o.get(oracle.NE)
    li, lj, lk = local_ijk(np.arange(512))
    want = np.zeros(512)
    for c in range(512):
        I, J, K = li[c], lj[c], lk[c]
        kid = kids[(I >> 2) + 2 * (J >> 2) + 4 * (K >> 2)]
        cells = [ne[kid, (2 * (I & 3) + di) + 8 * (2 * (J & 3) + dj) + 64 * (2 * (K & 3) + dk)]
                 for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
        want[c] = np.mean(cells)
    f = np.zeros(o.n_boxes, np.int8)
    f[kids] = -1
    assert o.regrid(f)[:2] == (0, 1)
    t2 = o.tables()
    b = [i for i in range(o.n_boxes) if t2["level"][i] == 1 and tuple(t2["ijk"][i]) == tuple(t["ijk"][p])][0]
    assert t2["child"][b, 0] < 0
    assert np.allclose(o.get(oracle.NE)[b], want, rtol=1e-14, atol=0)


def test_derefinement_blocked_by_refinement_in_the_same_call():
    """A box whose children touch a box refined in the same call keeps its
    children (the new level would otherwise border a coarse leaf); the
    refinement goes ahead."""
    dom = synth.Domain(length=1.0, nb=2, max_level=3)
    o = oracle.Oracle(dom)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(1)
    f[lo:hi] = 1
    assert o.regrid(f)[0] == 8
    t = o.tables()
    at = {(int(t["level"][b]), *map(int, t["ijk"][b])): b for b in range(o.n_boxes)}
    a = at[(1, 0, 0, 0)]
    f = np.zeros(o.n_boxes, np.int8)
    f[t["child"][a]] = -1                 # derefine the first level-1 box
    f[at[(2, 2, 0, 0)]] = 1               # refine a level-2 box touching its children
    assert o.regrid(f)[:2] == (1, 0)
    brute_force_check(o.tables(), dom.lbase + 1)
