"""Pins of the 2-D / axisymmetric oracle's refinement criterion and
regridding (Sec. 2.5, Eq. 8: dx < c0 c1 / alpha(c1 |E|), c0 = 1, c1 = 1.2,
a three-cell buffer, derefinement with c0 = 1/8 and dx < 30 um, the 3-D
rules on the quadtree) against brute force over cell coordinates."""
import numpy as np
import pytest

import synth
from oracle import quad

C0, C1, C0D, DXD, BUF = 1.0, 1.2, 0.125, 30e-6, 3
DIRS2 = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy]


def mesh(name="axi_small"):
    dom, st = synth.workload2(name)
    o = quad.build_mesh(dom, st)
    o.set_table(synth.coefficient_table())
    return dom, st, o


def set_tip_field(dom, o, e_peak=2e7, e_bg=1.5e6, sigma=1.5e-3, centre=(4e-3, 5e-3)):
    """|E| on every cell: a Gaussian peak (closed form) on a background; the
    peak at (4, 5) mm asks for refinements (some dropped by nesting) and
    leaves derefinable boxes elsewhere on both small meshes."""
    t = o.tables()
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2
    o.set(quad.EMAG, e_bg + e_peak * np.exp(-r2 / (2 * sigma ** 2)))
    return t


def check_tables(t, lbase):
    """Every entry of the quadtree tables recomputed from coordinates."""
    n = len(t["level"])
    pos = {(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])): b for b in range(n)}
    keys = [(int(t["level"][b]), synth_morton2(int(t["ij"][b, 0]), int(t["ij"][b, 1]))) for b in range(n)]
    assert keys == sorted(keys)
    for b in range(n):
        l, i, j = int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])
        assert t["parent"][b] == (pos[(l - 1, i >> 1, j >> 1)] if l else -1)
        kids = [pos.get((l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))) for c in range(4)]
        assert (all(k is None for k in kids) and list(t["child"][b]) == [-1] * 4) or \
            list(t["child"][b]) == kids
        for d, (dx, dy) in enumerate(DIRS2):
            ii, jj = i + dx, j + dy
            want = -1 if not (0 <= ii < (1 << l) and 0 <= jj < (1 << l)) else pos.get((l, ii, jj), -2)
            assert t["nbr"][b, d] == want
        if l > lbase:   # proper nesting: every neighbour position of the parent is covered
            p = t["parent"][b]
            assert all(t["nbr"][p, d] != -2 for d in range(8))


def synth_morton2(i, j):
    k = 0
    for b in range(31):
        k |= ((i >> b) & 1) << (2 * b) | ((j >> b) & 1) << (2 * b + 1)
    return k


def brute_flags(dom, o, t, c0=C0, c1=C1, c0d=C0D, dxd=DXD, buf=BUF):
    em = o.get(quad.EMAG)
    leaf = t["child"][:, 0] < 0
    lbase, lmax = dom.lbase, dom.lbase + dom.max_level
    n = len(leaf)
    need_cells, fine = {}, np.zeros(n, bool)
    li, lj = np.arange(64) & 7, np.arange(64) >> 3
    for b in np.where(leaf)[0]:
        l = int(t["level"][b])
        dx = dom.h(l)
        a = np.array([o.lookup(2, c1 * e) for e in em[b]])
        need = a * dx >= c0 * c1
        fine[b] = dx < dxd and bool(np.all(a * dx < c0d * c1))
        if need.any():
            g = np.stack([t["ij"][b, 0] * 8 + li, t["ij"][b, 1] * 8 + lj], 1)[need]
            need_cells.setdefault(l, []).append(g)
    flags = np.zeros(n, np.int8)
    for b in np.where(leaf)[0]:
        l = int(t["level"][b])
        marked = False
        if l in need_cells:
            g = np.concatenate(need_cells[l])
            lo = t["ij"][b] * 8
            d = np.maximum(np.maximum(lo[None, :] - g, g - (lo + 7)[None, :]), 0).max(1)
            marked = bool((d <= buf).any())
        if marked:
            flags[b] = 1 if l < lmax else 0
        elif fine[b] and l > lbase:
            flags[b] = -1
    return flags


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_criterion_flags_bruteforce(name):
    dom, st, o = mesh(name)
    t = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    assert np.array_equal(f, brute_flags(dom, o, t))
    assert (f == 1).sum() > 0 and (f == 0).sum() > 0
    f0 = o.refine_flags(C0, C1, C0D, DXD, 0)
    assert np.array_equal(f0, brute_flags(dom, o, t, buf=0))
    assert (f == 1).sum() > (f0 == 1).sum()
    fd = o.refine_flags(C0, C1, C0D, 1.0, BUF)        # dx_deref large: derefinements too
    assert np.array_equal(fd, brute_flags(dom, o, t, dxd=1.0))
    assert (fd == -1).sum() > 0


def expected_mesh(dom, t, flags):
    n = len(t["level"])
    lmax = dom.lbase + dom.max_level
    where = {(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])): b for b in range(n)}
    leaf = t["child"][:, 0] < 0
    par = {b: where.get((int(t["level"][b]) - 1, int(t["ij"][b, 0]) // 2, int(t["ij"][b, 1]) // 2), -1)
           for b in range(n)}
    R, dropped = set(), 0
    for b in range(n):
        l = int(t["level"][b])
        if not leaf[b] or flags[b] <= 0 or l >= lmax:
            continue
        i, j = int(t["ij"][b, 0]), int(t["ij"][b, 1])
        side = 1 << l
        ok = all((l, i + dx, j + dy) in where for dx, dy in DIRS2
                 if 0 <= i + dx < side and 0 <= j + dy < side)
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
            l, i, j = int(t["level"][c]), int(t["ij"][c, 0]), int(t["ij"][c, 1])
            for dx, dy in DIRS2:
                nb = where.get((l, i + dx, j + dy))
                if nb is not None and par[nb] != p and (not leaf[nb] or nb in R):
                    ok = False
        if ok:
            D.add(p)
    keys = [(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])) for b in range(n)
            if par[b] == -1 or par[b] not in D]
    for b in R:
        l, i, j = int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])
        keys += [(l + 1, 2 * i + (c & 1), 2 * j + (c >> 1)) for c in range(4)]
    keys.sort(key=lambda q: (q[0], synth_morton2(q[1], q[2])))
    return keys, len(R), len(D), dropped


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_regrid_tables_bruteforce(name):
    dom, st, o = mesh(name)
    t = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, 1.0, BUF)
    keys, nr, nd, ndrop = expected_mesh(dom, t, f)
    assert nr > 0 and nd > 0 and ndrop > 0
    assert o.regrid(f) == (nr, nd, ndrop)
    t2 = o.tables()
    assert [(int(t2["level"][b]), int(t2["ij"][b, 0]), int(t2["ij"][b, 1])) for b in range(o.n_boxes)] == keys
    check_tables(t2, dom.lbase)


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_regrid_data_prolongation_and_kept_boxes(name):
    """Kept leaves keep their data bit for bit; new children get the
    prolongation (2c + c_sx + c_sy)/4 of their parent's cells (wall ghosts
    for the potential, mirrors for densities limited to 2c), recomputed
    here by coordinates from the old data; a linear potential is exact."""
    dom, st, o = mesh(name)
    t = set_tip_field(dom, o)
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    g0, g1 = dom.bc_val[2], dom.bc_val[3]
    lin = lambda yy: g0 + (g1 - g0) * (yy - dom.origin[1]) / dom.length
    o.set(quad.PHI, lin(y))
    rng = np.random.default_rng(7)
    # densities over several orders of magnitude, so that the 2c limit acts
    ne = 1e18 * rng.random((o.n_boxes, 64)) ** 4
    o.set(quad.NE, ne)
    o.set(quad.NI, 2.0 * ne)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    o.regrid(np.zeros(o.n_boxes, np.int8))           # the densities' restriction, as the regrid does
    t = o.tables()
    old = {v: o.get(v) for v in (quad.PHI, quad.NE, quad.NI)}
    leaf = t["child"][:, 0] < 0
    li, lj = np.arange(64) & 7, np.arange(64) >> 3
    cells = {}
    for v in old:
        d = {}
        for b in range(o.n_boxes):
            l = int(t["level"][b])
            for c in range(64):
                d[(l, t["ij"][b, 0] * 8 + li[c], t["ij"][b, 1] * 8 + lj[c])] = old[v][b, c]
        cells[v] = d
    oldkey = {(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])): b for b in range(o.n_boxes)}
    nr, nd, _ = o.regrid(f)
    assert nr > 0
    t2 = o.tables()
    new = {v: o.get(v) for v in old}

    def cval(v, l, g, frm):
        side = 8 << l
        if min(g) < 0 or max(g) >= side:
            inner = cells[v][(l, *frm)]
            if v != quad.PHI:
                return inner
            for a in range(2):
                if g[a] < 0 or g[a] >= side:
                    fc = 2 * a + (1 if g[a] >= side else 0)
                    axis = dom.geom == synth.AXISYMMETRIC and fc == 0
                    return (2.0 * dom.bc_val[fc] - inner) if (dom.bc_type[fc] and not axis) else inner
        return cells[v][(l, *g)]

    n_new = 0
    for b in range(o.n_boxes):
        key = (int(t2["level"][b]), int(t2["ij"][b, 0]), int(t2["ij"][b, 1]))
        if key in oldkey:
            if leaf[oldkey[key]]:
                for v in old:
                    assert np.array_equal(new[v][b], old[v][oldkey[key]]), (key, v)
            continue
        n_new += 1
        l = key[0] - 1
        for c in range(64):
            G = (key[1] * 8 + li[c], key[2] * 8 + lj[c])
            cc = (G[0] >> 1, G[1] >> 1)
            for v in old:
                c0v = cells[v][(l, *cc)]
                s = 2.0 * c0v
                for a in range(2):
                    q = list(cc)
                    q[a] += 1 if (G[a] & 1) else -1
                    s += cval(v, l, tuple(q), cc)
                want = 0.25 * s
                if v != quad.PHI and want > 2.0 * c0v:
                    want = 2.0 * c0v
                assert new[v][b, c] == want, (key, c, v)
    assert n_new == 4 * nr
    x2, y2 = synth.cell_centres2(dom, t2["level"], t2["ij"])
    assert np.abs(new[quad.PHI] - lin(y2)).max() <= 1e-12 * max(abs(g0), abs(g1))


def test_regrid_round_trip_and_dropped_requests():
    dom, st, o = mesh()
    t0 = set_tip_field(dom, o)
    f = o.refine_flags(C0, C1, C0D, DXD, BUF)
    keys0 = [(int(t0["level"][b]), int(t0["ij"][b, 0]), int(t0["ij"][b, 1])) for b in range(o.n_boxes)]
    nr, nd, _ = o.regrid(f)
    assert nr > 0 and nd == 0
    t1 = o.tables()
    keys1 = [(int(t1["level"][b]), int(t1["ij"][b, 0]), int(t1["ij"][b, 1])) for b in range(o.n_boxes)]
    added = set(keys1) - set(keys0)
    back = np.array([-1 if k in added else 0 for k in keys1], np.int8)
    assert o.regrid(back)[:2] == (0, nr)
    t2 = o.tables()
    assert [(int(t2["level"][b]), int(t2["ij"][b, 0]), int(t2["ij"][b, 1])) for b in range(o.n_boxes)] == keys0
    # one refined box at level 1 of a 2^2 base: of its children only the
    # corner one has every neighbour position covered or outside the domain
    o2 = quad.Quad(synth.Domain2(1.0, 2, 3, synth.CARTESIAN))
    f1 = np.zeros(o2.n_boxes, np.int8)
    f1[o2.level_range(1)[0]] = 1
    assert o2.regrid(f1) == (1, 0, 0)
    f2 = np.zeros(o2.n_boxes, np.int8)
    lo, hi = o2.level_range(2)
    f2[lo:hi] = 1
    assert o2.regrid(f2) == (1, 0, 3)
    t2 = o2.tables()
    assert tuple(t2["ij"][t2["parent"][o2.level_range(3)[0]]]) == (0, 0)
    check_tables(t2, 1)


def test_regrid_derefinement_blocked_by_nesting():
    o = quad.Quad(synth.Domain2(1.0, 2, 3, synth.CARTESIAN))
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(1)
    f[lo:hi] = 1
    assert o.regrid(f)[0] == 4                      # all of level 2 (16 boxes)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo:lo + 4] = 1                                # the children of the first level-1 box
    assert o.regrid(f)[0] == 4
    assert o.level_range(3)[1] - o.level_range(3)[0] == 16
    check_tables(o.tables(), 1)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo + 4:hi] = -1                               # blocked while level 3 touches them
    assert o.regrid(f)[:2] == (0, 0)
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(3)
    f[lo:hi] = -1
    assert o.regrid(f)[:2] == (0, 4)
    assert o.n_levels == 3
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(2)
    f[lo:hi] = -1
    assert o.regrid(f)[:2] == (0, 4)
    assert o.n_levels == 2
    check_tables(o.tables(), 1)


@pytest.mark.parametrize("geom", [synth.CARTESIAN, synth.AXISYMMETRIC])
def test_derefined_box_holds_the_content_of_its_children(geom):
    """Densities are restricted before the mesh changes: a derefined box
    becomes a leaf whose cells hold the content of their four child cells,
    the mean weighted by the cell volumes (the centre radii in cylindrical
    coordinates)."""
    o = quad.Quad(synth.Domain2(1.0, 2, 3, geom))
    f = np.zeros(o.n_boxes, np.int8)
    p = o.level_range(1)[0]
    f[p] = 1
    assert o.regrid(f)[0] == 1
    rng = np.random.default_rng(12)
    o.set(quad.NE, rng.random((o.n_boxes, 64)))
    o.set(quad.NI, np.zeros((o.n_boxes, 64)))
    t = o.tables()
    kids = t["child"][p]
    ne = o.get(quad.NE)
    want = np.zeros(64)
    for c in range(64):
        I, J = c % 8, c // 8
        kid = kids[(I >> 2) + 2 * (J >> 2)]
        s = ws = 0.0
        for dj in (0, 1):
            for di in (0, 1):
                i, j = 2 * (I & 3) + di, 2 * (J & 3) + dj
                gx = int(t["ij"][kid, 0]) * 8 + i
                w = gx + 0.5 if geom == synth.AXISYMMETRIC else 1.0
                s += w * ne[kid, i + 8 * j]
                ws += w
        want[c] = s / ws
    f = np.zeros(o.n_boxes, np.int8)
    f[kids] = -1
    assert o.regrid(f)[:2] == (0, 1)
    t2 = o.tables()
    b = [i for i in range(o.n_boxes) if t2["level"][i] == 1 and tuple(t2["ij"][i]) == tuple(t["ij"][p])][0]
    assert t2["child"][b, 0] < 0
    assert np.allclose(o.get(quad.NE)[b], want, rtol=1e-14, atol=0)


def test_derefinement_blocked_by_refinement_in_the_same_call():
    """A box whose children touch a box refined in the same call keeps its
    children; the refinement goes ahead."""
    o = quad.Quad(synth.Domain2(1.0, 2, 3, synth.CARTESIAN))
    f = np.zeros(o.n_boxes, np.int8)
    lo, hi = o.level_range(1)
    f[lo:hi] = 1
    assert o.regrid(f)[0] == 4
    t = o.tables()
    at = {(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])): b for b in range(o.n_boxes)}
    a = at[(1, 0, 0)]
    f = np.zeros(o.n_boxes, np.int8)
    f[t["child"][a]] = -1               # derefine the first level-1 box
    f[at[(2, 2, 0)]] = 1                # refine a level-2 box touching its children
    assert o.regrid(f)[:2] == (1, 0)
    check_tables(o.tables(), 1)
