"""Parity of the 2-D / axisymmetric CUDA path (sm_quad_* through the C ABI)
with the CPU oracle (oracle/quad.c).

Tables: bit-exact.  FP64 potential, field, densities: max |gpu - oracle| <=
1e-12 x max |oracle| (both sides FP64; they differ only in rounding order
and fused multiply-adds); |E| after a Heun step within that bound times
max|phi| / (h_min max|E|), the amplification of a potential difference by
the field's division by h.  Cycle counts to a tolerance agree exactly.
"""
import os

import numpy as np
import pytest

import synth
from oracle import quad

pytestmark = pytest.mark.gpu
TOL = 1e-12
Q, EPS0 = synth.E_CHARGE, synth.EPS0


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def pkg():
    import paper_1708_08434_gb300 as p
    return p


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def gpu_quad(dom, st=None, max_boxes=1 << 15):
    g = pkg().Quad(dom, max_boxes)
    if st is not None:
        synth.refine_all2(dom, st, g.level_ij, g.refine_level)
    return g


def pair(name):
    dom, st = synth.workload2(name)
    return dom, st, quad.build_mesh(dom, st), gpu_quad(dom, st)


def load(dom, st, o, g):
    t = o.tables()
    ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
    p = pkg()
    o.set(quad.NE, ne)
    o.set(quad.NI, ni)
    g.upload(p.NE, ne)
    g.upload(p.NI, ni)
    tab = synth.coefficient_table()
    o.set_table(tab)
    g.set_table(tab)
    o.charge_rhs(Q, EPS0)
    g.charge_rhs(Q, EPS0)
    return t


@pytest.mark.parametrize("name", ["axi_small", "cart_small", "axi_streamer"])
def test_tables_bit_exact(name):
    dom, st, o, g = pair(name)
    to, tg = o.tables(), g.tables()
    for k in ("level", "ij", "morton", "parent", "child", "nbr", "level_offset"):
        assert np.array_equal(to[k], tg[k]), k


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_fmg_parity(name):
    dom, st, o, g = pair(name)
    load(dom, st, o, g)
    # the two sides' residual norms differ by the rounding of f - L phi
    # (about 2e-15 of the denominator here), the floor below which a
    # relative residual carries no digits
    so = o.fmg(1e-8, 40)
    sg = g.fmg(1e-8, 40)
    assert so[0] == sg[0] == 0
    assert so[2] == sg[2]
    assert abs(so[1] - sg[1]) <= 1e-6 * so[1] + 1e-13
    assert rel_err(g.download(pkg().PHI), o.get(quad.PHI)) <= TOL


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_fixed_cycles_parity(name):
    """Three V-cycles from zero (no stopping test): every box of every level
    agrees, coarse levels included."""
    dom, st, o, g = pair(name)
    load(dom, st, o, g)
    o.vcycles(3)
    rc, rel, cyc = g.solve(0.0, 3)
    assert cyc == 3
    assert abs(rel - o.rel_residual()) <= 1e-6 * rel + 1e-13
    assert rel_err(g.download(pkg().PHI), o.get(quad.PHI)) <= TOL


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_field_dt_and_stage_parity(name):
    dom, st, o, g = pair(name)
    t = load(dom, st, o, g)
    o.fmg(1e-10, 40)
    g.fmg(1e-10, 40)
    o.compute_field()
    g.compute_field()
    p = pkg()
    leaf = t["child"][:, 0] < 0
    assert rel_err(g.download(p.EMAG)[leaf], o.get(quad.EMAG)[leaf]) <= TOL
    dt = o.dt_limit(Q, EPS0)
    assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
    o.fluid_stage(dt)
    g.fluid_stage(dt)
    assert rel_err(g.download(p.NE)[leaf], o.get(quad.NE)[leaf]) <= TOL
    assert rel_err(g.download(p.NI)[leaf], o.get(quad.NI)[leaf]) <= TOL
    # refined boxes hold the restriction of their children on both sides
    assert rel_err(g.download(p.NE), o.get(quad.NE)) <= TOL


def check_advance(name, threads=1):
    dom, st, o, g = pair(name)
    t = load(dom, st, o, g)
    quad.set_threads(threads)
    try:
        so = o.fmg(1e-8, 40)
        sg = g.fmg(1e-8, 40)
        assert so[2] == sg[2]
        o.compute_field()
        g.compute_field()
        dt = o.dt_limit(Q, EPS0)
        assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
        ro = o.advance(dt, Q, EPS0, 1e-8, 40)
        rg = g.advance(dt, Q, EPS0, 1e-8, 40)
    finally:
        quad.set_threads(1)
    assert ro[0] == rg[0] == 0
    assert ro[2:] == rg[2:], (ro, rg)
    assert rg[1] == pytest.approx(ro[1], rel=TOL)
    leaf = t["child"][:, 0] < 0
    p = pkg()
    for vo, vg in ((quad.NE, p.NE), (quad.NI, p.NI), (quad.PHI, p.PHI)):
        e = rel_err(g.download(vg)[leaf], o.get(vo)[leaf])
        assert e <= TOL, (vo, e)
    # |E| is a difference of potentials over h: a potential difference of
    # TOL max|phi| becomes TOL max|phi| / h_min in |E|, i.e. the relative
    # bound grows by max|phi| / (h_min max|E|) (2e4 on the benchmark mesh,
    # whose finest spacing is 0.12 um)
    eo, po = o.get(quad.EMAG)[leaf], o.get(quad.PHI)[leaf]
    amp = max(1.0, np.abs(po).max() / (dom.h(o.n_levels - 1) * np.abs(eo).max()))
    e = rel_err(g.download(p.EMAG)[leaf], eo)
    assert e <= TOL * amp, (e, amp)
    return g, leaf


@pytest.mark.parametrize("name", ["axi_small", "cart_small", "axi_streamer"])
def test_field_from_the_same_potential(name):
    """|E| of the field kernel against the oracle's field computed from the
    GPU's own solved potential (all boxes, so the refinement ghosts are
    formed from the same values): with the solver's conditioning out of the
    comparison, every leaf cell agrees to 1e-12 of its own value plus one
    unit in the last place of max|phi| over the cell's own spacing h (the
    two sides round the interpolated ghost potentials differently, and |E|
    divides potential differences by h)."""
    dom, st, o, g = pair(name)
    t = load(dom, st, o, g)
    g.fmg(1e-8, 40)
    p = pkg()
    phi = g.download(p.PHI)
    o.set(quad.PHI, phi)
    o.compute_field()
    g.compute_field()
    leaf = t["child"][:, 0] < 0
    eo, eg = o.get(quad.EMAG)[leaf], g.download(p.EMAG)[leaf]
    h = np.array([dom.h(l) for l in t["level"][leaf]])[:, None]
    bound = TOL * np.abs(eo) + 2.0 ** -52 * np.abs(phi).max() / h
    bad = np.abs(eg - eo) > bound
    assert not bad.any(), (np.abs(eg - eo)[bad][:5], eo[bad][:5])
    print("%s: max |dE| / bound %.3e" % (name, (np.abs(eg - eo) / bound).max()))


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_heun_step_parity(name):
    check_advance(name)


def test_full_size_axi_streamer_parity():
    """The benchmark workload (axisymmetric 16 mm, base 512^2 cells + 8
    levels, 10113 boxes, 4.9e5 leaf cells): FMG to 1e-8, field, one Heun
    step, element-wise parity (the oracle on all host cores)."""
    g, leaf = check_advance("axi_streamer", threads=os.cpu_count() or 1)
    assert leaf.sum() * 64 > 4.5e5


def test_single_box_and_uniform_domains():
    """Degenerate meshes: one box (FMG is the exact level-0 solve) and a
    uniform grid without refinement, in both geometries."""
    p = pkg()
    for geom in (synth.CARTESIAN, synth.AXISYMMETRIC):
        for nb in (1, 8):
            dom = synth.Domain2(0.01, nb, 0, geom, bc_val=(0.0, 0.0, 0.0, 1e3))
            o, g = quad.Quad(dom), gpu_quad(dom)
            t = o.tables()
            x, y = synth.cell_centres2(dom, t["level"], t["ij"])
            rho = 1e-6 * np.exp(-((x - 0.004) ** 2 + (y - 0.005) ** 2) / 2e-6)
            o.set(quad.RHO, rho)
            g.upload(p.RHO, rho)
            o.charge_rhs(1.0, EPS0, True)
            g.charge_rhs(1.0, EPS0, True)
            so, sg = o.fmg(1e-11, 40), g.fmg(1e-11, 40)
            assert so[2] == sg[2]
            assert rel_err(g.download(p.PHI), o.get(quad.PHI)) <= TOL


@pytest.mark.parametrize("bct", [(1, 1, 0, 0), (1, 0, 1, 0), (0, 1, 0, 1)])
def test_boundary_condition_mixes(bct):
    p = pkg()
    dom = synth.Domain2(1.0, 4, 2, synth.CARTESIAN, bc_type=bct, bc_val=(0.3, -0.2, 0.5, 1.0))
    st = synth.Streamer2(length=1.0, radius=0.05, z_head=0.5, edge=0.01, shell=0.005, x_axis=0.5,
                         refine_c=1.0, refine_tip=0.5)
    o, g = quad.build_mesh(dom, st), gpu_quad(dom, st)
    t = o.tables()
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    rho = np.sin(3 * x) * np.cos(2 * y)
    o.set(quad.RHO, rho)
    g.upload(p.RHO, rho)
    o.charge_rhs(1.0, 1.0, True)
    g.charge_rhs(1.0, 1.0, True)
    so, sg = o.fmg(1e-11, 40), g.fmg(1e-11, 40)
    assert so[2] == sg[2]
    assert rel_err(g.download(p.PHI), o.get(quad.PHI)) <= TOL


def test_error_paths():
    p = pkg()
    dom, st = synth.workload2("axi_small")
    g = gpu_quad(dom)
    with pytest.raises(p.SmError):
        g.refine_level(0, np.ones(1, np.int8))          # not the finest level
    with pytest.raises(p.SmError):
        g.dt_limit(Q, EPS0)                             # no table yet
    with pytest.raises(p.SmError):
        g.fluid_stage(1e-12)
    small = p.Quad(dom, 21 + 3)                         # room for the uniform levels only
    with pytest.raises(p.SmError):
        small.refine_level(2, np.ones(16, np.int8))


def test_graph_and_host_paths_identical():
    """V-cycles as CUDA graphs or from the host, with or without programmatic
    dependent launch, give the same bits and the same launch count."""
    p = pkg()
    out = []
    for graphs, pdl in ((True, True), (True, False), (False, True), (False, False)):
        dom, st = synth.workload2("axi_small")
        g = gpu_quad(dom, st)
        g.set_graphs(graphs)
        g.set_pdl(pdl)
        o = quad.build_mesh(dom, st)
        load(dom, st, o, g)
        l0 = g.launch_count()
        rc, rel, cyc = g.fmg(1e-9, 40)
        out.append((cyc, rel, g.download(p.PHI), g.launch_count() - l0))
    for o_ in out[1:]:
        assert o_[0] == out[0][0] and o_[1] == out[0][1] and o_[3] == out[0][3]
        assert np.array_equal(o_[2], out[0][2])


# ---- refinement criterion and regridding (Sec. 2.5, Eq. 8) ----
def tip_field(dom, t, centre=(4e-3, 5e-3), e_peak=2e7, e_bg=1.5e6, sigma=1.5e-3):
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    return e_bg + e_peak * np.exp(-((x - centre[0]) ** 2 + (y - centre[1]) ** 2) / (2 * sigma ** 2))


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_refine_flags_bit_exact(name):
    """The same |E| on both sides: flags agree entry by entry, with and
    without the buffer, with derefinements."""
    p = pkg()
    dom, st, o, g = pair(name)
    load(dom, st, o, g)
    em = tip_field(dom, o.tables())
    o.set(quad.EMAG, em)
    g.upload(p.EMAG, em)
    for args in ((1.0, 1.2, 0.125, 30e-6, 3), (1.0, 1.2, 0.125, 30e-6, 0), (1.0, 1.2, 0.125, 1.0, 3),
                 (0.05, 1.2, 0.125, 1.0, 8)):
        fo, fg = o.refine_flags(*args), g.refine_flags(*args)
        assert np.array_equal(fo, fg), args
    assert (fo == 1).sum() > 0 and (fo == -1).sum() > 0


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_regrid_parity(name):
    """The oracle's flags applied on both sides: tables bit-exact, kept and
    prolonged data equal, then FMG on the new mesh agrees."""
    p = pkg()
    dom, st, o, g = pair(name)
    load(dom, st, o, g)
    t = o.tables()
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    phi = dom.bc_val[3] * y / dom.length + 50.0 * np.sin(x * 400.0)
    for side, var in ((o, quad.PHI), (g, p.PHI)):
        (side.set if side is o else side.upload)(var, phi)
    em = tip_field(dom, t)
    o.set(quad.EMAG, em)
    g.upload(p.EMAG, em)
    f = o.refine_flags(1.0, 1.2, 0.125, 1.0, 3)
    ro, rg = o.regrid(f), g.regrid(f)
    assert ro == rg and ro[0] > 0 and ro[1] > 0 and ro[2] > 0, (ro, rg)
    to, tg = o.tables(), g.tables()
    for k in ("level", "ij", "morton", "parent", "child", "nbr", "level_offset"):
        assert np.array_equal(to[k], tg[k]), k
    for vo, vg in ((quad.PHI, p.PHI), (quad.NE, p.NE), (quad.NI, p.NI)):
        assert rel_err(g.download(vg), o.get(vo)) <= TOL, vo
    o.charge_rhs(Q, EPS0)
    g.charge_rhs(Q, EPS0)
    so, sg = o.fmg(1e-8, 40), g.fmg(1e-8, 40)
    assert so[2] == sg[2]
    assert rel_err(g.download(p.PHI), o.get(quad.PHI)) <= TOL


def test_regrid_parity_full_size_axi_streamer():
    """The benchmark mesh (10113 boxes): a regrid that refines and
    derefines hundreds of boxes, with prefix sums over many entries per
    thread, gives the oracle's tables and data."""
    p = pkg()
    dom, st = synth.workload2("axi_streamer")
    o = quad.build_mesh(dom, st)
    g = gpu_quad(dom, st, max_boxes=1 << 16)
    t = load(dom, st, o, g)
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    phi = dom.bc_val[3] * y / dom.length + 50.0 * np.sin(x * 400.0)
    o.set(quad.PHI, phi)
    g.upload(p.PHI, phi)
    em = tip_field(dom, t)
    o.set(quad.EMAG, em)
    g.upload(p.EMAG, em)
    f = o.refine_flags(0.25, 1.2, 0.125, 30e-6, 3)
    ro, rg = o.regrid(f), g.regrid(f)
    assert ro == rg and ro[0] > 100 and ro[1] > 100, (ro, rg)
    to, tg = o.tables(), g.tables()
    assert len(to["level"]) > 9000
    for k in ("level", "ij", "morton", "parent", "child", "nbr", "level_offset"):
        assert np.array_equal(to[k], tg[k]), k
    for vo, vg in ((quad.PHI, p.PHI), (quad.NE, p.NE), (quad.NI, p.NI), (quad.EMAG, p.EMAG)):
        assert rel_err(g.download(vg), o.get(vo)) <= TOL, vo
    # a second regrid from the device's own tables (derefining what the
    # first one refined is allowed, the rules decide)
    f2 = o.refine_flags(1.0, 1.2, 0.125, 30e-6, 3)
    assert np.array_equal(f2, g.refine_flags(1.0, 1.2, 0.125, 30e-6, 3))
    assert o.regrid(f2) == g.regrid(f2)
    to, tg = o.tables(), g.tables()
    for k in ("level", "ij", "morton", "parent", "child", "nbr", "level_offset"):
        assert np.array_equal(to[k], tg[k]), k


@pytest.mark.parametrize("name,c0,dxd", [("axi_small", 0.005, 1.0), ("cart_small", 0.05, 30e-6)])
def test_adaptive_step_parity(name, c0, dxd):
    """Solve, field, flags from each side's own field (a stricter c0 than
    the paper's, so that these small meshes refine), regrid, solve and one
    Heun step on the new mesh."""
    p = pkg()
    dom, st, o, g = pair(name)
    t = load(dom, st, o, g)
    o.fmg(1e-8, 40)
    g.fmg(1e-8, 40)
    o.compute_field()
    g.compute_field()
    fo, fg = o.refine_flags(c0, 1.2, 0.125, dxd, 3), g.refine_flags(c0, 1.2, 0.125, dxd, 3)
    assert np.array_equal(fo, fg)
    ro, rg = o.regrid(fo), g.regrid(fg)
    assert ro == rg and ro[0] > 0
    to, tg = o.tables(), g.tables()
    for k in ("level", "ij", "child", "nbr"):
        assert np.array_equal(to[k], tg[k]), k
    o.charge_rhs(Q, EPS0)
    g.charge_rhs(Q, EPS0)
    so, sg = o.fmg(1e-8, 40), g.fmg(1e-8, 40)
    assert so[2] == sg[2]
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
    ao, ag = o.advance(dt, Q, EPS0, 1e-8, 40), g.advance(dt, Q, EPS0, 1e-8, 40)
    assert ao[2:] == ag[2:]
    leaf = to["child"][:, 0] < 0
    for vo, vg in ((quad.NE, p.NE), (quad.PHI, p.PHI)):
        assert rel_err(g.download(vg)[leaf], o.get(vo)[leaf]) <= TOL, vo


def test_regrid_capacity_and_argument_errors():
    """A regrid past max_boxes fails with SM_ENOMEM and leaves the mesh as it
    was; a buffer outside 0..8 is rejected; a refinement with no flags adds
    nothing."""
    p = pkg()
    dom, st = synth.workload2("axi_small")
    o = quad.build_mesh(dom, st)
    n0 = o.n_boxes
    g = gpu_quad(dom, st, max_boxes=n0 + 3)          # room for less than one refinement
    load(dom, st, o, g)
    t0 = g.tables()
    em = tip_field(dom, t0)
    g.upload(p.EMAG, em)
    f = g.refine_flags(1.0, 1.2, 0.125, 30e-6, 3)
    assert (f == 1).sum() > 0
    with pytest.raises(p.SmError) as ei:
        g.regrid(f)
    assert ei.value.code == p.SM_ENOMEM
    t1 = g.tables()
    for k in ("level", "ij", "child", "nbr", "level_offset"):
        assert np.array_equal(t0[k], t1[k]), k
    for bad in (-1, 9):
        with pytest.raises(p.SmError) as ei:
            g.refine_flags(1.0, 1.2, 0.125, 30e-6, bad)
        assert ei.value.code == p.SM_EINVAL
    g2 = gpu_quad(synth.Domain2(1.0, 2, 2, synth.CARTESIAN))
    assert g2.refine_level(1, np.zeros(4, np.int8)) == 0
    assert g2.n_boxes == 5 and g2.n_levels == 2


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_paper_schedule_multi_step(name):
    """The paper's schedule in 2-D (Sec. 2.1.2, 2.4): one FMG solve, then
    eight Heun steps with exactly two V-cycles per potential update and the
    time step from the limits of Sec. 2.4; both sides advance with the
    oracle's time step, the GPU's own limit is compared with it, and the
    fields agree element by element after every step."""
    p = pkg()
    dom, st, o, g = pair(name)
    t = load(dom, st, o, g)
    o.fmg(1e-8, 40)
    g.fmg(1e-8, 40)
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
    leaf = t["child"][:, 0] < 0
    for step in range(8):
        ro = o.advance(dt, Q, EPS0, 0.0, 2)
        rg = g.advance(dt, Q, EPS0, 0.0, 2)
        assert ro[2:] == rg[2:] == (2, 2), (step, ro, rg)
        assert rg[1] == pytest.approx(ro[1], rel=TOL), step
        for vo, vg in ((quad.NE, p.NE), (quad.NI, p.NI), (quad.PHI, p.PHI)):
            e = rel_err(g.download(vg)[leaf], o.get(vo)[leaf])
            assert e <= TOL, (step, vo, e)
        eo, po = o.get(quad.EMAG)[leaf], o.get(quad.PHI)[leaf]
        amp = max(1.0, np.abs(po).max() / (dom.h(o.n_levels - 1) * np.abs(eo).max()))
        assert rel_err(g.download(p.EMAG)[leaf], eo) <= TOL * amp, step
        dt = ro[1]
    assert 1e-14 < o.rel_residual() < 1e-2


def test_repeatable_bits_full_size_axi_streamer():
    """The same FMG solve and Heun step on two fresh quadtree solvers give
    the same bits (no block of a launch reads what another block of it
    writes)."""
    p = pkg()
    dom, st = synth.workload2("axi_streamer")
    runs = []
    for _ in range(2):
        g = gpu_quad(dom, st)
        t = g.tables()
        ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
        g.upload(p.NE, ne)
        g.upload(p.NI, ni)
        g.set_table(synth.coefficient_table())
        g.charge_rhs(Q, EPS0)
        c1 = g.fmg(1e-8, 40)[2]
        g.compute_field()
        dt = g.dt_limit(Q, EPS0)
        c2 = g.advance(dt, Q, EPS0, 1e-8, 40)[2:]
        runs.append((c1, c2, g.download(p.PHI).view(np.int64).copy(), g.download(p.NE).view(np.int64).copy()))
    assert runs[0][0] == runs[1][0] and runs[0][1] == runs[1][1]
    assert np.array_equal(runs[0][2], runs[1][2]) and np.array_equal(runs[0][3], runs[1][3])
