"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Tables: bit-exact.  FP64 potential and field: max |gpu - oracle| <= 1e-12 x
max |oracle| (the FP64 tolerance of the method's solve).  Densities after a
fluid stage or Heun step: same 1e-12 relative bound (FP64 throughout; the
two sides differ only in rounding order and fused multiply-adds).
Cycle counts to a tolerance must agree exactly (max-norm residuals).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import EPS0, Q, gpu_mesh, load_inputs, pair, rel_err, rel_err_local

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


TABLE_KEYS = ("level", "ijk", "morton", "parent", "child", "nbr")


def assert_tables_equal(o, g):
    to, tg = o.tables(), g.tables()
    for k in TABLE_KEYS:
        assert to[k].shape == tg[k].shape, k
        assert np.array_equal(to[k], tg[k]), k
    assert np.array_equal(to["level_offset"], tg["level_offset"])
    leaf = np.where(to["child"][:, 0] < 0)[0]
    assert np.array_equal(leaf, tg["leaf"])
    return to


@pytest.mark.parametrize("name", ["uniform64", "streamer_small", "streamer6"])
def test_tables_bit_exact(name):
    dom, st, o, g = pair(name)
    assert_tables_equal(o, g)
    if st is not None:
        assert o.dropped == g.dropped


def test_tables_nesting_drop_and_empty_refinement():
    dom = synth.Domain(length=1.0, nb=2, max_level=3)
    o = oracle.Oracle(dom)
    g = gpu_mesh(dom)
    f1 = np.zeros(8, np.int8)
    f1[0] = 1
    assert o.refine_level(1, f1) == g.refine_level(1, f1) == 8
    lo, hi = o.level_range(2)
    f2 = np.zeros(hi - lo, np.int8)
    ijk2 = o.level_ijk(2)
    for b, q in enumerate(map(tuple, ijk2)):
        if q in ((1, 1, 1), (0, 0, 0)):
            f2[b] = 1
    o.refine_level(2, f2)
    g.refine_level(2, f2)
    assert o.dropped == g.dropped == 1
    assert_tables_equal(o, g)
    # a request list with nothing to refine leaves the octree unchanged
    lo, hi = o.level_range(3)
    z = np.zeros(hi - lo, np.int8)
    assert o.refine_level(3, z) == 0 and g.refine_level(3, z) == 0
    assert_tables_equal(o, g)


@pytest.mark.parametrize("name", ["uniform64", "streamer_small"])
def test_fmg_fixed_cycles_and_tolerance(name):
    dom, st, o, g = pair(name)
    t = assert_tables_equal(o, g)
    load_inputs(dom, st, o, g, t)
    # identical work: FMG plus 2 more cycles regardless of tolerance
    so = o.fmg(0.0, 3)
    sg = g.fmg(0.0, 3)
    assert so[2] == sg[2] == 3
    p = pkg()
    po, pg = o.get(oracle.PHI), g.download(p.PHI)
    assert rel_err(pg, po) <= TOL
    assert abs(so[1] - sg[1]) <= 1e-6 * so[1]
    # same stopping decision to a tolerance from a warm start
    ro = o.solve(1e-10, 30)
    rg = g.solve(1e-10, 30)
    assert ro[0] == rg[0] == 0 and ro[2] == rg[2]
    assert rel_err(g.download(p.PHI), o.get(oracle.PHI)) <= TOL


def test_vcycle_residual_history_matches():
    dom, st, o, g = pair("streamer_small")
    load_inputs(dom, st, o, g)
    for _ in range(4):
        ro = o.vcycles(1)
        rg = g.vcycles(1)
        assert rg == pytest.approx(ro, rel=1e-6)


def test_field_parity():
    dom, st, o, g = pair("streamer_small")
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    o.fmg(1e-10, 30)
    g.fmg(1e-10, 30)
    o.compute_field()
    g.compute_field()
    leaf = t["child"][:, 0] < 0
    p = pkg()
    assert rel_err(g.download(p.EMAG)[leaf], o.get(oracle.EMAG)[leaf]) <= TOL
    assert g.dt_limit(Q, EPS0) == pytest.approx(o.dt_limit(Q, EPS0), rel=TOL)


@pytest.mark.parametrize("name", ["streamer_small", "streamer_small_bg"])
def test_field_from_the_same_potential(name):
    """|E| of k_field against the oracle's field computed from the GPU's own
    solved potential (all boxes, so refinement ghosts agree too): without
    the solver's conditioning every leaf cell agrees to 1e-12 of its own
    value, plus 1e-15 max|E| where the field nearly vanishes; and the time
    step from the same potential and field to 1e-12."""
    dom, st, o, g = pair(name)
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    g.fmg(1e-10, 30)
    p = pkg()
    o.set(oracle.PHI, g.download(p.PHI))
    o.compute_field()
    g.compute_field()
    leaf = t["child"][:, 0] < 0
    eo, eg = o.get(oracle.EMAG)[leaf], g.download(p.EMAG)[leaf]
    bad = np.abs(eg - eo) > TOL * np.abs(eo) + 1e-3 * TOL * np.abs(eo).max()
    assert not bad.any(), (np.abs(eg - eo)[bad][:5], eo[bad][:5])
    assert g.dt_limit(Q, EPS0) == pytest.approx(o.dt_limit(Q, EPS0), rel=TOL)


@pytest.mark.parametrize("name", ["streamer_small", "streamer_small_bg", "uniform64"])
def test_row_kernels_bit_identical(name):
    """The row kernels of the fixed-point cycle (colour pass, residual and
    restriction), forced onto every level, give the same bits as the box
    kernels: FMG, then a warm-started solve to a tighter tolerance, on the
    captured graphs and on the host loop."""
    dom, st = synth.workload(name)
    p = pkg()
    out = []
    for rows in (1 << 30, 0):
        g = gpu_mesh(dom, st)
        t = g.tables()
        if st is None:
            rho = synth.gaussian_charge(dom, t["level"], t["ijk"], np.arange(len(t["level"])))
            g.upload(p.RHO, rho)
            g.charge_rhs(1.0, 1.0, True)
        else:
            ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
            g.upload(p.NE, ne)
            g.upload(p.NI, ni)
            g.charge_rhs(Q, EPS0)
        g.set_row_kernels(rows)
        r1 = g.fmg(1e-8, 30)
        phi1 = g.download(p.PHI)
        r2 = g.solve(1e-11, 30)
        phi2 = g.download(p.PHI)
        g.set_graphs(False)
        r3 = g.solve(1e-12, 30)
        phi3 = g.download(p.PHI)
        out.append((r1, r2, r3, phi1, phi2, phi3))
        g.close()
    a, b = out
    for x, y in zip(a[:3], b[:3]):
        assert x == y
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(x.view(np.int64), y.view(np.int64))


def test_fluid_stage_parity():
    dom, st, o, g = pair("streamer_small")
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    o.fmg(1e-10, 30)
    g.fmg(1e-10, 30)
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    o.fluid_stage(dt)
    g.fluid_stage(dt)
    leaf = t["child"][:, 0] < 0
    p = pkg()
    assert rel_err(g.download(p.NE)[leaf], o.get(oracle.NE)[leaf]) <= TOL
    assert rel_err(g.download(p.NI)[leaf], o.get(oracle.NI)[leaf]) <= TOL
    # refined boxes hold the average of their children on both sides
    assert rel_err(g.download(p.NE), o.get(oracle.NE)) <= TOL


def check_advance(name, tol_solve=1e-8):
    dom, st, o, g = pair(name)
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    so = o.fmg(tol_solve, 40)
    sg = g.fmg(tol_solve, 40)
    assert so[2] == sg[2]
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
    ro = o.advance(dt, Q, EPS0, tol_solve, 40)
    rg = g.advance(dt, Q, EPS0, tol_solve, 40)
    assert ro[0] == rg[0] == 0
    assert ro[2:] == rg[2:], (ro, rg)
    assert rg[1] == pytest.approx(ro[1], rel=TOL)
    leaf = t["child"][:, 0] < 0
    p = pkg()
    for vo, vg in ((oracle.NE, p.NE), (oracle.NI, p.NI), (oracle.PHI, p.PHI), (oracle.EMAG, p.EMAG)):
        e = rel_err(g.download(vg)[leaf], o.get(vo)[leaf])
        assert e <= TOL, (vo, e)
    return g


def test_heun_step_parity_small():
    check_advance("streamer_small")


def test_heun_step_parity_with_stochastic_background():
    """The streamer with the seeded stochastic background of the learned-form
    workload (mean 1e13 m^-3 against 1e19-1e20 in the channel and head):
    densities after FMG, field and one Heun step are compared cell by cell
    against max(|oracle|, the largest |oracle| in the cell's box and its
    neighbours), so background cells are held to their own scale, not to
    the head's.  The error of an FP64 finite-volume update is a few units of
    rounding of the largest density it combines; the same bound holds in
    the streamer boxes, where the local scale is the head's."""
    dom, st, o, g = pair("streamer_small_bg")
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    so = o.fmg(1e-8, 40)
    sg = g.fmg(1e-8, 40)
    assert so[2] == sg[2]
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    ro = o.advance(dt, Q, EPS0, 1e-8, 40)
    rg = g.advance(dt, Q, EPS0, 1e-8, 40)
    assert ro[2:] == rg[2:]
    leaf = t["child"][:, 0] < 0
    p = pkg()
    for vo, vg in ((oracle.NE, p.NE), (oracle.NI, p.NI)):
        ref, got = o.get(vo), g.download(vg)
        assert ref[leaf].min() > 0.0
        e = rel_err_local(got, ref, t)
        print("density", vo, "local-scale rel err %.3e" % e)
        assert e <= TOL, (vo, e)
    for vo, vg in ((oracle.PHI, p.PHI), (oracle.EMAG, p.EMAG)):
        assert rel_err(g.download(vg)[leaf], o.get(vo)[leaf]) <= TOL


@pytest.mark.slow
def test_full_size_streamer6_parity():
    """The benchmark workload (16 mm cube, base 64^3 + 6 levels, 2.4e6 leaf
    cells): FMG to 1e-8, field, one Heun step, element-wise parity."""
    g = check_advance("streamer6")
    assert g.n_leaves * 512 > 2.0e6


@pytest.mark.slow
def test_full_size_streamer8_parity():
    """The 8-level workload (1.7e7 leaf cells, 37481 boxes, 12 levels) in
    the default launch configuration: bit-exact tables, then FMG to 1e-8,
    field, time step and one Heun step, element-wise parity.  Seven of its
    levels hold at least 2048 boxes, so the row kernels (colour pass,
    residual-restriction, prolongation) run there as they do on the
    largest meshes.  The oracle runs its per-box loops on every host core
    (its results do not depend on the thread count)."""
    import os
    dom, st = synth.workload("streamer8")
    o = oracle.build_mesh(dom, st)
    g = gpu_mesh(dom, st, max_boxes=1 << 16)
    t = assert_tables_equal(o, g)
    per_level = np.bincount(t["level"])
    assert (per_level >= 2048).sum() >= 5 and g.n_leaves * 512 > 1.5e7
    n0 = oracle.threads()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        load_inputs(dom, st, o, g, t)
        so = o.fmg(1e-8, 40)
        sg = g.fmg(1e-8, 40)
        assert so[2] == sg[2]
        assert so[1] <= 1e-8 and sg[1] <= 1e-8
        # the two sides' FMG residuals differ (4.6e-9 against 3.4e-9): at
        # 1e-8 the max-norm residual of the 1 um level is within about a
        # hundred units of rounding of phi, so only the tolerance is
        # compared, and the oracle's operator, handed the GPU potential,
        # must find it met as well
        p = pkg()
        leaf = t["child"][:, 0] < 0
        phi_o, phi_g = o.get(oracle.PHI), g.download(p.PHI)
        assert rel_err(phi_g[leaf], phi_o[leaf]) <= TOL
        o.set(oracle.PHI, phi_g)
        assert o.rel_residual() <= 1.01e-8
        o.set(oracle.PHI, phi_o)
        o.compute_field()
        g.compute_field()
        dt = o.dt_limit(Q, EPS0)
        assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
        ro = o.advance(dt, Q, EPS0, 1e-8, 40)
        rg = g.advance(dt, Q, EPS0, 1e-8, 40)
    finally:
        oracle.set_threads(n0)
    assert ro[0] == rg[0] == 0
    assert ro[2:] == rg[2:], (ro, rg)
    for vo, vg in ((oracle.NE, p.NE), (oracle.NI, p.NI), (oracle.PHI, p.PHI), (oracle.EMAG, p.EMAG)):
        e = rel_err(g.download(vg)[leaf], o.get(vo)[leaf])
        assert e <= TOL, (vo, e)


def test_paper_schedule_multi_step():
    """The paper's schedule (Sec. 2.1.2, Sec. 2.4): one FMG solve at the
    start, then every Heun step with exactly two V-cycles per potential
    update (no tolerance) and the time step from the limits of Sec. 2.4.
    Eight steps on the small streamer mesh; both sides advance with the
    oracle's time step, the GPU's own limit is compared with it, and
    densities, potential and field agree element by element after every
    step."""
    dom, st, o, g = pair("streamer_small")
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    o.fmg(1e-8, 40)
    g.fmg(1e-8, 40)
    o.compute_field()
    g.compute_field()
    dt = o.dt_limit(Q, EPS0)
    assert g.dt_limit(Q, EPS0) == pytest.approx(dt, rel=TOL)
    leaf = t["child"][:, 0] < 0
    p = pkg()
    for step in range(8):
        ro = o.advance(dt, Q, EPS0, 0.0, 2)
        rg = g.advance(dt, Q, EPS0, 0.0, 2)
        assert ro[2:] == rg[2:] == (2, 2), (step, ro, rg)
        assert rg[1] == pytest.approx(ro[1], rel=TOL), step
        for vo, vg in ((oracle.NE, p.NE), (oracle.NI, p.NI), (oracle.PHI, p.PHI), (oracle.EMAG, p.EMAG)):
            e = rel_err(g.download(vg)[leaf], o.get(vo)[leaf])
            assert e <= TOL, (step, vo, e)
        dt = ro[1]
    # the fixed schedule leaves an algebraic error: the residual is small
    # but above what a converged solve reaches
    assert 1e-14 < o.rel_residual() < 1e-2


def test_single_box_domain():
    """nb = 1: the whole solve is the exact level-0 solve."""
    dom = synth.Domain(length=2.0, nb=1, max_level=0, bc_type=(1, 0, 0, 1, 1, 0),
                       bc_val=(1.0, 0.0, 0.0, -2.0, 0.5, 0.0))
    o = oracle.Oracle(dom)
    g = gpu_mesh(dom)
    t = assert_tables_equal(o, g)
    rho = synth.gaussian_charge(dom, t["level"], t["ijk"], np.arange(1), sigma=0.3)
    p = pkg()
    o.set(oracle.RHO, rho); g.upload(p.RHO, rho)
    o.charge_rhs(1.0, 1.0, True); g.charge_rhs(1.0, 1.0, True)
    so = o.fmg(1e-12, 3)
    sg = g.fmg(1e-12, 3)
    assert so[2] == sg[2] == 1 and so[1] < 1e-13 and sg[1] < 1e-13
    assert rel_err(g.download(p.PHI), o.get(oracle.PHI)) <= TOL


@pytest.mark.parametrize("bct", [(1, 1, 1, 1, 1, 1), (0, 1, 1, 0, 0, 1)])
def test_boundary_condition_mixes(bct):
    dom = synth.Domain(length=1.0, nb=4, max_level=2, bc_type=bct,
                       bc_val=(0.3, -0.2, 0.0, 1.0, 0.0, 2.0))
    st = synth.Streamer(length=1.0, radius=0.1, z_head=0.45, refine_c=2.0, refine_tip=0.4)
    o = oracle.build_mesh(dom, st)
    g = gpu_mesh(dom, st)
    t = assert_tables_equal(o, g)
    assert o.n_levels == 5
    rho = synth.gaussian_charge(dom, t["level"], t["ijk"], np.arange(len(t["level"])))
    p = pkg()
    o.set(oracle.RHO, rho); g.upload(p.RHO, rho)
    o.charge_rhs(1.0, 1.0, True); g.charge_rhs(1.0, 1.0, True)
    so = o.fmg(1e-11, 30)
    sg = g.fmg(1e-11, 30)
    assert so[2] == sg[2]
    assert rel_err(g.download(p.PHI), o.get(oracle.PHI)) <= TOL


def test_error_paths():
    p = pkg()
    dom = synth.domain_uniform_cube(64)
    g = p.Solver(dom, 600)
    with pytest.raises(p.SmError) as e:
        g.solve(1e-8, 5)
    assert e.value.code == p.SM_ESTATE
    g.build_octree()
    dom2, st = synth.workload("streamer_small")
    g2 = p.Solver(dom2, 80)
    g2.build_octree()
    with pytest.raises(p.SmError) as e:
        synth.refine_all(dom2, st, g2.level_ijk, g2.refine_level)
    assert e.value.code == p.SM_ENOMEM
    with pytest.raises(p.SmError) as e:
        g.refine_level(1, np.ones(8, np.int8))    # not the finest level
    assert e.value.code == p.SM_EINVAL
    # max_cycles reached: SM_ENOCONV reported, potential still updated
    rho = np.ones((g.n_boxes, 512))
    g.upload(p.RHO, rho)
    g.charge_rhs(1.0, 1.0, True)
    rc, rel, cyc = g.fmg(1e-30, 2)
    assert rc == p.SM_ENOCONV and cyc == 2 and rel < 1e-2


def test_graph_direct_pdl_and_persistent_paths_identical():
    """Captured solves (device-side cycle loop) launch the same work in the
    same order as the host-driven path; programmatic dependent launch only
    lets a kernel start waiting early; the persistent kernel runs the same
    per-box operations between grid barriers: every combination gives
    bit-identical results."""
    dom, st = synth.workload("streamer_small")
    p = pkg()
    out = []
    for graphs, pdl, persist in ((True, True, True), (False, True, True), (True, True, False),
                                 (False, True, False), (True, False, False), (False, False, False)):
        g = gpu_mesh(dom, st)
        g.set_graphs(graphs)
        g.set_pdl(pdl)
        g.set_persistent(persist)
        t = g.tables()
        ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
        g.upload(p.NE, ne); g.upload(p.NI, ni)
        g.charge_rhs(Q, EPS0)
        r1 = g.fmg(1e-9, 30)
        r2 = g.solve(1e-11, 30)
        r3 = g.vcycles(2)
        out.append((r1, r2, r3, g.download(p.PHI)))
        g.close()
    a1, a2, a3, pa = out[0]
    for b1, b2, b3, pb in out[1:]:
        assert a1[2] == b1[2] and a2[2] == b2[2]
        assert a1[1] == b1[1] and a2[1] == b2[1] and a3 == b3
        assert np.array_equal(pa, pb)


def test_persistent_barrier_wait_is_bounded():
    """A persistent launch whose grid barriers cannot complete (every wait
    expects one block more than the grid) ends by itself within seconds with
    SM_ETIMEOUT; afterwards the same context solves normally."""
    import time
    dom, st = synth.workload("streamer_small")
    p = pkg()
    g = gpu_mesh(dom, st)
    t = g.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    g.upload(p.NE, ne); g.upload(p.NI, ni)
    g.charge_rhs(Q, EPS0)
    t0 = time.perf_counter()
    rc = g.persist_barrier_selftest()
    waited = time.perf_counter() - t0
    print("barrier self-test: status %d after %.2f s" % (rc, waited))
    assert rc == p.SM_ETIMEOUT and waited < 30.0
    for persist in (True, False):
        g.set_persistent(persist)
        rc, rel, cyc = g.fmg(1e-9, 30)
        assert rc == 0 and rel <= 1e-9
    g.close()


def test_repeated_graph_launch_and_launch_count():
    dom, st, o, g = pair("streamer_small")
    load_inputs(dom, st, o, g)
    n0 = g.launch_count()
    r1 = g.fmg(1e-8, 30)
    n1 = g.launch_count()
    r2 = g.fmg(1e-8, 30)       # second launch of the cached graph
    n2 = g.launch_count()
    assert r1[:3] == r2[:3]
    assert n2 - n1 == n1 - n0 - 1  # first call also built the level-0 basis
    # two fused red-black sweeps per level and repetition, integer arithmetic only
    us, n, by, fl = g.kernel_bench(0, 3)
    assert us > 0 and n == 3 * 2 * (g.n_levels - 1) and by > 0 and fl == 0
    us, n, by, fl = g.kernel_bench(1, 3)
    assert us > 0 and n == 3 and by > 0 and fl > 0
    us2, n2, by2, fl2 = g.kernel_bench(2, 3)
    assert us2 > 0 and n2 == 3 and by2 == by and fl2 == fl


def test_boundary_layout_ghosts_and_wrappers():
    """The layout call, the ghost-range fill and its readable result, and
    the wrappers sm_refine / sm_advance_fluid_coeffs: the stored
    interpolation value of every refinement-face ghost equals
    c/2 + c_t1/4 + c_t2/4 of the coarse cell c containing the ghost and its
    two tangential neighbours on the ghost's side (Sec. 2.1.1), formed here
    in numpy from the downloaded potential."""
    import ctypes as C
    dom, st, o, g = pair("streamer_small")
    t = o.tables()
    load_inputs(dom, st, o, g, t)
    o.fmg(1e-8, 30)
    g.fmg(1e-8, 30)
    p = pkg()
    ptr, ld, nb = g.var_layout(p.PHI)
    assert ld == 512 and nb == g.n_boxes and ptr == g.var(p.PHI).data_ptr()
    L = int(t["level"].max()) + 1
    g.fill_ghosts_range(1, L - 1)
    gh = g.ghosts()
    phi = g.download(p.PHI)
    where = {(int(l), *map(int, c)): b for b, (l, c) in enumerate(zip(t["level"], t["ijk"]))}

    def val(l, G):
        b = where.get((l, G[0] // 8, G[1] // 8, G[2] // 8))
        if b is None:
            return None
        return phi[b, (G[0] % 8) + 8 * (G[1] % 8) + 64 * (G[2] % 8)]

    checked = 0
    for b in range(g.n_boxes):
        l = int(t["level"][b])
        if l == 0:
            continue
        for f in range(6):
            a, side = f >> 1, f & 1
            nbpos = list(t["ijk"][b])
            nbpos[a] += 1 if side else -1
            if (l, *nbpos) in where or not all(0 <= x < 2 ** l for x in nbpos):
                continue  # same-level neighbour or domain wall
            t1, t2 = (a + 1) % 3, (a + 2) % 3
            for w in range(8):
                for u in range(8):
                    cg = [0, 0, 0]
                    cg[a], cg[t1], cg[t2] = (8 if side else -1), u, w
                    G = [8 * int(t["ijk"][b][d]) + cg[d] for d in range(3)]
                    cc = [x >> 1 for x in G]
                    vals = [val(l - 1, cc)]
                    for e in (t1, t2):
                        q = list(cc)
                        q[e] += 1 if G[e] & 1 else -1
                        vals.append(val(l - 1, q))
                    if any(v is None for v in vals):
                        continue  # a tangential neighbour across a wall
                    ref = 0.5 * vals[0] + 0.25 * vals[1] + 0.25 * vals[2]
                    assert gh[b, f, u + 8 * w] == pytest.approx(ref, rel=1e-14, abs=1e-14 * np.abs(phi).max())
                    checked += 1
    assert checked > 1000
    # the wrappers: sm_refine with no flags set changes nothing
    nbox = C.c_int()
    flags = np.zeros(g.n_boxes, np.int8)
    assert g._lib.sm_refine(g._h, flags.ctypes.data, C.byref(nbox)) == 0 and nbox.value == g.n_boxes
    g.compute_field()
    o.compute_field()
    dt = o.dt_limit(Q, EPS0)

    class Coeffs(C.Structure):
        _fields_ = [("q", C.c_double), ("eps", C.c_double), ("tol", C.c_double), ("max_cycles", C.c_int)]
    cf = Coeffs(Q, EPS0, 1e-8, 40)
    dtn, cyc = C.c_double(), (C.c_int * 2)()
    assert g._lib.sm_advance_fluid_coeffs(g._h, dt, C.byref(cf), C.byref(dtn), cyc) == 0
    ro = o.advance(dt, Q, EPS0, 1e-8, 40)
    assert (cyc[0], cyc[1]) == tuple(ro[2:])
    assert dtn.value == pytest.approx(ro[1], rel=TOL)


def test_repeatable_bits_full_size_streamer6():
    """Blocks of one launch never read what another block of it writes: the
    same solves on fresh solvers give the same bits, on the captured graphs
    and on the host loop, with and without programmatic dependent launch
    and with the persistent kernel (FMG, one more V-cycle, a warm-started
    solve to 1e-11; 2.4e6 leaf cells, where every level is one partial wave
    of blocks)."""
    dom, st = synth.workload("streamer6")
    p = __import__("paper_1708_08434_gb300")
    runs = []
    for graphs, pdl, persist in ((True, True, False), (True, True, False), (False, True, False),
                                 (False, False, False), (True, True, True)):
        g = gpu_mesh(dom, st, max_boxes=8192)
        t = g.tables()
        ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
        g.upload(p.NE, ne)
        g.upload(p.NI, ni)
        g.charge_rhs(Q, EPS0)
        g.set_graphs(graphs)
        g.set_pdl(pdl)
        g.set_persistent(persist)
        out = [g.fmg(1e-30, 1)[2]]
        out.append(g.download(p.PHI).view(np.int64).copy())
        g.vcycles(1)
        out.append(g.download(p.PHI).view(np.int64).copy())
        out.append(g.solve(1e-11, 30)[2])
        out.append(g.download(p.PHI).view(np.int64).copy())
        runs.append(out)
        g.close()
    for r in runs[1:]:
        assert r[0] == runs[0][0] and r[3] == runs[0][3]
        for k in (1, 2, 4):
            assert np.array_equal(r[k], runs[0][k]), k


def test_repeatable_bits_heun_step_fp64_and_mixed():
    """An FMG solve, the field, the time step and a Heun step (two Euler
    stages, two warm-started solves) on streamer6 give the same bits on two
    fresh solvers, for the FP64 and the mixed-precision forms."""
    dom, st = synth.workload("streamer6")
    p = __import__("paper_1708_08434_gb300")
    for prec in (p.FP64, p.MIXED):
        runs = []
        for _ in range(2):
            g = gpu_mesh(dom, st, max_boxes=8192, precision=prec)
            t = g.tables()
            ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
            g.upload(p.NE, ne)
            g.upload(p.NI, ni)
            g.set_table(synth.coefficient_table())
            g.charge_rhs(Q, EPS0)
            c0 = g.fmg(1e-8, 30)[2]
            g.compute_field()
            dt = g.dt_limit(Q, EPS0)
            r = g.advance(dt, Q, EPS0, 1e-8, 30)
            runs.append((c0, r, [g.download(v).view(np.int64).copy() for v in (p.PHI, p.NE, p.NI, p.EMAG)]))
            g.close()
        assert runs[0][0] == runs[1][0] and runs[0][1] == runs[1][1], prec
        for a, b in zip(runs[0][2], runs[1][2]):
            assert np.array_equal(a, b), prec
