"""Pins of the 2-D / axisymmetric oracle (quadtree of 8^2-cell boxes;
Sec. 1 and 2.1.1 support 2-D, axisymmetric and 3-D runs): tables by brute
force, the level-0 solve against closed-form eigenvectors, the cylindrical
operator exact on r^2, linear exactness across refinement boundaries,
second-order convergence to continuum solutions in both geometries, the
FAS fixed point against a sparse direct solve, conservation of the
restriction and of the fluid step, closed-form Heun growth."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import quad

N, D = synth.NEUMANN, synth.DIRICHLET
AXI, CART = synth.AXISYMMETRIC, synth.CARTESIAN
Q, EPS0 = synth.E_CHARGE, synth.EPS0


def morton2_bits(i, j, bits=31):
    key = 0
    for b in range(bits):
        key |= ((i >> b) & 1) << (2 * b)
        key |= ((j >> b) & 1) << (2 * b + 1)
    return key


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_tables_brute_force(name):
    dom, st = synth.workload2(name)
    o = quad.build_mesh(dom, st)
    t = o.tables()
    n = o.n_boxes
    pos = {(int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])): b for b in range(n)}
    assert len(pos) == n
    # sorted by (level, Morton key); keys by an independent bit loop
    keys = [(int(t["level"][b]), morton2_bits(int(t["ij"][b, 0]), int(t["ij"][b, 1]))) for b in range(n)]
    assert keys == sorted(keys)
    assert all(int(t["morton"][b]) == keys[b][1] for b in range(n))
    for b in range(n):
        l, i, j = int(t["level"][b]), int(t["ij"][b, 0]), int(t["ij"][b, 1])
        par = t["parent"][b]
        assert (l == 0 and par == -1) or pos[(l - 1, i >> 1, j >> 1)] == par
        for c in range(4):
            ch = t["child"][b, c]
            key = (l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))
            assert (ch == -1 and key not in pos) or (ch >= 0 and pos[key] == ch)
        d = 0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == 0 and dy == 0:
                    continue
                ii, jj = i + dx, j + dy
                want = -1 if not (0 <= ii < (1 << l) and 0 <= jj < (1 << l)) else pos.get((l, ii, jj), -2)
                assert t["nbr"][b, d] == want
                d += 1
    # proper nesting: a request whose neighbourhood is not covered is dropped
    o2 = quad.Quad(synth.Domain2(1.0, 2, 2, CART))
    f = np.zeros(4, np.int8)
    f[0] = 1
    assert o2.refine_level(1, f) == 4
    f2 = np.zeros(4, np.int8)
    f2[3] = 1          # box (1,1) of level 2 touches uncovered level-2 positions
    assert o2.refine_level(2, f2) == 0 and o2.dropped == 1


def eig1d(kind, n, p, idx):
    """Eigenvector of the 1-D cell-centred 3-point operator (ghost = inner
    for Neumann, -inner for Dirichlet-0) and its eigenvalue times h^2."""
    t = idx + 0.5
    if kind == "NN":
        return np.cos(np.pi * p * t / n), -4 * np.sin(np.pi * p / (2 * n)) ** 2
    if kind == "DD":
        return np.sin(np.pi * p * t / n), -4 * np.sin(np.pi * p / (2 * n)) ** 2
    return np.sin(np.pi * (p + 0.5) * t / n), -4 * np.sin(np.pi * (p + 0.5) / (2 * n)) ** 2


BCT = {"NN": (N, N), "DD": (D, D), "DN": (D, N)}


@pytest.mark.parametrize("kinds,modes", [(("NN", "DD"), (1, 2)), (("DD", "DN"), (3, 0)),
                                         (("DN", "NN"), (2, 5))])
def test_single_box_exact_solve_eigenvector(kinds, modes):
    dom = synth.Domain2(1.0, 1, 0, CART, bc_type=BCT[kinds[0]] + BCT[kinds[1]], bc_val=(0.0,) * 4)
    o = quad.Quad(dom)
    t = o.tables()
    x, y = synth.cell_centres2(dom, t["level"], t["ij"])
    h = 1.0 / 8
    v, lam = np.ones_like(x), 0.0
    for a, c in enumerate((x, y)):
        va, la = eig1d(kinds[a], 8, modes[a], np.rint(c / h - 0.5))
        v, lam = v * va, lam + la / h ** 2
    o.set(quad.RHO, -lam * v)
    o.charge_rhs(1.0, 1.0, True)
    o.coarse_solve()
    assert np.max(np.abs(o.get(quad.PHI) - v)) <= 1e-12 * np.max(np.abs(v))


def test_axisymmetric_operator_exact_on_r_squared():
    """The finite-volume operator (1/r) d/dr (r d/dr) is exact on phi = r^2
    (L phi = 4 in every cell not touching the outer radial wall, the axis
    cells included), on every uniform level."""
    dom = synth.Domain2(1.0, 4, 0, AXI, bc_type=(N, N, N, N), bc_val=(0.0,) * 4)
    o = quad.Quad(dom)
    t = o.tables()
    x, _ = synth.cell_centres2(dom, t["level"], t["ij"])
    o.set(quad.PHI, x ** 2)
    o.set(quad.RHO, np.full_like(x, -4.0))
    o.charge_rhs(1.0, 1.0, True)                   # f = 4
    r = o.composite_residual()
    lo, hi = o.level_range(o.n_levels - 1)
    h = dom.h(o.n_levels - 1)
    inner = x[lo:hi] < 1.0 - h
    assert np.max(np.abs(r[lo:hi][inner])) <= 1e-11
    # the outer wall cells see the Neumann ghost (no outward face flux)
    assert np.min(np.abs(r[lo:hi][~inner])) > 1.0


def test_axisymmetric_coarse_solve_inverts_operator():
    dom = synth.Domain2(1.0, 1, 0, AXI, bc_type=(N, D, D, N), bc_val=(0.0,) * 4)
    o = quad.Quad(dom)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((1, 64))
    o.set(quad.RHO, np.zeros((1, 64)))
    o.charge_rhs(1.0, 1.0, True)
    o.set(quad.PHI, phi)
    lphi = -o.composite_residual()                 # f = 0: r = -L phi
    o.set(quad.RHO, -lphi)
    o.charge_rhs(1.0, 1.0, True)
    o.set(quad.PHI, np.zeros((1, 64)))
    o.coarse_solve()
    assert np.max(np.abs(o.get(quad.PHI) - phi)) <= 1e-12 * np.max(np.abs(phi))


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_plate_gap_linear_exact(name):
    """phi = V z / L with no charge is reproduced to roundoff across the
    refinement boundaries (linear-exact ghosts, restriction, prolongation)."""
    dom, st = synth.workload2(name)
    o = quad.build_mesh(dom, st)
    t = o.tables()
    _, y = synth.cell_centres2(dom, t["level"], t["ij"])
    exact = dom.bc_val[3] * y / dom.length
    o.set(quad.RHO, np.zeros_like(exact))
    o.charge_rhs(1.0, 1.0, True)
    o.set(quad.PHI, exact)
    assert o.rel_residual() <= 1e-13
    leaf = t["child"][:, 0] < 0
    o.set(quad.PHI, np.zeros_like(exact))
    st_, rel, cyc = o.fmg(1e-13, 40)
    assert np.max(np.abs(o.get(quad.PHI)[leaf] - exact[leaf])) <= 1e-11 * dom.bc_val[3]


@pytest.mark.parametrize("geom", [CART, AXI])
def test_second_order_convergence(geom):
    """phi* = z + exp(-rho^2/(2 sigma^2)), sigma = 0.05, on 64^2, 128^2 and
    256^2 cells: the max error falls by >= 3.7 per halving of h (second
    order; wrong cylindrical weights or a first-order rule give about 2 or
    no convergence)."""
    errs = []
    for nb in (8, 16, 32):
        dom = synth.Domain2(1.0, nb, 0, geom)
        o = quad.Quad(dom)
        t = o.tables()
        phi_star, rho = synth.manufactured_gaussian2(dom, t["level"], t["ij"])
        o.set(quad.RHO, rho)
        o.charge_rhs(1.0, 1.0, True)
        st, rel, cyc = o.fmg(1e-12, 40)
        assert st == 0
        lo, hi = o.level_range(o.n_levels - 1)
        errs.append(np.max(np.abs(o.get(quad.PHI)[lo:hi] - phi_star[lo:hi])))
    assert errs[0] / errs[1] >= 3.7 and errs[1] / errs[2] >= 3.7, errs


def tiny_amr(geom):
    dom = synth.Domain2(1.0, 2, 1, geom, bc_val=(0.0,) * 4)
    o = quad.Quad(dom)
    f = np.zeros(4, np.int8)
    f[0] = 1                                       # the box on the axis
    assert o.refine_level(1, f) == 4
    return dom, o


@pytest.mark.parametrize("geom", [CART, AXI])
def test_fixed_point_is_composite_direct_solve(geom):
    """The FAS V-cycle fixed point equals the sparse direct solve of the
    composite leaf operator (columns from unit vectors)."""
    dom, o = tiny_amr(geom)
    t = o.tables()
    leaf = np.where(t["child"][:, 0] < 0)[0]
    nbox, n = o.n_boxes, len(leaf) * 64
    o.set(quad.RHO, np.zeros((nbox, 64)))
    o.charge_rhs(1.0, 1.0, True)
    rows, cols, vals = [], [], []
    for col in range(n):
        phi = np.zeros((nbox, 64))
        phi[leaf[col // 64], col % 64] = 1.0
        o.set(quad.PHI, phi)
        r = -o.composite_residual()[leaf].ravel()
        nz = np.nonzero(r)[0]
        rows.extend(nz)
        cols.extend([col] * len(nz))
        vals.extend(r[nz])
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    f_leaf = np.random.default_rng(11).standard_normal(n)
    direct = spla.spsolve(A, f_leaf)
    rho = np.zeros((nbox, 64))
    rho[leaf] = -f_leaf.reshape(len(leaf), 64)
    o.set(quad.RHO, rho)
    o.charge_rhs(1.0, 1.0, True)
    o.set(quad.PHI, np.zeros((nbox, 64)))
    o.fmg(1e-14, 80)
    mg = o.get(quad.PHI)[leaf].ravel()
    assert np.max(np.abs(mg - direct)) <= 1e-11 * np.max(np.abs(direct))


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_vcycle_contracts(name):
    dom, st = synth.workload2(name)
    o = quad.build_mesh(dom, st)
    t = o.tables()
    ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
    o.set(quad.NE, ne)
    o.set(quad.NI, ni)
    o.charge_rhs(Q, EPS0)
    prev = 1.0
    for _ in range(5):
        r = o.vcycles(1)
        assert r < prev / 4
        prev = r


def leaf_volume(dom, o):
    """leaf mask and cell volumes (area in Cartesian, r dr dz in cylindrical)"""
    t = o.tables()
    leaf = t["child"][:, 0] < 0
    x, _ = synth.cell_centres2(dom, t["level"], t["ij"])
    h = dom.length / (8.0 * 2.0 ** t["level"])
    vol = h[:, None] ** 2 * (x if dom.geom == AXI else 1.0)
    return leaf, vol


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_restriction_conserves_content(name):
    """Every refined box holds the content (n times volume) of its children
    after restriction: volume-weighted in cylindrical coordinates."""
    dom, st = synth.workload2(name)
    o = quad.build_mesh(dom, st)
    t = o.tables()
    rng = np.random.default_rng(5)
    o.set(quad.NE, rng.random((o.n_boxes, 64)))
    o.restrict_all(quad.NE)
    n = o.get(quad.NE)
    _, vol = leaf_volume(dom, o)
    for b in np.where(t["child"][:, 0] >= 0)[0]:
        kids = t["child"][b]
        assert np.sum(n[b] * vol[b]) == pytest.approx(np.sum(n[kids] * vol[kids]), rel=1e-14)


def table_quad(dom, st, alpha=None):
    o = quad.build_mesh(dom, st)
    tab = synth.coefficient_table()
    if alpha is not None:
        tab["alpha"] = np.full_like(tab["alpha"], alpha)
    o.set_table(tab)
    return o


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_uniform_density_in_uniform_field_is_steady(name):
    dom, st = synth.workload2(name)
    o = table_quad(dom, st, alpha=0.0)
    nb = o.n_boxes
    o.set(quad.NE, np.full((nb, 64), 1e18))
    o.set(quad.NI, np.full((nb, 64), 1e18))
    o.set(quad.RHO, np.zeros((nb, 64)))
    o.charge_rhs(1.0, 1.0, True)
    o.fmg(1e-12, 40)
    o.compute_field()
    dt = o.dt_limit(Q, EPS0)
    o.fluid_stage(dt)
    leaf, _ = leaf_volume(dom, o)
    assert np.max(np.abs(o.get(quad.NE)[leaf] / 1e18 - 1.0)) <= 1e-12


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_mass_conservation_across_refinement(name):
    """Advection + diffusion, no source, no density at the walls: the total
    content over leaves is conserved (the coarse flux at a refinement
    boundary is the area-weighted mean of the fine fluxes)."""
    dom, st = synth.workload2(name)
    o = table_quad(dom, st, alpha=0.0)
    t = o.tables()
    ne, ni = synth.streamer_densities2(dom, st, t["level"], t["ij"])
    _, y = synth.cell_centres2(dom, t["level"], t["ij"])
    ne, ni = ne * (y < 12e-3), ni * (y < 12e-3)
    o.set(quad.NE, ne)
    o.set(quad.NI, ni)
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-10, 40)
    o.compute_field()
    leaf, vol = leaf_volume(dom, o)
    m0 = np.sum(o.get(quad.NE)[leaf] * vol[leaf])
    dt = o.dt_limit(Q, EPS0)
    for _ in range(3):
        o.fluid_stage(dt)
    m1 = np.sum(o.get(quad.NE)[leaf] * vol[leaf])
    assert m1 == pytest.approx(m0, rel=1e-13)
    assert np.max(np.abs(o.get(quad.NE)[leaf] - ne[leaf])) > 1e-3 * ne.max()


def test_dt_limits_hand_computed():
    """Uniform field V/L along z and uniform n_e on one uniform level:
    dt = 0.9 min(0.5 h/(mu E), 1/(mu E/h + 4D/h^2), eps0/(e mu n_e))."""
    V, L = 1e4, 0.016
    dom = synth.Domain2(L, 4, 0, AXI, bc_val=(0.0, 0.0, 0.0, V))
    o = table_quad(dom, None)
    nb = o.n_boxes
    n = 1e14
    o.set(quad.NE, np.full((nb, 64), n))
    o.set(quad.RHO, np.zeros((nb, 64)))
    o.charge_rhs(1.0, 1.0, True)
    o.fmg(1e-13, 40)
    o.compute_field()
    h = dom.h(o.n_levels - 1)
    E = V / L
    adv = synth.MOBILITY * E / h
    ad = adv + 4.0 * synth.DIFFUSION / h ** 2
    drt = EPS0 / (Q * synth.MOBILITY * n)
    want = 0.9 * min(0.5 / adv, 1.0 / ad, drt)
    assert o.dt_limit(Q, EPS0) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("geom", [CART, AXI])
def test_heun_growth_closed_form(geom):
    """Uniform field and densities, constant alpha: one Heun step multiplies
    n_e by 1 + a + a^2/2, a = alpha mu E dt (the field does not change: the
    charge stays uniform and neutral)."""
    V, L, alpha = 1e4, 0.016, 2e3
    dom = synth.Domain2(L, 2, 0, geom, bc_val=(0.0, 0.0, 0.0, V))
    o = table_quad(dom, None, alpha=alpha)
    nb = o.n_boxes
    o.set(quad.NE, np.full((nb, 64), 1e12))
    o.set(quad.NI, np.full((nb, 64), 1e12))
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-13, 40)
    o.compute_field()
    E = V / L
    dt = 1e-3 / (alpha * synth.MOBILITY * E) * 50
    st, dtn, c1, c2 = o.advance(dt, Q, EPS0, 1e-12, 40)
    a = alpha * synth.MOBILITY * E * dt
    lo, hi = o.level_range(o.n_levels - 1)
    got = o.get(quad.NE)[lo:hi] / 1e12
    assert np.max(np.abs(got - (1 + a + a * a / 2))) <= 1e-9


def test_koren_matches_paper_form_and_textbook_limiter():
    """The 2-D oracle's limiter: psi(a/b) b with psi as printed in Sec. 2.3
    (division form), the textbook Koren limiter in the reciprocal variable,
    and the midpoint on linear data."""
    from test_oracle_fluid import koren_textbook, psi_paper
    rng = np.random.default_rng(2)
    for a, b in rng.standard_normal((2000, 2)) * 10.0 ** rng.integers(-3, 4, (2000, 2)):
        assert quad.koren(a, b) == pytest.approx(psi_paper(a / b) * b, rel=1e-14, abs=1e-300)
    assert quad.koren(1.0, 0.0) == 0.0 and quad.koren(0.0, 0.0) == 0.0
    for x in np.linspace(0.01, 10.0, 499):
        assert quad.koren(x, 1.0) == pytest.approx(0.5 * x * koren_textbook(1.0 / x), rel=1e-14)
    for slope in (0.3, -2.0, 7.5):
        assert quad.koren(slope, slope) == pytest.approx(0.5 * slope, rel=1e-15)


def uniform_quad(geom, V, alpha=0.0, diff=None):
    """One uniform level of 32^2 cells, phi = 0 / V on the z faces, a
    neutral uniform charge (so the field is V/L along z), the coefficient
    table with the given alpha (and D when given)."""
    L = 0.016
    dom = synth.Domain2(L, 4, 0, geom, bc_val=(0.0, 0.0, 0.0, V))
    o = table_quad(dom, None, alpha=alpha)
    if diff is not None:
        tab = synth.coefficient_table()
        tab["alpha"] = np.full_like(tab["alpha"], alpha)
        tab["diff"] = np.full_like(tab["diff"], diff)
        o.set_table(tab)
    nb = o.n_boxes
    o.set(quad.NE, np.full((nb, 64), 1e10))
    o.set(quad.NI, np.full((nb, 64), 1e10))
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-13, 40)
    o.compute_field()
    return dom, o


@pytest.mark.parametrize("geom", [CART, AXI])
def test_density_step_moves_by_first_order_upwind(geom):
    """Koren upwinding reduces to first-order upwinding at a discontinuity
    (the limiter vanishes there): a step n_e = 1 below z = L/2, 0 above, in
    a uniform field along z with no diffusion and no source puts exactly
    v dt / h into the first cell above the step after one Euler stage and
    leaves every other cell unchanged (the axial fluxes carry no radial
    weight)."""
    V = 1e4
    dom, o = uniform_quad(geom, V, diff=0.0)
    t = o.tables()
    _, z = synth.cell_centres2(dom, t["level"], t["ij"])
    n0 = (z < 0.5 * dom.length).astype(np.float64)
    o.set(quad.NE, n0)
    o.set(quad.NI, np.zeros_like(n0))
    h = dom.h(o.n_levels - 1)
    v = synth.MOBILITY * V / dom.length
    o.fluid_stage(0.25 * h / v)
    lo, hi = o.level_range(o.n_levels - 1)
    zl = z[lo:hi]
    first = (zl > 0.5 * dom.length) & (zl < 0.5 * dom.length + h)
    want = n0[lo:hi].copy()
    want[first] = 0.25
    assert first.sum() == 32
    assert np.max(np.abs(o.get(quad.NE)[lo:hi] - want)) <= 1e-13


def test_dt_diffusion_limit_without_field():
    """No field: the advection terms vanish and, with a tiny n_e, Sec. 2.4's
    limit is the diffusion one, dt = 0.9 h^2 / (4 D) in two dimensions."""
    dom, o = uniform_quad(AXI, 0.0)
    h = dom.h(o.n_levels - 1)
    assert o.dt_limit(Q, EPS0) == pytest.approx(0.9 * h ** 2 / (4.0 * synth.DIFFUSION), rel=1e-12)


@pytest.mark.parametrize("geom", [CART, AXI])
def test_field_exact_on_quadratic_potential(geom):
    """The cell field is the mean of each axis's two face fields, a centred
    difference, exact on quadratics in both geometries: phi = a (z - zc)^2
    + b (x - xc)^2 gives |E| = hypot(2 b (x - xc), 2 a (z - zc)) in the
    interior cells."""
    dom, o = uniform_quad(geom, 0.0)
    t = o.tables()
    x, z = synth.cell_centres2(dom, t["level"], t["ij"])
    L = dom.length
    a, b, xc, zc = 3.0 / L, -1.5 / L, 0.37 * L, 0.61 * L
    o.set(quad.PHI, a * (z - zc) ** 2 + b * (x - xc) ** 2)
    o.compute_field()
    lo, hi = o.level_range(o.n_levels - 1)
    h = dom.h(o.n_levels - 1)
    n = int(round(L / h))
    inner = np.ones((hi - lo, 64), bool)
    for c in (x, z):
        i = np.floor(c[lo:hi] / h).astype(int)
        inner &= (i >= 1) & (i <= n - 2)
    want = np.hypot(2 * b * (x[lo:hi] - xc), 2 * a * (z[lo:hi] - zc))
    got = o.get(quad.EMAG)[lo:hi]
    assert inner.sum() == (n - 2) ** 2
    assert np.max(np.abs(got[inner] - want[inner])) <= 1e-12 * np.max(want)


@pytest.mark.parametrize("name", ["axi_small", "cart_small"])
def test_fmg_does_not_depend_on_the_starting_potential(name):
    """Each finer level of the FMG ladder starts from the interpolated coarse
    solution, replacing what it held: a random starting potential gives
    the same bits as zero."""
    dom, st = synth.workload2(name)
    out = []
    for seed in (None, 5):
        o = quad.build_mesh(dom, st)
        nb = o.n_boxes
        o.set(quad.RHO, np.random.default_rng(9).standard_normal((nb, 64)))
        o.charge_rhs(1.0, 1.0, True)
        o.set(quad.PHI, np.zeros((nb, 64)) if seed is None else np.random.default_rng(seed).standard_normal((nb, 64)))
        o.fmg(1e-10, 40)
        out.append(o.get(quad.PHI))
    assert np.array_equal(out[0], out[1])
