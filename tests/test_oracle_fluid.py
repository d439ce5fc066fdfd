"""Pins of the oracle's drift-diffusion-reaction step (Sec. 2.2-2.4: Eq. 2-3,
Koren flux Eq. 6-7, lookup table, refinement-boundary fluxes, Heun step,
time-step limits)."""
import numpy as np
import pytest

import oracle
import synth

Q, EPS0 = synth.E_CHARGE, synth.EPS0


def psi_paper(x):
    """Koren limiter as printed in Sec. 2.3 (division form)."""
    return max(0.0, min(1.0, (2.0 + x) / 6.0, x))


def koren_textbook(r):
    """Koren (1993) limiter phi(r) = max(0, min(2r, (1+2r)/3, 2))."""
    return max(0.0, min(2.0 * r, (1.0 + 2.0 * r) / 3.0, 2.0))


def test_koren_division_free_matches_paper_form():
    rng = np.random.default_rng(1)
    for a, b in rng.standard_normal((4000, 2)) * 10.0 ** rng.integers(-3, 4, (4000, 2)):
        want = psi_paper(a / b) * b
        assert oracle.koren(a, b) == pytest.approx(want, rel=1e-14, abs=1e-300)
    assert oracle.koren(1.0, 0.0) == 0.0 and oracle.koren(0.0, 0.0) == 0.0


def test_koren_is_textbook_limiter_in_reciprocal_variable():
    # psi(x) = x/2 * phi(1/x) for x > 0: the face value n_i + psi (n_{i+1}-n_i)
    # equals n_i + phi(r)/2 (n_i - n_{i-1}), r = (n_{i+1}-n_i)/(n_i-n_{i-1})
    for x in np.linspace(0.01, 10.0, 997):
        assert oracle.koren(x, 1.0) == pytest.approx(0.5 * x * koren_textbook(1.0 / x), rel=1e-14)


def test_koren_linear_profile_gives_midpoint():
    for slope in (0.3, -2.0, 7.5):
        assert oracle.koren(slope, slope) == pytest.approx(0.5 * slope, rel=1e-15)


def table_oracle(dom, st=None, alpha=None):
    o = oracle.build_mesh(dom, st)
    tab = synth.coefficient_table()
    if alpha is not None:
        tab["alpha"] = np.full_like(tab["alpha"], alpha)
    o.set_table(tab)
    return o, tab


def test_lookup_table_interpolation():
    dom = synth.domain_uniform_cube(16)
    o, tab = table_oracle(dom)
    E = tab["E"]
    for k in (0, 1, 500, 998, 999):
        assert o.lookup(2, E[k]) == tab["alpha"][k]
    for k in (3, 200, 777):
        mid = 0.5 * (E[k] + E[k + 1])
        assert o.lookup(2, mid) == pytest.approx(0.5 * (tab["alpha"][k] + tab["alpha"][k + 1]), rel=1e-13)
    assert o.lookup(2, 40e6) == tab["alpha"][-1] and o.lookup(2, -1.0) == tab["alpha"][0]
    # interpolation error bound against the closed form: dE^2/8 max|alpha''|
    Es = np.linspace(1e5, 35e6, 5001)
    dE = E[1] - E[0]
    a = synth.alpha_closed(Es)
    a2 = np.abs(np.gradient(np.gradient(synth.alpha_closed(np.linspace(1e5, 35e6, 200001)),
                                        35e6 / 200000), 35e6 / 200000)).max()
    err = max(abs(o.lookup(2, e) - av) for e, av in zip(Es, a))
    assert err <= 1.05 * dE ** 2 / 8 * a2


def plate_setup(name, voltage, alpha=0.0, n=1e6):
    dom, st = synth.workload(name)
    dom.bc_val = (0.0, 0.0, 0.0, 0.0, 0.0, voltage)
    o, tab = table_oracle(dom, st, alpha)
    nb = o.n_boxes
    o.set(oracle.NE, np.full((nb, 512), n))
    o.set(oracle.NI, np.full((nb, 512), n))
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-12, 40)
    o.compute_field()
    return dom, o, tab


@pytest.mark.parametrize("name", ["uniform32", "streamer_small"])
def test_uniform_density_in_uniform_field_is_steady(name):
    dom, o, tab = plate_setup(name, 1e4)
    leaf = o.tables()["child"][:, 0] < 0
    em = o.get(oracle.EMAG)[leaf]
    assert np.allclose(em, 1e4 / dom.length, rtol=1e-10)
    dt = o.dt_limit(Q, EPS0)
    o.fluid_stage(dt)
    ne = o.get(oracle.NE)[leaf]
    assert np.max(np.abs(ne / 1e6 - 1.0)) <= 1e-12


def leaf_volume(dom, o):
    t = o.tables()
    leaf = t["child"][:, 0] < 0
    h = dom.length / (8.0 * 2.0 ** t["level"])
    return leaf, h ** 3


def test_mass_conservation_across_refinement():
    """Advection + diffusion, no source, density zero at the walls: the
    total sum of n*volume over leaves is conserved (coarse flux at a
    refinement boundary = mean of the fine fluxes, Sec. 2.3)."""
    dom, st = synth.workload("streamer_small")
    o, tab = table_oracle(dom, st, alpha=0.0)
    t = o.tables()
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    # the synthetic channel reaches the top electrode; cut it at 12 mm so
    # that no density (hence no flux) touches a wall
    _, _, z = synth.cell_centres(dom, t["level"], t["ijk"])
    ne, ni = ne * (z < 12e-3), ni * (z < 12e-3)
    o.set(oracle.NE, ne)
    o.set(oracle.NI, ni)
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-10, 40)
    o.compute_field()
    leaf, vol = leaf_volume(dom, o)
    m0 = np.sum(o.get(oracle.NE)[leaf] * vol[leaf, None])
    dt = o.dt_limit(Q, EPS0)
    for _ in range(3):
        o.fluid_stage(dt)
    m1 = np.sum(o.get(oracle.NE)[leaf] * vol[leaf, None])
    assert m1 == pytest.approx(m0, rel=1e-14)
    # the step did move electrons
    assert np.max(np.abs(o.get(oracle.NE)[leaf] - ne[leaf])) > 1e-3 * ne.max()


def test_diffusion_maximum_principle():
    dom, o, tab = plate_setup("uniform32", 0.0)
    rng = np.random.default_rng(3)
    n0 = rng.uniform(1.0, 2.0, (o.n_boxes, 512))
    o.set(oracle.NE, n0)
    dt = o.dt_limit(Q, EPS0)
    o.fluid_stage(dt)
    lo, hi = o.level_range(o.n_levels - 1)
    n1 = o.get(oracle.NE)[lo:hi]
    assert n1.min() >= n0[lo:hi].min() - 1e-14 and n1.max() <= n0[lo:hi].max() + 1e-14
    assert np.std(n1) < np.std(n0[lo:hi])


def test_dt_limits_hand_computed():
    """Uniform field V/L and uniform n_e: the three limits of Sec. 2.4."""
    V, n = 2e4, 1e17
    dom, o, tab = plate_setup("uniform32", V, n=n)
    h = dom.h(o.n_levels - 1)
    E = V / dom.length
    adv = synth.MOBILITY * E / h
    ad = adv + 6.0 * synth.DIFFUSION / h ** 2
    drt = EPS0 / (Q * synth.MOBILITY * n)
    want = 0.9 * min(0.5 / adv, 1.0 / ad, drt)
    assert o.dt_limit(Q, EPS0) == pytest.approx(want, rel=1e-12)


def test_heun_growth_closed_form():
    """Source only (uniform tiny n, uniform field, constant alpha): one Heun
    step multiplies n by 1 + a + a^2/2, a = alpha mu E dt (Sec. 2.4)."""
    V, alpha = 1e4, 40.0
    dom, o, tab = plate_setup("uniform32", V, alpha=alpha)
    E = V / dom.length
    dt = 1e-3 / (alpha * synth.MOBILITY * E) * 50
    st, dtn, c1, c2 = o.advance(dt, Q, EPS0, tol=1e-10)
    a = alpha * synth.MOBILITY * E * dt
    lo, hi = o.level_range(o.n_levels - 1)
    ne = o.get(oracle.NE)[lo:hi]
    ni = o.get(oracle.NI)[lo:hi]
    g = 1.0 + a + 0.5 * a * a
    assert np.max(np.abs(ne / 1e6 / g - 1.0)) <= 1e-12
    assert np.max(np.abs(ni / 1e6 / g - 1.0)) <= 1e-12


def test_density_step_moves_by_first_order_upwind():
    """The Koren-limited upwind face value (Eq. 6-7) reduces to first-order
    upwinding at a discontinuity, where the limiter vanishes (a slope is
    zero or changes sign).  A step n_e = 1 below z = L/2, 0 above, in a
    uniform field with no diffusion and no source, after one Euler stage:
    the first cell above the step holds exactly v dt / h and every other
    cell is unchanged (electrons drift against E, here towards +z)."""
    V = 1e4
    dom, o, tab = plate_setup("uniform32", V)      # uniform field, no charge
    tab = dict(tab, diff=np.zeros_like(tab["diff"]))
    o.set_table(tab)
    t = o.tables()
    _, _, z = synth.cell_centres(dom, t["level"], t["ijk"])
    n0 = (z < 0.5 * dom.length).astype(np.float64)
    o.set(oracle.NE, n0)
    o.set(oracle.NI, np.zeros_like(n0))
    h = dom.h(o.n_levels - 1)
    v = synth.MOBILITY * V / dom.length
    dt = 0.25 * h / v
    o.fluid_stage(dt)
    lo, hi = o.level_range(o.n_levels - 1)
    zl = z[lo:hi]
    first = (zl > 0.5 * dom.length) & (zl < 0.5 * dom.length + h)
    want = n0[lo:hi].copy()
    want[first] = 0.25
    assert first.sum() == 32 * 32
    assert np.max(np.abs(o.get(oracle.NE)[lo:hi] - want)) <= 1e-13


def test_field_exact_on_quadratic_potential():
    """The cell field (Sec. 2.3) is the mean of each axis's two face fields,
    a centred difference, exact on quadratics: for phi = a (z - zc)^2 +
    b (x - xc)^2 the interior cells get |E| = hypot(2 b (x - xc),
    2 a (z - zc)) to rounding."""
    dom = synth.workload("uniform32")[0]
    o = oracle.build_mesh(dom)
    t = o.tables()
    x, y, z = synth.cell_centres(dom, t["level"], t["ijk"])
    a, b, xc, zc = 3.0, -1.5, 0.37, 0.61
    o.set(oracle.PHI, a * (z - zc) ** 2 + b * (x - xc) ** 2)
    o.compute_field()
    lo, hi = o.level_range(o.n_levels - 1)
    h = dom.h(o.n_levels - 1)
    n = int(round(dom.length / h))
    inner = np.ones((hi - lo, 512), bool)
    for c in (x, y, z):
        i = np.floor(c[lo:hi] / h).astype(int)
        inner &= (i >= 1) & (i <= n - 2)
    want = np.hypot(2 * b * (x[lo:hi] - xc), 2 * a * (z[lo:hi] - zc))
    got = o.get(oracle.EMAG)[lo:hi]
    assert inner.sum() == (n - 2) ** 3
    assert np.max(np.abs(got[inner] - want[inner])) <= 1e-12 * np.max(want)


def test_dt_diffusion_limit_without_field():
    """No field: the advection terms vanish and, with a tiny n_e, Sec. 2.4's
    limit is the diffusion one, dt = 0.9 h^2 / (6 D) in three dimensions."""
    dom, o, tab = plate_setup("uniform32", 0.0, n=1e6)
    h = dom.h(o.n_levels - 1)
    assert o.dt_limit(Q, EPS0) == pytest.approx(0.9 * h ** 2 / (6.0 * synth.DIFFUSION), rel=1e-12)
