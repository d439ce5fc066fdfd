"""The seeded input generators (no method arithmetic): the stochastic
background of the learned-form workload, in the manner of the paper's
Sec. 3.2 (case 3: 2U times the mean, drawn per coarse cell, linearly
interpolated to finer grids)."""
import numpy as np

import synth


def _bg_setup():
    dom, st = synth.workload("streamer_small_bg")
    return dom, st


def test_background_reproduces_the_coarse_draws_at_coarse_centres():
    dom, st = _bg_setup()
    n = int(round(dom.length / st.noise_cell))
    i = np.arange(n)
    xc = dom.origin[0] + (i + 0.5) * st.noise_cell
    # every coarse-cell centre of one line along x, at the centre row in y, z
    j = k = n // 2
    y = np.full(n, dom.origin[1] + (j + 0.5) * st.noise_cell)
    z = np.full(n, dom.origin[2] + (k + 0.5) * st.noise_cell)
    got = synth.background_density(dom, st, xc, y, z)
    u = synth.uniform01(synth.SEED, i.astype(np.uint64) + np.uint64(n * j) + np.uint64(n * n * k))
    assert np.allclose(got, 2.0 * st.background * u, rtol=1e-15, atol=0.0)


def test_background_is_seeded_bounded_linear_and_has_the_stated_mean():
    dom, st = _bg_setup()
    rng = np.random.default_rng(3)
    x, y, z = (dom.origin[0] + dom.length * rng.random(20000) for _ in range(3))
    a = synth.background_density(dom, st, x, y, z)
    b = synth.background_density(dom, st, x, y, z)
    assert np.array_equal(a, b)
    c = synth.background_density(dom, st, x, y, z, seed=synth.SEED + 1)
    assert not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 2.0 * st.background
    # E[2U] = 1: the mean over many points is the stated background
    assert abs(a.mean() / st.background - 1.0) < 0.05
    # linear between two neighbouring coarse centres along x
    n = int(round(dom.length / st.noise_cell))
    x0 = dom.origin[0] + 3.5 * st.noise_cell
    yy = np.full(5, dom.origin[1] + 7.5 * st.noise_cell)
    zz = np.full(5, dom.origin[2] + 9.5 * st.noise_cell)
    xs = x0 + st.noise_cell * np.linspace(0.0, 1.0, 5)
    v = synth.background_density(dom, st, xs, yy, zz)
    assert np.allclose(np.diff(v, 2), 0.0, atol=1e-6 * st.background)
    assert n == 32


def test_streamer_densities_carry_the_background_and_are_unchanged_without_it():
    dom, st = synth.workload("streamer_small_bg")
    dom0, st0 = synth.workload("streamer_small")
    levels = np.array([dom.lbase] * 2)
    ijk = np.array([[0, 0, 0], [1, 1, 1]])
    ne, ni = synth.streamer_densities(dom, st, levels, ijk)
    ne0, ni0 = synth.streamer_densities(dom0, st0, levels, ijk)
    x, y, z = synth.cell_centres(dom, levels, ijk)
    bg = synth.background_density(dom, st, x, y, z)
    assert np.array_equal(ne, ne0 + bg) and np.array_equal(ni, ni0 + bg)
    assert bg.min() > 0.0
