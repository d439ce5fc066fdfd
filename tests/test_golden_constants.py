"""The constants the paper fixes (tests/golden/paper_constants.txt, each line
with its section) are the ones the oracle, the GPU binding and the
benchmark use: the refinement-criterion defaults of Eq. 8, the box size,
the V-cycles of the paper's schedule and the three time-step limits of
Sec. 2.4, the last checked through the oracle's time step on a state whose
limits have a closed form."""
import inspect
import os
import re

import numpy as np
import pytest

import oracle
import synth
from helpers import EPS0, Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            assert cite.startswith("Sec. "), line
            out[name] = float(value)
    return out


def test_fixture_lists_every_constant():
    g = golden()
    assert set(g) == {"cfl_number", "adv_diff_bound", "dt_safety", "refine_c0", "refine_c1",
                      "refine_buffer", "deref_c0", "deref_dx", "box_cells_per_side",
                      "vcycles_per_update"}


def test_refinement_defaults_are_the_papers():
    import oracle.quad as quad
    import paper_1708_08434_gb300 as pkg
    g = golden()
    want = {"c0": g["refine_c0"], "c1": g["refine_c1"], "c0_deref": g["deref_c0"],
            "dx_deref": g["deref_dx"], "buffer": g["refine_buffer"]}
    for cls in (oracle.Oracle, quad.Quad, pkg.Solver, pkg.Quad):
        params = inspect.signature(cls.refine_flags).parameters
        got = {k: params[k].default for k in want}
        assert got == pytest.approx(want), cls


def test_box_size_and_schedule_are_the_papers():
    import bench
    g = golden()
    n = int(g["box_cells_per_side"])
    hdr = open(os.path.join(ROOT, "include", "sm_streamer.h")).read()
    assert int(re.search(r"#define SM_BOX (\d+)", hdr).group(1)) == n
    for src in ("oracle.c", "quad.c"):
        text = open(os.path.join(ROOT, "oracle", src)).read()
        assert int(re.search(r"#define NC (\d+)", text).group(1)) == n, src
    assert bench.PAPER_VCYCLES == int(g["vcycles_per_update"])


@pytest.mark.parametrize("V, n, active", [(2e4, 1e6, 0), (1.0, 1e6, 1), (2e4, 1e17, 2)])
def test_time_step_limits_use_the_papers_constants(V, n, active):
    """Uniform field V/L and uniform n_e on the uniform 32^3 mesh (3-D): the
    advective rate mu E / dx, the advective-diffusive rate plus 2 D D_e /
    dx^2 with D = 3, and the dielectric relaxation time eps / (q mu n_e)
    give dt = safety x min(cfl / rate, bound / rate', t_drt).  The three
    states make each limit the active one in turn, so each constant
    decides a result."""
    g = golden()
    dom, st = synth.workload("uniform32")
    dom.bc_val = (0.0, 0.0, 0.0, 0.0, 0.0, V)
    o = oracle.build_mesh(dom, st)
    o.set_table(synth.coefficient_table())
    nb = o.n_boxes
    o.set(oracle.NE, np.full((nb, 512), n))
    o.set(oracle.NI, np.full((nb, 512), n))
    o.charge_rhs(Q, EPS0)
    o.fmg(1e-12, 40)
    o.compute_field()
    h = dom.h(o.n_levels - 1)
    E = V / dom.length
    adv = synth.MOBILITY * E / h
    adv_diff = adv + 2 * 3 * synth.DIFFUSION / h ** 2
    t_drt = EPS0 / (Q * synth.MOBILITY * n)
    limits = [g["cfl_number"] / adv, g["adv_diff_bound"] / adv_diff, t_drt]
    assert int(np.argmin(limits)) == active
    assert o.dt_limit(Q, EPS0) == pytest.approx(g["dt_safety"] * min(limits), rel=1e-12)
