"""Shared helpers of the parity tests: the same synthetic mesh and inputs
on the CUDA library and on the CPU oracle."""
import numpy as np

import oracle
import synth

Q, EPS0 = synth.E_CHARGE, synth.EPS0


def gpu_mesh(dom, st=None, max_boxes=None, **kw):
    import paper_1708_08434_gb300 as pkg
    if max_boxes is None:
        max_boxes = 1 << 16
    g = pkg.Solver(dom, max_boxes, **kw)
    g.build_octree()
    if st is not None:
        synth.refine_all(dom, st, g.level_ijk, g.refine_level)
    return g


def pair(name, **kw):
    dom, st = synth.workload(name)
    return dom, st, oracle.build_mesh(dom, st), gpu_mesh(dom, st, **kw)


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def load_inputs(dom, st, o, g, tables=None):
    """Same charge (Gaussian for the unit cube, streamer densities otherwise)
    and coefficient table on both sides; returns the charge-rhs arguments."""
    import paper_1708_08434_gb300 as pkg
    t = tables if tables is not None else o.tables()
    if st is None:
        rho = synth.gaussian_charge(dom, t["level"], t["ijk"], np.arange(len(t["level"])))
        o.set(oracle.RHO, rho)
        g.upload(pkg.RHO, rho)
        o.charge_rhs(1.0, 1.0, True)
        g.charge_rhs(1.0, 1.0, True)
        return (1.0, 1.0, True)
    ne, ni = synth.streamer_densities(dom, st, t["level"], t["ijk"])
    o.set(oracle.NE, ne); o.set(oracle.NI, ni)
    g.upload(pkg.NE, ne); g.upload(pkg.NI, ni)
    tab = synth.coefficient_table()
    o.set_table(tab); g.set_table(tab)
    o.charge_rhs(Q, EPS0); g.charge_rhs(Q, EPS0)
    return (Q, EPS0, False)


def box_scale(t, ref):
    """Per box: max |ref| over the box, its 26 same-level neighbours and, at
    refinement faces, its parent's neighbours -- the magnitudes that the
    finite-volume update of the box combines, so the scale of its rounding
    errors (ref: [nbox, 512])."""
    m = np.abs(ref).max(axis=1)
    nbr = t["nbr"]
    s = np.maximum(m, np.where(nbr >= 0, m[np.clip(nbr, 0, None)], 0.0).max(axis=1))
    par = t["parent"]
    coarse = (nbr == -2).any(axis=1) & (par >= 0)
    pn = nbr[np.clip(par, 0, None)]
    ps = np.maximum(m[np.clip(par, 0, None)], np.where(pn >= 0, m[np.clip(pn, 0, None)], 0.0).max(axis=1))
    return np.where(coarse, np.maximum(s, ps), s)


def rel_err_local(a, b, t):
    """max over cells of |a - b| / max(|b|, box_scale of the cell's box)."""
    den = np.maximum(np.abs(b), box_scale(t, b)[:, None])
    den = np.where(den > 0, den, 1.0)
    return (np.abs(a - b) / den).max()
