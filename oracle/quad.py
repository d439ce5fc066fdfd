"""CPU oracle of the 2-D and axisymmetric variants (quadtree of 8^2-cell
boxes): multigrid Poisson solve and fluid step.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The arithmetic lives in
``quad.c`` (plain C, fp64, ``-O2 -ffp-contract=off``); this module only
compiles and marshals.

Parity status: pinned by ``tests/test_oracle_quad.py`` (brute-force tables,
closed-form eigenvectors, exactness on r^2 and on the plate-gap field,
second-order convergence to a continuum solution in both geometries, a
sparse direct solve of the composite operator, conservation, closed-form
growth); none is unpinned.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import QUAD_LIB_PATH, build

PHI, RHS, RES, NE, NI, EMAG, RHO = range(7)
_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(QUAD_LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        sig = {
            "q2_create": ([D, dp, I, I, I, ip, dp], P),
            "q2_destroy": ([P], None),
            "q2_set_threads": ([I], I),
            "q2_n_boxes": ([P], I),
            "q2_n_levels": ([P], I),
            "q2_level_offset": ([P, I], I),
            "q2_refine_level": ([P, I, P, ip], I),
            "q2_get_tables": ([P] * 7, None),
            "q2_set": ([P, I, P], None),
            "q2_get": ([P, I, P], None),
            "q2_set_table": ([P, I, D, P, P, P], None),
            "q2_charge_rhs": ([P, D, D, I], None),
            "q2_fmg": ([P, D, I, I, I, dp, ip], I),
            "q2_solve": ([P, D, I, I, I, dp, ip], I),
            "q2_vcycles": ([P, I, I, I, dp], I),
            "q2_rel_residual": ([P], D),
            "q2_composite_residual": ([P], None),
            "q2_restrict_all": ([P, I], None),
            "q2_compute_field": ([P], None),
            "q2_dt_limit": ([P, D, D], D),
            "q2_fluid_stage": ([P, D], None),
            "q2_advance": ([P, D, D, D, D, I, I, I, dp, ip, ip], I),
            "q2_coarse_solve": ([P], None),
            "q2_refine_flags": ([P, D, D, D, D, I, P], None),
            "q2_lookup": ([P, I, D], D),
            "q2_koren": ([D, D], D),
            "q2_regrid": ([P, P, ip, ip, ip], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        lib.q2_set_threads(1)
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    return _load().q2_set_threads(int(n))


def koren(a: float, b: float) -> float:
    """psi(a/b) b of the Koren limiter (Eq. 7), as the 2-D oracle applies it."""
    return _load().q2_koren(float(a), float(b))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Quad:
    """One quadtree + its fields on the CPU."""

    def __init__(self, dom):
        lib = _load()
        self._lib = lib
        self.dom = dom
        org = (C.c_double * 2)(*dom.origin)
        bct = (C.c_int * 4)(*dom.bc_type)
        bcv = (C.c_double * 4)(*dom.bc_val)
        self._h = lib.q2_create(dom.length, org, dom.nb, dom.max_level, dom.geom, bct, bcv)
        if not self._h:
            raise ValueError("quad oracle: bad domain")

    def close(self):
        if self._h:
            self._lib.q2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_boxes(self) -> int:
        return self._lib.q2_n_boxes(self._h)

    @property
    def n_levels(self) -> int:
        return self._lib.q2_n_levels(self._h)

    def level_range(self, level: int):
        return self._lib.q2_level_offset(self._h, level), self._lib.q2_level_offset(self._h, level + 1)

    def tables(self) -> dict:
        n = self.n_boxes
        t = {"level": np.zeros(n, np.int32), "ij": np.zeros((n, 2), np.int32),
             "morton": np.zeros(n, np.uint64), "parent": np.zeros(n, np.int32),
             "child": np.zeros((n, 4), np.int32), "nbr": np.zeros((n, 8), np.int32)}
        self._lib.q2_get_tables(self._h, *(_ptr(t[k]) for k in
                                           ("level", "ij", "morton", "parent", "child", "nbr")))
        t["level_offset"] = np.array([self._lib.q2_level_offset(self._h, l)
                                      for l in range(self.n_levels + 1)], np.int32)
        return t

    def level_ij(self, level: int) -> np.ndarray:
        if level >= self.n_levels:
            return np.zeros((0, 2), np.int32)
        lo, hi = self.level_range(level)
        return self.tables()["ij"][lo:hi]

    def refine_level(self, level: int, flags) -> int:
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        dropped = C.c_int(0)
        r = self._lib.q2_refine_level(self._h, level, _ptr(flags), C.byref(dropped))
        if r < 0:
            raise ValueError("quad oracle refine_level(%d) refused" % level)
        self.dropped = dropped.value
        return r

    def refine_flags(self, c0=1.0, c1=1.2, c0_deref=0.125, dx_deref=30e-6, buffer=3) -> np.ndarray:
        """Per-box flags from the stored |E| (Eq. 8): +1 refine, -1 derefinable, 0."""
        f = np.zeros(self.n_boxes, np.int8)
        self._lib.q2_refine_flags(self._h, c0, c1, c0_deref, dx_deref, buffer, _ptr(f))
        return f

    def regrid(self, flags):
        """Apply per-box flags; returns (refined, derefined, dropped)."""
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.n_boxes,)
        r, d, x = C.c_int(0), C.c_int(0), C.c_int(0)
        self._lib.q2_regrid(self._h, _ptr(flags), C.byref(r), C.byref(d), C.byref(x))
        return r.value, d.value, x.value

    def set(self, var: int, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.n_boxes, 64)
        self._lib.q2_set(self._h, var, _ptr(a))

    def get(self, var: int) -> np.ndarray:
        a = np.zeros((self.n_boxes, 64), np.float64)
        self._lib.q2_get(self._h, var, _ptr(a))
        return a

    def set_table(self, tab: dict):
        mu = np.ascontiguousarray(tab["mu"], np.float64)
        dc = np.ascontiguousarray(tab["diff"], np.float64)
        al = np.ascontiguousarray(tab["alpha"], np.float64)
        self._lib.q2_set_table(self._h, len(mu), tab["e_max"], _ptr(mu), _ptr(dc), _ptr(al))

    def lookup(self, which: int, e: float) -> float:
        return self._lib.q2_lookup(self._h, which, e)

    def charge_rhs(self, q=1.0, eps=1.0, use_rho=False):
        self._lib.q2_charge_rhs(self._h, q, eps, int(use_rho))

    def fmg(self, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        rel, cyc = C.c_double(0), C.c_int(0)
        st = self._lib.q2_fmg(self._h, tol, max_cycles, nu1, nu2, C.byref(rel), C.byref(cyc))
        return st, rel.value, cyc.value

    def solve(self, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        rel, cyc = C.c_double(0), C.c_int(0)
        st = self._lib.q2_solve(self._h, tol, max_cycles, nu1, nu2, C.byref(rel), C.byref(cyc))
        return st, rel.value, cyc.value

    def vcycles(self, n, nu1=2, nu2=2):
        rel = C.c_double(0)
        self._lib.q2_vcycles(self._h, n, nu1, nu2, C.byref(rel))
        return rel.value

    def rel_residual(self) -> float:
        return self._lib.q2_rel_residual(self._h)

    def composite_residual(self) -> np.ndarray:
        self._lib.q2_composite_residual(self._h)
        return self.get(RES)

    def restrict_all(self, var: int):
        self._lib.q2_restrict_all(self._h, var)

    def coarse_solve(self):
        self._lib.q2_coarse_solve(self._h)

    def compute_field(self):
        self._lib.q2_compute_field(self._h)

    def dt_limit(self, q, eps) -> float:
        return self._lib.q2_dt_limit(self._h, q, eps)

    def fluid_stage(self, dt):
        self._lib.q2_fluid_stage(self._h, dt)

    def advance(self, dt, q, eps, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        dtn, c1, c2 = C.c_double(0), C.c_int(0), C.c_int(0)
        st = self._lib.q2_advance(self._h, dt, q, eps, tol, max_cycles, nu1, nu2,
                                  C.byref(dtn), C.byref(c1), C.byref(c2))
        return st, dtn.value, c1.value, c2.value


def build_mesh(dom, st=None):
    """Quadtree for a domain, refined level by level with the synthetic
    streamer requests when `st` is given."""
    import synth
    o = Quad(dom)
    if st is not None:
        synth.refine_all2(dom, st, o.level_ij, o.refine_level)
    return o
