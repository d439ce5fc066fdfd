"""CPU oracle for the octree multigrid Poisson solve and the fluid step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports
it.  The arithmetic lives in ``oracle.c`` (plain C, fp64, compiled with
``-O2 -ffp-contract=off``); this module only compiles and marshals.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, brute force, invariants, direct
solves); none is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
QUAD_LIB_PATH = os.path.join(_BUILD, "libquad.so")
_lock = threading.Lock()
_lib = None

PHI, RHS, RES, NE, NI, EMAG, RHO = range(7)


def _compile(src: str, hdr: str, out: str, force: bool) -> str:
    """gcc -O2 -ffp-contract=off src -> out (OpenMP when available)."""
    if not force and os.path.exists(out) and \
            os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    # OpenMP over boxes when the compiler has it; plain loops otherwise
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:],
                      stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so and quad.c into
    _build/libquad.so (gcc, no GPU needed); returns the first path."""
    _compile(os.path.join(_HERE, "quad.c"), os.path.join(_HERE, "quad.h"), QUAD_LIB_PATH, force)
    return _compile(os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h"), _LIB_PATH, force)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.c_double, dp, C.c_int, C.c_int, ip, dp]
        lib.orc_destroy.argtypes = [P]
        for name in ("orc_n_boxes", "orc_n_levels"):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = C.c_int
        lib.orc_level_offset.argtypes = [P, C.c_int]
        lib.orc_level_offset.restype = C.c_int
        lib.orc_refine_level.argtypes = [P, C.c_int, P, ip]
        lib.orc_refine_level.restype = C.c_int
        lib.orc_get_tables.argtypes = [P] * 7
        lib.orc_set.argtypes = [P, C.c_int, P]
        lib.orc_get.argtypes = [P, C.c_int, P]
        lib.orc_set_table.argtypes = [P, C.c_int, C.c_double, P, P, P]
        lib.orc_charge_rhs.argtypes = [P, C.c_double, C.c_double, C.c_int]
        lib.orc_fmg.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_int, dp, ip]
        lib.orc_fmg.restype = C.c_int
        lib.orc_solve.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_int, dp, ip]
        lib.orc_solve.restype = C.c_int
        lib.orc_vcycles.argtypes = [P, C.c_int, C.c_int, C.c_int, dp]
        lib.orc_vcycles.restype = C.c_int
        lib.orc_rel_residual.argtypes = [P]
        lib.orc_rel_residual.restype = C.c_double
        lib.orc_composite_residual.argtypes = [P]
        lib.orc_compute_field.argtypes = [P]
        lib.orc_dt_limit.argtypes = [P, C.c_double, C.c_double]
        lib.orc_dt_limit.restype = C.c_double
        lib.orc_advance.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_int, dp, ip, ip]
        lib.orc_advance.restype = C.c_int
        lib.orc_fluid_stage.argtypes = [P, C.c_double]
        lib.orc_koren.argtypes = [C.c_double, C.c_double]
        lib.orc_koren.restype = C.c_double
        lib.orc_lookup.argtypes = [P, C.c_int, C.c_double]
        lib.orc_lookup.restype = C.c_double
        lib.orc_coarse_solve.argtypes = [P]
        lib.orc_refine_flags.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, P]
        lib.orc_regrid.argtypes = [P, P, ip, ip, ip]
        lib.orc_regrid.restype = C.c_int
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_set_threads.restype = C.c_int
        lib.orc_set_threads(1)
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Threads for the per-box loops (1 at load; results do not depend on
    it).  Returns the count in effect, 1 if built without OpenMP."""
    return _load().orc_set_threads(int(n))


def threads() -> int:
    """Threads the per-box loops use now."""
    return _load().orc_set_threads(0)


def koren(a: float, b: float) -> float:
    """psi(a/b)*b of the Koren limiter (division-free form)."""
    return _load().orc_koren(a, b)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One octree + its fields on the CPU."""

    def __init__(self, dom):
        lib = _load()
        self._lib = lib
        self.dom = dom
        org = (C.c_double * 3)(*dom.origin)
        bct = (C.c_int * 6)(*dom.bc_type)
        bcv = (C.c_double * 6)(*dom.bc_val)
        self._h = lib.orc_create(dom.length, org, dom.nb, dom.max_level, bct, bcv)
        if not self._h:
            raise ValueError("oracle: bad domain")

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tables ----
    @property
    def n_boxes(self) -> int:
        return self._lib.orc_n_boxes(self._h)

    @property
    def n_levels(self) -> int:
        return self._lib.orc_n_levels(self._h)

    def level_range(self, level: int):
        return (self._lib.orc_level_offset(self._h, level),
                self._lib.orc_level_offset(self._h, level + 1))

    def tables(self) -> dict:
        n = self.n_boxes
        t = {
            "level": np.zeros(n, np.int32), "ijk": np.zeros((n, 3), np.int32),
            "morton": np.zeros(n, np.uint64), "parent": np.zeros(n, np.int32),
            "child": np.zeros((n, 8), np.int32), "nbr": np.zeros((n, 26), np.int32),
        }
        self._lib.orc_get_tables(self._h, *(_ptr(t[k]) for k in
                                            ("level", "ijk", "morton", "parent", "child", "nbr")))
        t["level_offset"] = np.array([self._lib.orc_level_offset(self._h, l)
                                      for l in range(self.n_levels + 1)], np.int32)
        return t

    def level_ijk(self, level: int) -> np.ndarray:
        if level >= self.n_levels:
            return np.zeros((0, 3), np.int32)
        lo, hi = self.level_range(level)
        return self.tables()["ijk"][lo:hi]

    def refine_level(self, level: int, flags) -> int:
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        dropped = C.c_int(0)
        r = self._lib.orc_refine_level(self._h, level, _ptr(flags), C.byref(dropped))
        if r < 0:
            raise ValueError("oracle refine_level(%d) refused" % level)
        self.dropped = dropped.value
        return r

    # ---- refinement criterion and regridding (Sec. 2.5, Eq. 8) ----
    def refine_flags(self, c0=1.0, c1=1.2, c0_deref=0.125, dx_deref=30e-6, buffer=3) -> np.ndarray:
        """Per-box flags from the stored |E|: +1 refine, -1 derefinable, 0."""
        f = np.zeros(self.n_boxes, np.int8)
        self._lib.orc_refine_flags(self._h, c0, c1, c0_deref, dx_deref, buffer, _ptr(f))
        return f

    def regrid(self, flags):
        """Apply per-box flags; returns (refined, derefined, dropped)."""
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.n_boxes,)
        r, d, x = C.c_int(0), C.c_int(0), C.c_int(0)
        self._lib.orc_regrid(self._h, _ptr(flags), C.byref(r), C.byref(d), C.byref(x))
        return r.value, d.value, x.value

    # ---- fields ----
    def set(self, var: int, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.n_boxes, 512)
        self._lib.orc_set(self._h, var, _ptr(a))

    def get(self, var: int) -> np.ndarray:
        a = np.zeros((self.n_boxes, 512), np.float64)
        self._lib.orc_get(self._h, var, _ptr(a))
        return a

    def set_table(self, tab: dict):
        mu = np.ascontiguousarray(tab["mu"], np.float64)
        dc = np.ascontiguousarray(tab["diff"], np.float64)
        al = np.ascontiguousarray(tab["alpha"], np.float64)
        self._lib.orc_set_table(self._h, len(mu), tab["e_max"], _ptr(mu), _ptr(dc), _ptr(al))

    def lookup(self, which: int, e: float) -> float:
        return self._lib.orc_lookup(self._h, which, e)

    # ---- operations ----
    def charge_rhs(self, q=1.0, eps=1.0, use_rho=False):
        self._lib.orc_charge_rhs(self._h, q, eps, int(use_rho))

    def fmg(self, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        rel = C.c_double(0)
        cyc = C.c_int(0)
        st = self._lib.orc_fmg(self._h, tol, max_cycles, nu1, nu2, C.byref(rel), C.byref(cyc))
        return st, rel.value, cyc.value

    def solve(self, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        rel = C.c_double(0)
        cyc = C.c_int(0)
        st = self._lib.orc_solve(self._h, tol, max_cycles, nu1, nu2, C.byref(rel), C.byref(cyc))
        return st, rel.value, cyc.value

    def vcycles(self, n, nu1=2, nu2=2):
        rel = C.c_double(0)
        self._lib.orc_vcycles(self._h, n, nu1, nu2, C.byref(rel))
        return rel.value

    def rel_residual(self) -> float:
        return self._lib.orc_rel_residual(self._h)

    def composite_residual(self) -> np.ndarray:
        self._lib.orc_composite_residual(self._h)
        return self.get(RES)

    def coarse_solve(self):
        self._lib.orc_coarse_solve(self._h)

    def compute_field(self):
        self._lib.orc_compute_field(self._h)

    def dt_limit(self, q, eps) -> float:
        return self._lib.orc_dt_limit(self._h, q, eps)

    def fluid_stage(self, dt):
        self._lib.orc_fluid_stage(self._h, dt)

    def advance(self, dt, q, eps, tol=1e-8, max_cycles=50, nu1=2, nu2=2):
        dtn = C.c_double(0)
        c1 = C.c_int(0)
        c2 = C.c_int(0)
        st = self._lib.orc_advance(self._h, dt, q, eps, tol, max_cycles, nu1, nu2,
                                   C.byref(dtn), C.byref(c1), C.byref(c2))
        return st, dtn.value, c1.value, c2.value


def build_mesh(dom, st=None):
    """Oracle octree for a domain, refined level by level with the synthetic
    streamer requests when `st` is given."""
    import synth
    o = Oracle(dom)
    if st is not None:
        synth.refine_all(dom, st, o.level_ijk, o.refine_level)
    return o
