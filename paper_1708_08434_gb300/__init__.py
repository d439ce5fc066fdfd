"""Python binding of the GB300 library for the per-time-step path of the
streamer fluid model of arXiv:1708.08434 (octree multigrid Poisson solve
and drift-diffusion-reaction step).

Argument marshalling only: every step runs in the CUDA kernels of
``libsm_streamer.so`` (C ABI in ``include/sm_streamer.h``).  PyTorch
provides the device memory (one arena tensor per solver) and the stream.
There is no CPU fallback: without the compiled library or a CUDA device,
constructing a ``Solver`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

SM_OK, SM_EINVAL, SM_ENOMEM, SM_ECUDA, SM_ENOCONV, SM_ETIMEOUT, SM_ESTATE = 0, -1, -2, -3, -4, -5, -6
PHI, RHS, RES, NE, NI, EMAG, RHO = range(7)
FP64, MIXED = 0, 1
MAX_LEVELS = 24
K_SMOOTH = 0
K_PERSIST = 1
K_VCYCLE = 2
K_VCYCLE32 = 3

_NAMES = {SM_EINVAL: "SM_EINVAL", SM_ENOMEM: "SM_ENOMEM", SM_ECUDA: "SM_ECUDA",
          SM_ENOCONV: "SM_ENOCONV", SM_ETIMEOUT: "SM_ETIMEOUT", SM_ESTATE: "SM_ESTATE"}


class SmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, code), msg))
        self.code = code


class _Domain(C.Structure):
    _fields_ = [("length", C.c_double), ("origin", C.c_double * 3), ("nb", C.c_int),
                ("max_level", C.c_int), ("bc_type", C.c_int * 6), ("bc_val", C.c_double * 6)]


class _Config(C.Structure):
    _fields_ = [("max_boxes", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("precision", C.c_int)]


class _Tables(C.Structure):
    _fields_ = [("n_boxes", C.c_int), ("n_levels", C.c_int), ("n_leaves", C.c_int),
                ("level_offset", C.c_int * (MAX_LEVELS + 1)),
                ("level", C.c_void_p), ("ijk", C.c_void_p), ("morton", C.c_void_p),
                ("parent", C.c_void_p), ("child", C.c_void_p), ("nbr", C.c_void_p),
                ("leaf", C.c_void_p)]


_lib = None

EXPORTS = ["sm_create", "sm_destroy", "sm_arena_size", "sm_bind_arena", "sm_build_octree",
           "sm_refine_level", "sm_get_tables", "sm_var_ptr", "sm_upload", "sm_download",
           "sm_set_table", "sm_charge_rhs", "sm_restrict_densities", "sm_fill_ghosts",
           "sm_mg_vcycle", "sm_mg_solve", "sm_mg_fmg", "sm_compute_field", "sm_dt_limit",
           "sm_fluid_stage", "sm_advance_fluid", "sm_kernel_bench", "sm_set_graphs", "sm_set_pdl",
           "sm_set_persistent", "sm_persist_barrier_selftest",
           "sm_launch_count", "sm_last_error", "sm_box_solve_noalloc", "sm_check_conversions", "sm_fp64_probe",
           "sm_refine_flags", "sm_regrid",
           "sm_batch_create", "sm_batch_destroy", "sm_batch_arena_size", "sm_batch_bind_arena",
           "sm_batch_ptrs", "sm_batch_solve", "sm_batch_tune", "sm_batch_set_schedule", "sm_batch_info",
           "sm_batch_set_graphs", "sm_batch_kernel_bench", "sm_cnn_create", "sm_cnn_destroy", "sm_cnn_arena_size",
           "sm_cnn_bind_arena", "sm_cnn_set_params", "sm_cnn_get_params", "sm_cnn_forward",
           "sm_cnn_gradient", "sm_cnn_adam_step", "sm_cnn_train", "sm_cnn_attach", "sm_cnn_stats",
           "sm_cnn_kernel_bench", "sm_cnn_load_samples", "sm_set_metrics_log",
           "sm_set_row_kernels", "sm_var_layout", "sm_fill_ghosts_range", "sm_get_ghosts", "sm_refine",
           "sm_advance_fluid_coeffs",
           "sm_cnn_last_error",
           "sm_batch_last_error",
           "sm_quad_create", "sm_quad_destroy", "sm_quad_arena_size", "sm_quad_bind_arena",
           "sm_quad_refine_level", "sm_quad_get_tables", "sm_quad_var_ptr", "sm_quad_upload",
           "sm_quad_download", "sm_quad_set_table", "sm_quad_charge_rhs", "sm_quad_fmg",
           "sm_quad_solve", "sm_quad_vcycles", "sm_quad_compute_field", "sm_quad_dt_limit", "sm_quad_fluid_stage",
           "sm_quad_advance", "sm_quad_refine_flags", "sm_quad_regrid", "sm_quad_set_graphs", "sm_quad_set_pdl", "sm_quad_launch_count", "sm_quad_last_error"]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libsm_streamer.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("CUDA library %s is not built (run __graft_entry__.build())" % path)
    lib = C.CDLL(path)
    for name, args in signatures().items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name.endswith("last_error") else C.c_int
    _lib = lib
    return lib


def signatures() -> dict:
    """ctypes argument types of every C-ABI entry point, by name (the
    prototypes of include/sm_streamer.h and include/sm_quad.h)."""
    P, I, D = C.c_void_p, C.c_int, C.c_double
    pI, pD = C.POINTER(C.c_int), C.POINTER(C.c_double)
    return {
        "sm_create": [C.POINTER(P), P, P, P],
        "sm_destroy": [P],
        "sm_arena_size": [P, C.POINTER(C.c_size_t)],
        "sm_bind_arena": [P, P, C.c_size_t],
        "sm_build_octree": [P, pI],
        "sm_refine_level": [P, I, P, pI, pI],
        "sm_get_tables": [P, P],
        "sm_var_ptr": [P, I, C.POINTER(P)],
        "sm_upload": [P, I, P, I],
        "sm_download": [P, I, P, I],
        "sm_set_table": [P, I, D, P, P, P],
        "sm_charge_rhs": [P, D, D, I],
        "sm_restrict_densities": [P],
        "sm_fill_ghosts": [P, I, I],
        "sm_mg_vcycle": [P, I, pD],
        "sm_mg_solve": [P, D, I, pI, pD],
        "sm_mg_fmg": [P, D, I, pI, pD],
        "sm_compute_field": [P],
        "sm_dt_limit": [P, D, D, pD],
        "sm_fluid_stage": [P, D],
        "sm_advance_fluid": [P, D, D, D, D, I, pD, pI],
        "sm_kernel_bench": [P, I, I, pD, C.POINTER(C.c_longlong), pD, pD],
        "sm_set_graphs": [P, I],
        "sm_set_pdl": [P, I],
        "sm_set_persistent": [P, I],
        "sm_persist_barrier_selftest": [P],
        "sm_launch_count": [P, C.POINTER(C.c_longlong)],
        "sm_box_solve_noalloc": [D, I, P, P, P, P, P],
        "sm_check_conversions": [C.c_longlong, C.c_ulonglong, P, P, P],
        "sm_fp64_probe": [C.c_longlong, P, pD, pD, P],
        "sm_refine_flags": [P, D, D, D, D, I, P],
        "sm_regrid": [P, P, pI, pI, pI],
        "sm_batch_create": [C.POINTER(P), I, P, D, P, P, I, I, P],
        "sm_batch_destroy": [P],
        "sm_batch_arena_size": [P, C.POINTER(C.c_size_t)],
        "sm_batch_bind_arena": [P, P, C.c_size_t],
        "sm_batch_ptrs": [P, C.POINTER(P), C.POINTER(P), P],
        "sm_batch_solve": [P, D, I, P, P],
        "sm_batch_tune": [P, I, pI, pI, pD],
        "sm_batch_set_schedule": [P, I, I],
        "sm_batch_set_graphs": [P, I],
        "sm_batch_kernel_bench": [P, I, I, pD, pD, pD],
        "sm_batch_info": [P, C.POINTER(C.c_longlong), pI, C.POINTER(C.c_longlong)],
        "sm_batch_last_error": [P],
        "sm_cnn_create": [C.POINTER(P), I, I, P],
        "sm_cnn_destroy": [P],
        "sm_cnn_arena_size": [P, C.POINTER(C.c_size_t)],
        "sm_cnn_bind_arena": [P, P, C.c_size_t],
        "sm_cnn_set_params": [P, P, I],
        "sm_cnn_get_params": [P, P, I],
        "sm_cnn_forward": [P, P, I, P, P],
        "sm_cnn_gradient": [P, P, P, I, P, C.POINTER(C.c_float)],
        "sm_cnn_adam_step": [P, P, C.c_float],
        "sm_cnn_train": [P, I, I, C.c_float, C.c_ulonglong, C.POINTER(C.c_float)],
        "sm_cnn_attach": [P, P, I, I, I, I, D],
        "sm_cnn_stats": [P, pI, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), pD],
        "sm_cnn_kernel_bench": [P, I, I, I, pD, pD, pD],
        "sm_cnn_load_samples": [P, P, P, I],
        "sm_set_metrics_log": [P, C.c_char_p, D],
        "sm_set_row_kernels": [P, I],
        "sm_var_layout": [P, I, C.POINTER(C.c_void_p), pI, pI],
        "sm_fill_ghosts_range": [P, I, I, I],
        "sm_get_ghosts": [P, I, P, I],
        "sm_refine": [P, P, pI],
        "sm_advance_fluid_coeffs": [P, D, P, pD, pI],
        "sm_cnn_last_error": [P],
        "sm_last_error": [P],
        "sm_quad_create": [C.POINTER(P), P, I, I, I, P],
        "sm_quad_destroy": [P],
        "sm_quad_arena_size": [P, C.POINTER(C.c_size_t)],
        "sm_quad_bind_arena": [P, P, C.c_size_t],
        "sm_quad_refine_level": [P, I, P, pI, pI],
        "sm_quad_get_tables": [P, pI, pI, P, P, P, P, P, P, P],
        "sm_quad_var_ptr": [P, I, C.POINTER(P)],
        "sm_quad_upload": [P, I, P],
        "sm_quad_download": [P, I, P],
        "sm_quad_set_table": [P, I, D, P, P, P],
        "sm_quad_charge_rhs": [P, D, D, I],
        "sm_quad_fmg": [P, D, I, pI, pD],
        "sm_quad_solve": [P, D, I, pI, pD],
        "sm_quad_vcycles": [P, I],
        "sm_quad_compute_field": [P],
        "sm_quad_dt_limit": [P, D, D, pD],
        "sm_quad_fluid_stage": [P, D],
        "sm_quad_advance": [P, D, D, D, D, I, pD, P],
        "sm_quad_refine_flags": [P, D, D, D, D, I, P],
        "sm_quad_regrid": [P, P, pI, pI, pI],
        "sm_quad_set_graphs": [P, I],
        "sm_quad_set_pdl": [P, I],
        "sm_quad_launch_count": [P, C.POINTER(C.c_longlong)],
        "sm_quad_last_error": [P],
    }


def _hp(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def check_conversions(n: int, seed: int = 0x5EED):
    """Mismatches (FP64->FP32, FP32->FP64, FP64->fixed point) of the
    library's integer-pipe conversions on n seeded bit patterns: the first
    two against the hardware conversions, the fixed-point one against exact
    FP64 scaling with the tie rule."""
    import torch
    lib = load()
    scratch = torch.zeros(3, dtype=torch.int64, device="cuda")
    out = np.zeros(3, np.uint64)
    stream = torch.cuda.current_stream()
    rc = lib.sm_check_conversions(int(n), int(seed), C.c_void_p(scratch.data_ptr()), _hp(out),
                                  C.c_void_p(stream.cuda_stream))
    if rc != SM_OK:
        raise SmError(rc, "sm_check_conversions failed")
    return tuple(int(v) for v in out)


def fp64_probe(iters: int = 1 << 16):
    """Measured FP64-pipe throughput of this GPU: (fused multiply-adds per
    second, duration of the timed launch in ms)."""
    import torch
    lib = load()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    rate, ms = C.c_double(0.0), C.c_double(0.0)
    stream = torch.cuda.current_stream()
    rc = lib.sm_fp64_probe(int(iters), C.c_void_p(sink.data_ptr()), C.byref(rate), C.byref(ms),
                           C.c_void_p(stream.cuda_stream))
    if rc != SM_OK:
        raise SmError(rc, "sm_fp64_probe failed")
    return rate.value, ms.value


class Solver:
    """One octree with its fields on the current CUDA device."""

    def __init__(self, dom, max_boxes: int, nu1: int = 2, nu2: int = 2, precision: int = FP64,
                 stream=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise SmError(SM_ECUDA, "no CUDA device")
        self._lib = lib
        self.torch = torch
        self.dom = dom
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d = _Domain(dom.length, (C.c_double * 3)(*dom.origin), dom.nb, dom.max_level,
                    (C.c_int * 6)(*dom.bc_type), (C.c_double * 6)(*dom.bc_val))
        cfg = _Config(max_boxes, nu1, nu2, precision)
        h = C.c_void_p()
        rc = lib.sm_create(C.byref(h), C.byref(cfg), C.byref(d), C.c_void_p(self.stream.cuda_stream))
        if rc != SM_OK:
            raise SmError(rc, "sm_create failed")
        self._h = h
        size = C.c_size_t()
        self._ck(lib.sm_arena_size(h, C.byref(size)))
        self.arena = torch.empty(size.value, dtype=torch.uint8, device="cuda")
        self._ck(lib.sm_bind_arena(h, C.c_void_p(self.arena.data_ptr()), size.value))
        self.max_boxes = max_boxes

    # -- plumbing --
    def _ck(self, rc):
        if rc != SM_OK:
            raise SmError(rc, self._lib.sm_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.sm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _view(self, ptr: int, count: int, dtype):
        """Zero-copy torch view of `count` elements at device pointer `ptr`."""
        off = ptr - self.arena.data_ptr()
        nbytes = count * dtype.itemsize
        assert 0 <= off and off + nbytes <= self.arena.numel()
        return self.arena[off:off + nbytes].view(dtype)

    # -- octree --
    def build_octree(self) -> int:
        n = C.c_int()
        self._ck(self._lib.sm_build_octree(self._h, C.byref(n)))
        return n.value

    def refine_level(self, level: int, flags) -> int:
        f = np.ascontiguousarray(flags, dtype=np.int8)
        new, dropped = C.c_int(), C.c_int()
        self._ck(self._lib.sm_refine_level(self._h, level, _hp(f), C.byref(new), C.byref(dropped)))
        self.dropped = dropped.value
        return new.value

    def _tables_raw(self) -> _Tables:
        t = _Tables()
        self._ck(self._lib.sm_get_tables(self._h, C.byref(t)))
        return t

    @property
    def n_boxes(self) -> int:
        return self._tables_raw().n_boxes

    @property
    def n_levels(self) -> int:
        return self._tables_raw().n_levels

    @property
    def n_leaves(self) -> int:
        return self._tables_raw().n_leaves

    def tables(self) -> dict:
        """Device tables copied to numpy (tests and input generation)."""
        torch = self.torch
        t = self._tables_raw()
        n = t.n_boxes
        self.stream.synchronize()
        i32 = torch.int32
        out = {
            "level": self._view(t.level, n, i32).cpu().numpy().copy(),
            "ijk": self._view(t.ijk, 3 * n, i32).cpu().numpy().reshape(n, 3).copy(),
            "morton": self._view(t.morton, 2 * n, i32).cpu().numpy().view(np.uint64).copy(),
            "parent": self._view(t.parent, n, i32).cpu().numpy().copy(),
            "child": self._view(t.child, 8 * n, i32).cpu().numpy().reshape(n, 8).copy(),
            "nbr": self._view(t.nbr, 26 * n, i32).cpu().numpy().reshape(n, 26).copy(),
            "leaf": self._view(t.leaf, t.n_leaves, i32).cpu().numpy().copy(),
            "level_offset": np.array(t.level_offset[:t.n_levels + 1], np.int32),
        }
        return out

    def level_ijk(self, level: int) -> np.ndarray:
        t = self._tables_raw()
        if level >= t.n_levels:
            return np.zeros((0, 3), np.int32)
        lo, hi = t.level_offset[level], t.level_offset[level + 1]
        self.stream.synchronize()
        v = self._view(t.ijk, 3 * t.n_boxes, self.torch.int32)
        return v[3 * lo:3 * hi].cpu().numpy().reshape(-1, 3)

    def level_range(self, level: int):
        t = self._tables_raw()
        return t.level_offset[level], t.level_offset[level + 1]

    # -- refinement criterion and regridding (Sec. 2.5, Eq. 8) --
    def refine_flags(self, c0=1.0, c1=1.2, c0_deref=0.125, dx_deref=30e-6, buffer=3) -> np.ndarray:
        """Per-box flags from the stored |E|: +1 refine, -1 derefinable, 0."""
        f = np.zeros(self.n_boxes, np.int8)
        self._ck(self._lib.sm_refine_flags(self._h, c0, c1, c0_deref, dx_deref, buffer, _hp(f)))
        return f

    def regrid(self, flags):
        """Apply per-box flags; returns (refined, derefined, dropped)."""
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.n_boxes,)
        r, d, x = C.c_int(), C.c_int(), C.c_int()
        self._ck(self._lib.sm_regrid(self._h, _hp(flags), C.byref(r), C.byref(d), C.byref(x)))
        return r.value, d.value, x.value

    # -- fields --
    def var(self, var: int):
        """Zero-copy [n_boxes, 512] float64 torch view of a variable."""
        p = C.c_void_p()
        self._ck(self._lib.sm_var_ptr(self._h, var, C.byref(p)))
        n = self.n_boxes
        return self._view(p.value, n * 512, self.torch.float64).view(n, 512)

    def upload(self, var: int, arr):
        """Host -> device for boxes [0, n); arr: numpy array or pinned torch CPU tensor."""
        if isinstance(arr, np.ndarray):
            a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1, 512)
            self._keep = a
            self._ck(self._lib.sm_upload(self._h, var, _hp(a), a.shape[0]))
            self.stream.synchronize()
        else:
            self._ck(self._lib.sm_upload(self._h, var, C.c_void_p(arr.data_ptr()), arr.numel() // 512))

    def download(self, var: int, out=None):
        n = self.n_boxes
        if out is None:
            out = np.empty((n, 512), np.float64)
        if isinstance(out, np.ndarray):
            self._ck(self._lib.sm_download(self._h, var, _hp(out), out.shape[0]))
        else:
            self._ck(self._lib.sm_download(self._h, var, C.c_void_p(out.data_ptr()), out.numel() // 512))
        return out

    def set_table(self, tab: dict):
        mu = np.ascontiguousarray(tab["mu"], np.float64)
        dc = np.ascontiguousarray(tab["diff"], np.float64)
        al = np.ascontiguousarray(tab["alpha"], np.float64)
        self._ck(self._lib.sm_set_table(self._h, len(mu), float(tab["e_max"]), _hp(mu), _hp(dc), _hp(al)))

    # -- method steps --
    def charge_rhs(self, q=1.0, eps=1.0, use_rho=False):
        self._ck(self._lib.sm_charge_rhs(self._h, q, eps, int(use_rho)))

    def restrict_densities(self):
        self._ck(self._lib.sm_restrict_densities(self._h))

    def fill_ghosts(self, level: int, var: int = PHI):
        self._ck(self._lib.sm_fill_ghosts(self._h, var, level))

    def fill_ghosts_range(self, level_lo: int, level_hi: int, var: int = PHI):
        self._ck(self._lib.sm_fill_ghosts_range(self._h, var, level_lo, level_hi))

    def ghosts(self, var: int = PHI) -> np.ndarray:
        """Stored interpolation values phihat, [n_boxes][6][64]."""
        out = np.zeros((self.n_boxes, 6, 64), np.float64)
        self._ck(self._lib.sm_get_ghosts(self._h, var, _hp(out), self.n_boxes))
        return out

    def var_layout(self, var: int):
        """(device pointer, doubles per box, boxes in use) of a variable."""
        p, ld, nb = C.c_void_p(), C.c_int(), C.c_int()
        self._ck(self._lib.sm_var_layout(self._h, var, C.byref(p), C.byref(ld), C.byref(nb)))
        return p.value, ld.value, nb.value

    def vcycles(self, n: int) -> float:
        rel = C.c_double()
        self._ck(self._lib.sm_mg_vcycle(self._h, n, C.byref(rel)))
        return rel.value

    def _solve(self, fn, tol, max_cycles, allow_noconv):
        rel, cyc = C.c_double(), C.c_int()
        rc = fn(self._h, tol, max_cycles, C.byref(cyc), C.byref(rel))
        if rc != SM_OK and not (allow_noconv and rc == SM_ENOCONV):
            self._ck(rc)
        return rc, rel.value, cyc.value

    def solve(self, tol=1e-8, max_cycles=50, allow_noconv=True):
        return self._solve(self._lib.sm_mg_solve, tol, max_cycles, allow_noconv)

    def fmg(self, tol=1e-8, max_cycles=50, allow_noconv=True):
        return self._solve(self._lib.sm_mg_fmg, tol, max_cycles, allow_noconv)

    def compute_field(self):
        self._ck(self._lib.sm_compute_field(self._h))

    def dt_limit(self, q, eps) -> float:
        dt = C.c_double()
        self._ck(self._lib.sm_dt_limit(self._h, q, eps, C.byref(dt)))
        return dt.value

    def fluid_stage(self, dt):
        self._ck(self._lib.sm_fluid_stage(self._h, dt))

    def advance(self, dt, q, eps, tol=1e-8, max_cycles=50, allow_noconv=True):
        dtn = C.c_double()
        cyc = (C.c_int * 2)()
        rc = self._lib.sm_advance_fluid(self._h, dt, q, eps, tol, max_cycles, C.byref(dtn), cyc)
        if rc != SM_OK and not (allow_noconv and rc == SM_ENOCONV):
            self._ck(rc)
        return rc, dtn.value, cyc[0], cyc[1]

    # -- diagnostics --
    def set_graphs(self, enable: bool):
        self._ck(self._lib.sm_set_graphs(self._h, int(enable)))

    def persist_barrier_selftest(self) -> int:
        """Status of a persistent launch whose grid barriers cannot complete
        (SM_ETIMEOUT expected); the context stays usable."""
        return int(self._lib.sm_persist_barrier_selftest(self._h))

    def set_pdl(self, enable: bool):
        """Programmatic dependent launch of the solver kernels on or off."""
        self._ck(self._lib.sm_set_pdl(self._h, int(enable)))

    def kernel_bench(self, kclass: int = K_SMOOTH, reps: int = 10):
        """(microseconds per launch, launches, algorithmic bytes and FP64
        operations per launch) of a kernel class."""
        us, n, by, fl = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        self._ck(self._lib.sm_kernel_bench(self._h, kclass, reps, C.byref(us), C.byref(n), C.byref(by),
                                           C.byref(fl)))
        return us.value, n.value, by.value, fl.value

    def set_metrics_log(self, path, hbm_peak_gbs: float = 0.0):
        """Append one JSON line per solve (cycles, residual history, time,
        algorithmic bytes, bandwidth) to `path`; None closes the log."""
        self._ck(self._lib.sm_set_metrics_log(self._h, path.encode() if path else None, float(hbm_peak_gbs)))

    def set_row_kernels(self, min_boxes: int):
        """Levels of at least min_boxes boxes run the row kernels (0: all)."""
        self._ck(self._lib.sm_set_row_kernels(self._h, int(min_boxes)))

    def set_persistent(self, enable: bool):
        """V-cycles as one persistent cooperative launch, or as per-level
        launches (default)."""
        self._ck(self._lib.sm_set_persistent(self._h, int(enable)))

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._ck(self._lib.sm_launch_count(self._h, C.byref(n)))
        return n.value


class Batch:
    """Many independent uniform-grid Poisson solves advanced together."""

    # restriction schedules: coarse-cell tiles (x, y, z), then fine columns
    SHAPES = ((8, 8, 8), (16, 8, 4), (32, 4, 4), (32, 8, 2), "columns")

    def __init__(self, sides, length=1.0, bc_type=(0, 0, 0, 0, 1, 1), bc_val=(0, 0, 0, 0, 0, 1.0),
                 nu1=2, nu2=2, stream=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise SmError(SM_ECUDA, "no CUDA device")
        self._lib, self.torch = lib, torch
        self.sides = np.ascontiguousarray(sides, dtype=np.int32)
        self.n = len(self.sides)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = lib.sm_batch_create(C.byref(h), self.n, _hp(self.sides), float(length),
                                 (C.c_int * 6)(*bc_type), (C.c_double * 6)(*bc_val), nu1, nu2,
                                 C.c_void_p(self.stream.cuda_stream))
        if rc != SM_OK:
            raise SmError(rc, "sm_batch_create failed")
        self._h = h
        size = C.c_size_t()
        self._ck(lib.sm_batch_arena_size(h, C.byref(size)))
        self.arena = torch.empty(size.value, dtype=torch.uint8, device="cuda")
        self._ck(lib.sm_batch_bind_arena(h, C.c_void_p(self.arena.data_ptr()), size.value))
        phi, rhs = C.c_void_p(), C.c_void_p()
        self.offsets = np.zeros(self.n, np.int64)
        self._ck(lib.sm_batch_ptrs(h, C.byref(phi), C.byref(rhs), _hp(self.offsets)))
        self.cells = int(np.sum(self.sides.astype(np.int64) ** 3))
        # grids start on aligned offsets: the arrays span the last grid's end
        length = int(self.offsets[-1] + int(self.sides[-1]) ** 3)
        self.phi = self._view(phi.value, length)
        self.rhs = self._view(rhs.value, length)

    def _ck(self, rc):
        if rc != SM_OK:
            raise SmError(rc, self._lib.sm_batch_last_error(self._h).decode())
        return rc

    def _view(self, ptr, count):
        off = ptr - self.arena.data_ptr()
        return self.arena[off:off + 8 * count].view(self.torch.float64)

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.sm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def grid(self, t, s):
        """Solve s's grid [z][y][x] as a view of flat device array t."""
        n = int(self.sides[s])
        o = int(self.offsets[s])
        return t[o:o + n ** 3].view(n, n, n)

    def solve(self, tol=1e-8, max_cycles=50, allow_noconv=True):
        cyc = np.zeros(self.n, np.int32)
        rel = np.zeros(self.n, np.float64)
        rc = self._lib.sm_batch_solve(self._h, tol, max_cycles, _hp(cyc), _hp(rel))
        if rc != SM_OK and not (allow_noconv and rc == SM_ENOCONV):
            self._ck(rc)
        return rc, cyc, rel

    def tune(self, iters=3):
        s, g, ms = C.c_int(), C.c_int(), C.c_double()
        self._ck(self._lib.sm_batch_tune(self._h, iters, C.byref(s), C.byref(g), C.byref(ms)))
        return s.value, g.value, ms.value

    def set_schedule(self, shape, grid_mult):
        self._ck(self._lib.sm_batch_set_schedule(self._h, shape, grid_mult))

    def set_graphs(self, enable: bool):
        self._ck(self._lib.sm_batch_set_graphs(self._h, int(enable)))

    def kernel_bench(self, kclass: int, reps: int = 10):
        """(microseconds per launch, algorithmic bytes, FP64 operations per
        launch) of a kernel class of the batched cycle (0 level-0 sweep,
        1 FP64 outer residual, 2 level-0 prolongation, 3 restriction)."""
        us, by, fl = C.c_double(), C.c_double(), C.c_double()
        self._ck(self._lib.sm_batch_kernel_bench(self._h, kclass, reps, C.byref(us), C.byref(by), C.byref(fl)))
        return us.value, by.value, fl.value

    def info(self):
        c, lv, nl = C.c_longlong(), C.c_int(), C.c_longlong()
        self._ck(self._lib.sm_batch_info(self._h, C.byref(c), C.byref(lv), C.byref(nl)))
        return c.value, lv.value, nl.value


CNN_PARAMS = 8241


class Network:
    """The learned warm-start network (weights, samples, training)."""

    def __init__(self, max_samples=4096, max_boxes=4096, stream=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise SmError(SM_ECUDA, "no CUDA device")
        self._lib, self.torch = lib, torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = lib.sm_cnn_create(C.byref(h), max_samples, max_boxes, C.c_void_p(self.stream.cuda_stream))
        if rc != SM_OK:
            raise SmError(rc, "sm_cnn_create failed")
        self._h = h
        size = C.c_size_t()
        self._ck(lib.sm_cnn_arena_size(h, C.byref(size)))
        self.arena = torch.empty(size.value, dtype=torch.uint8, device="cuda")
        self._ck(lib.sm_cnn_bind_arena(h, C.c_void_p(self.arena.data_ptr()), size.value))

    def _ck(self, rc):
        if rc != SM_OK:
            raise SmError(rc, self._lib.sm_cnn_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.sm_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        self._ck(self._lib.sm_cnn_set_params(self._h, _hp(a), a.size))

    def get_params(self):
        a = np.zeros(CNN_PARAMS, np.float32)
        self._ck(self._lib.sm_cnn_get_params(self._h, _hp(a), a.size))
        return a

    def forward(self, x, acts=False):
        """x: [n][1000][2] float32 (position-major); returns out [n][512]
        and, with acts, [min(n,16)][4][16][512] = z1, a1, z2, a2."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = x.shape[0]
        out = np.zeros((n, 512), np.float32)
        ac = np.zeros((min(n, 16), 4, 16, 512), np.float32) if acts else None
        self._ck(self._lib.sm_cnn_forward(self._h, _hp(x), n, _hp(out), _hp(ac) if acts else None))
        return (out, ac) if acts else out

    def gradient(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(CNN_PARAMS, np.float32)
        loss = C.c_float()
        self._ck(self._lib.sm_cnn_gradient(self._h, _hp(x), _hp(t), x.shape[0], _hp(g), C.byref(loss)))
        return g, loss.value

    def load_samples(self, x, t):
        """Explicit (input, target) pairs ([n][1000][2], [n][512]) as the
        recorded samples that train() and kernel_bench() use."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        self._ck(self._lib.sm_cnn_load_samples(self._h, _hp(x), _hp(t), x.shape[0]))

    def adam_step(self, g, lr):
        g = np.ascontiguousarray(g, dtype=np.float32)
        self._ck(self._lib.sm_cnn_adam_step(self._h, _hp(g), lr))

    def train(self, epochs, batch, lr, seed=0x5EED):
        loss = C.c_float()
        self._ck(self._lib.sm_cnn_train(self._h, epochs, batch, lr, seed, C.byref(loss)))
        return loss.value

    def attach(self, solver, mode, per_solve=512, stride=1, taper=False, accept=1.0):
        self._ck(self._lib.sm_cnn_attach(solver._h, self._h, mode, per_solve, stride, int(taper), accept))

    def kernel_bench(self, kind: int, n: int, reps: int = 10):
        """(us per launch, model FLOPs, tensor-core FLOPs) of the forward
        kernel (kind 0) or a training gradient pass (kind 1) over the first n
        recorded samples."""
        us, fl, tf = C.c_double(), C.c_double(), C.c_double()
        self._ck(self._lib.sm_cnn_kernel_bench(self._h, kind, n, reps, C.byref(us), C.byref(fl), C.byref(tf)))
        return us.value, fl.value, tf.value

    def stats(self):
        n, p, k = C.c_int(), C.c_longlong(), C.c_longlong()
        rel = (C.c_double * 2)()
        self._ck(self._lib.sm_cnn_stats(self._h, C.byref(n), C.byref(p), C.byref(k), rel))
        return {"samples": n.value, "predictions": p.value, "kept": k.value, "last_rel": (rel[0], rel[1])}


class _QuadDomain(C.Structure):
    _fields_ = [("length", C.c_double), ("origin", C.c_double * 2), ("nb", C.c_int),
                ("max_level", C.c_int), ("geometry", C.c_int), ("bc_type", C.c_int * 4),
                ("bc_val", C.c_double * 4)]


class Quad:
    """A quadtree of 8^2-cell boxes with its fields on the current CUDA
    device: the 2-D (geometry 0) or axisymmetric (geometry 1) variant."""

    def __init__(self, dom, max_boxes: int, nu1: int = 2, nu2: int = 2, stream=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise SmError(SM_ECUDA, "no CUDA device")
        self._lib, self.torch, self.dom = lib, torch, dom
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d = _QuadDomain(dom.length, (C.c_double * 2)(*dom.origin), dom.nb, dom.max_level, dom.geom,
                        (C.c_int * 4)(*dom.bc_type), (C.c_double * 4)(*dom.bc_val))
        h = C.c_void_p()
        rc = lib.sm_quad_create(C.byref(h), C.byref(d), int(max_boxes), nu1, nu2,
                                C.c_void_p(self.stream.cuda_stream))
        if rc != SM_OK:
            raise SmError(rc, "sm_quad_create failed")
        self._h = h
        size = C.c_size_t()
        self._ck(lib.sm_quad_arena_size(h, C.byref(size)))
        self.arena = torch.empty(size.value, dtype=torch.uint8, device="cuda")
        self._ck(lib.sm_quad_bind_arena(h, C.c_void_p(self.arena.data_ptr()), size.value))
        self.max_boxes = int(max_boxes)

    def _ck(self, rc):
        if rc not in (SM_OK, SM_ENOCONV):
            raise SmError(rc, self._lib.sm_quad_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.sm_quad_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tables ----
    def counts(self):
        nb, nl = C.c_int(), C.c_int()
        self._ck(self._lib.sm_quad_get_tables(self._h, C.byref(nb), C.byref(nl), *([None] * 7)))
        return nb.value, nl.value

    @property
    def n_boxes(self) -> int:
        return self.counts()[0]

    @property
    def n_levels(self) -> int:
        return self.counts()[1]

    def tables(self) -> dict:
        n, nl = self.counts()
        t = {"level_offset": np.zeros(nl + 1, np.int32), "level": np.zeros(n, np.int32),
             "ij": np.zeros((n, 2), np.int32), "morton": np.zeros(n, np.uint64),
             "parent": np.zeros(n, np.int32), "child": np.zeros((n, 4), np.int32),
             "nbr": np.zeros((n, 8), np.int32)}
        self._ck(self._lib.sm_quad_get_tables(self._h, None, None, *(_hp(t[k]) for k in (
            "level_offset", "level", "ij", "morton", "parent", "child", "nbr"))))
        return t

    def level_ij(self, level: int) -> np.ndarray:
        t = self.tables()
        if level >= len(t["level_offset"]) - 1:
            return np.zeros((0, 2), np.int32)
        return t["ij"][t["level_offset"][level]:t["level_offset"][level + 1]]

    def refine_level(self, level: int, flags) -> int:
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        new, dropped = C.c_int(), C.c_int()
        self._ck(self._lib.sm_quad_refine_level(self._h, level, _hp(flags), C.byref(new), C.byref(dropped)))
        self.dropped = dropped.value
        return new.value

    # ---- fields ----
    def upload(self, var: int, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.n_boxes, 64)
        self._ck(self._lib.sm_quad_upload(self._h, var, _hp(a)))

    def download(self, var: int) -> np.ndarray:
        a = np.zeros((self.n_boxes, 64), np.float64)
        self._ck(self._lib.sm_quad_download(self._h, var, _hp(a)))
        return a

    def view(self, var: int):
        """[n_boxes][64] device tensor view of a field (no copy)."""
        ptr = C.c_void_p()
        self._ck(self._lib.sm_quad_var_ptr(self._h, var, C.byref(ptr)))
        off = ptr.value - self.arena.data_ptr()
        n = self.n_boxes
        return self.arena[off:off + 8 * 64 * n].view(self.torch.float64).view(n, 64)

    def set_table(self, tab: dict):
        mu = np.ascontiguousarray(tab["mu"], np.float64)
        dc = np.ascontiguousarray(tab["diff"], np.float64)
        al = np.ascontiguousarray(tab["alpha"], np.float64)
        self._ck(self._lib.sm_quad_set_table(self._h, len(mu), float(tab["e_max"]), _hp(mu), _hp(dc), _hp(al)))

    # ---- operations ----
    def charge_rhs(self, q=1.0, eps=1.0, use_rho=False):
        self._ck(self._lib.sm_quad_charge_rhs(self._h, q, eps, int(use_rho)))

    def fmg(self, tol=1e-8, max_cycles=50):
        cyc, rel = C.c_int(), C.c_double()
        rc = self._ck(self._lib.sm_quad_fmg(self._h, tol, max_cycles, C.byref(cyc), C.byref(rel)))
        return rc, rel.value, cyc.value

    def solve(self, tol=1e-8, max_cycles=50):
        cyc, rel = C.c_int(), C.c_double()
        rc = self._ck(self._lib.sm_quad_solve(self._h, tol, max_cycles, C.byref(cyc), C.byref(rel)))
        return rc, rel.value, cyc.value

    def vcycles(self, n: int):
        """n V-cycles, enqueued on the stream (no residual evaluation)."""
        self._ck(self._lib.sm_quad_vcycles(self._h, int(n)))

    def compute_field(self):
        self._ck(self._lib.sm_quad_compute_field(self._h))

    def dt_limit(self, q, eps) -> float:
        dt = C.c_double()
        self._ck(self._lib.sm_quad_dt_limit(self._h, q, eps, C.byref(dt)))
        return dt.value

    def fluid_stage(self, dt):
        self._ck(self._lib.sm_quad_fluid_stage(self._h, dt))

    def advance(self, dt, q, eps, tol=1e-8, max_cycles=50):
        dtn = C.c_double()
        cyc = np.zeros(2, np.int32)
        rc = self._ck(self._lib.sm_quad_advance(self._h, dt, q, eps, tol, max_cycles, C.byref(dtn), _hp(cyc)))
        return rc, dtn.value, int(cyc[0]), int(cyc[1])

    def refine_flags(self, c0=1.0, c1=1.2, c0_deref=0.125, dx_deref=30e-6, buffer=3) -> np.ndarray:
        """Per-box flags from the stored |E| (Eq. 8): +1 refine, -1 derefinable, 0."""
        f = np.zeros(self.n_boxes, np.int8)
        self._ck(self._lib.sm_quad_refine_flags(self._h, c0, c1, c0_deref, dx_deref, int(buffer), _hp(f)))
        return f

    def regrid(self, flags):
        """Apply per-box flags; returns (refined, derefined, dropped)."""
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.n_boxes,)
        r, d, x = C.c_int(), C.c_int(), C.c_int()
        self._ck(self._lib.sm_quad_regrid(self._h, _hp(flags), C.byref(r), C.byref(d), C.byref(x)))
        return r.value, d.value, x.value

    def set_graphs(self, on: bool):
        self._ck(self._lib.sm_quad_set_graphs(self._h, int(bool(on))))

    def set_pdl(self, on: bool):
        self._ck(self._lib.sm_quad_set_pdl(self._h, int(bool(on))))

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._ck(self._lib.sm_quad_launch_count(self._h, C.byref(n)))
        return n.value
