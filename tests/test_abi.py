"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/sm_streamer.h declares; argument checks that need no
device work reject bad input.  No compute calls are made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "sm_streamer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_08434_gb300 import _build
    import paper_1708_08434_gb300 as pkg
    _build.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 20
    import paper_1708_08434_gb300 as pkg
    assert sorted(pkg.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_library_is_sm103a_only():
    from paper_1708_08434_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_rejects_bad_domains(lib):
    import paper_1708_08434_gb300 as pkg
    cfg = pkg._Config(4096, 2, 2, 0)
    base = dict(length=1.0, origin=(C.c_double * 3)(0, 0, 0), nb=4, max_level=2,
                bc_type=(C.c_int * 6)(0, 0, 0, 0, 1, 1), bc_val=(C.c_double * 6)(0, 0, 0, 0, 0, 1))
    h = C.c_void_p()
    for change in (dict(nb=3), dict(nb=0), dict(max_level=-1), dict(max_level=40),
                   dict(bc_type=(C.c_int * 6)(0, 0, 0, 0, 0, 0)), dict(length=-1.0)):
        d = pkg._Domain(**{**base, **change})
        assert lib.sm_create(C.byref(h), C.byref(cfg), C.byref(d), None) == pkg.SM_EINVAL
    d = pkg._Domain(**base)
    for bad in (pkg._Config(10, 2, 2, 0), pkg._Config(4096, 0, 2, 0), pkg._Config(4096, 2, 2, 7)):
        assert lib.sm_create(C.byref(h), C.byref(bad), C.byref(d), None) == pkg.SM_EINVAL


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1708_08434_gb300 as pkg
    cfg = pkg._Config(4096, 2, 2, 0)
    d = pkg._Domain(1.0, (C.c_double * 3)(0, 0, 0), 4, 2, (C.c_int * 6)(0, 0, 0, 0, 1, 1),
                    (C.c_double * 6)(0, 0, 0, 0, 0, 1))
    h = C.c_void_p()
    assert lib.sm_create(C.byref(h), C.byref(cfg), C.byref(d), None) == pkg.SM_ECUDA
    with pytest.raises(pkg.SmError):
        pkg.Solver(__import__("synth").domain_uniform_cube(32), 4096)
