"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/*.h declares; argument checks that need no
device work reject bad input.  No compute calls are made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
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


def prototypes():
    """{name: [parameter type class, ...]} of every prototype in include/*.h
    (a pointer of any type is "ptr")."""
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    scalar = {"int": "i32", "double": "f64", "float": "f32", "long long": "i64",
              "unsigned long long": "u64", "size_t": "u64"}
    out = {}
    for name, params in re.findall(r"\b(?:int|const\s+char\s*\*)\s*(sm_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", src):
        kinds = []
        for p in params.split(","):
            p = " ".join(p.split())
            if not p or p == "void":
                continue
            if "*" in p:
                kinds.append("ptr")
                continue
            words = p.replace("const ", "").split()
            assert " ".join(words[:-1]) in scalar, (name, p)
            kinds.append(scalar[" ".join(words[:-1])])
        out[name] = kinds
    return out


def ctypes_kind(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    for kind, types in (("i32", (C.c_int,)), ("f64", (C.c_double,)), ("f32", (C.c_float,)),
                        ("i64", (C.c_longlong,)), ("u64", (C.c_ulonglong, C.c_size_t))):
        if t in types:
            return kind
    raise AssertionError(t)


def test_binding_signatures_match_the_headers():
    """Every ctypes signature of the binding has the parameter count and
    the scalar types of its prototype (a mismatch would pass garbage
    through the C ABI without any error)."""
    import paper_1708_08434_gb300 as pkg
    protos = prototypes()
    sigs = pkg.signatures()
    assert sorted(protos) == sorted(sigs) == sorted(pkg.EXPORTS)
    for name, kinds in protos.items():
        assert [ctypes_kind(t) for t in sigs[name]] == kinds, name


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


def test_quad_create_rejects_bad_domains(lib):
    """sm_quad_create validates its arguments before touching a device."""
    import paper_1708_08434_gb300 as pkg

    def dom(**kw):
        base = dict(length=1.0, origin=(0.0, 0.0), nb=4, max_level=2, geometry=1,
                    bc_type=(0, 0, 1, 1), bc_val=(0.0, 0.0, 0.0, 1.0))
        base.update(kw)
        return pkg._QuadDomain(base["length"], (C.c_double * 2)(*base["origin"]), base["nb"],
                               base["max_level"], base["geometry"], (C.c_int * 4)(*base["bc_type"]),
                               (C.c_double * 4)(*base["bc_val"]))
    h = C.c_void_p()
    for d in (dom(nb=3), dom(nb=0), dom(max_level=-1), dom(max_level=40), dom(length=0.0),
              dom(geometry=2), dom(origin=(1.0, 0.0)),           # the axis must be at x = 0
              dom(bc_type=(1, 0, 0, 0)),                          # only the axis is Dirichlet
              dom(bc_type=(0, 0, 2, 1))):
        assert lib.sm_quad_create(C.byref(h), C.byref(d), 4096, 2, 2, None) == pkg.SM_EINVAL
    good = dom()
    for mb, nu1, nu2 in ((20, 2, 2), (4096, 0, 2), (4096, 2, 0)):  # 21 uniform boxes needed
        assert lib.sm_quad_create(C.byref(h), C.byref(good), mb, nu1, nu2, None) == pkg.SM_EINVAL
