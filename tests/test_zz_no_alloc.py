"""The allocation-free entry point sm_box_solve_noalloc, called through the
C ABI, against the existing path that solves the same single-box problem
(sm_mg_fmg on a one-box domain, whose whole solve is the exact level-0
solve) and against the CPU oracle's dense LU solve of that box.  Callers
that cannot allocate device memory use this entry point; its scratch is a
fixed device array shared by all calls, so two calls in a row with
different inputs must both be right.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08434_gb300 as pkg
    torch.cuda.set_device(0)
    return pkg, pkg.load()


def _call(pkg, lib, length, bct, bcv, f):
    import torch
    stream = torch.cuda.current_stream()
    n = len(bct)
    vp = lambda t: C.c_void_p(t.data_ptr())
    d_bct = torch.from_numpy(np.ascontiguousarray(bct, np.int32)).cuda()
    d_bcv = torch.from_numpy(np.ascontiguousarray(bcv, np.float64)).cuda()
    d_f = torch.from_numpy(np.ascontiguousarray(f, np.float64)).cuda()
    d_phi = torch.full((n, 512), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.sm_box_solve_noalloc(length, n, vp(d_bct), vp(d_bcv), vp(d_f), vp(d_phi),
                                  C.c_void_p(stream.cuda_stream))
    assert rc == pkg.SM_OK
    stream.synchronize()
    return d_phi.cpu().numpy()


def _fmg_and_oracle(pkg, length, bct, bcv, f):
    """phi of one box by the GPU's one-box FMG and by the oracle's dense LU."""
    dom = synth.Domain(length=length, nb=1, max_level=0, bc_type=tuple(int(x) for x in bct),
                       bc_val=tuple(float(x) for x in bcv))
    s = pkg.Solver(dom, max_boxes=1)
    s.build_octree()
    s.upload(pkg.RHO, -f[None, :])
    s.charge_rhs(1.0, 1.0, True)
    s.fmg(1e-12, 1)
    gpu = s.download(pkg.PHI)[0]
    s.close()
    o = oracle.Oracle(dom)
    o.set(oracle.RHO, -f[None, :])
    o.charge_rhs(1.0, 1.0, True)
    o.fmg(1e-12, 1)
    return gpu, o.get(oracle.PHI)[0]


def test_noalloc_box_solve_matches_fmg_and_oracle_twice():
    pkg, lib = _lib()
    rng = np.random.default_rng(20261202)
    length = 0.37
    for call in range(2):
        n = 7 + call
        bct = rng.integers(0, 2, size=(n, 6)).astype(np.int32)
        bct[np.arange(n), rng.integers(0, 6, n)] = 1          # at least one Dirichlet face
        bcv = rng.uniform(-2.0, 2.0, size=(n, 6))
        f = rng.standard_normal((n, 512)) * (10.0 ** call)
        got = _call(pkg, lib, length, bct, bcv, f)
        for p in range(n):
            want, ref = _fmg_and_oracle(pkg, length, bct[p], bcv[p], f[p])
            err = np.abs(got[p] - want).max() / np.abs(want).max()
            assert err <= TOL, (call, p, err)
            # the oracle's level-0 solve is a dense LU of the same operator
            err_o = np.abs(got[p] - ref).max() / np.abs(ref).max()
            assert err_o <= TOL, (call, p, err_o)


def _laplacian_neumann(phi, h):
    """7-point cell-centred Laplacian of one 8^3 box, every face Neumann
    zero (ghost = inner value)."""
    u = phi.reshape(8, 8, 8)  # [k][j][i]
    p = np.pad(u, 1, mode="edge")
    s = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1] +
         p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] - 6.0 * u)
    return (s / (h * h)).reshape(512)


def test_noalloc_all_neumann_and_full_scratch():
    """A problem without a Dirichlet face (zero-mean f) gets the solution of
    zero mean that satisfies L phi = f; a call with the largest problem count
    uses the last scratch slot and still matches the oracle there."""
    pkg, lib = _lib()
    rng = np.random.default_rng(7)
    length = 1.0
    n = 1024
    bct = rng.integers(0, 2, size=(n, 6)).astype(np.int32)
    bct[np.arange(n), rng.integers(0, 6, n)] = 1
    bct[0] = 0                                                # all Neumann
    bcv = rng.uniform(-1.0, 1.0, size=(n, 6))
    f = rng.standard_normal((n, 512))
    f[0] -= f[0].mean()
    got = _call(pkg, lib, length, bct, bcv, f)
    assert abs(got[0].mean()) <= 1e-12 * np.abs(got[0]).max()
    lap = _laplacian_neumann(got[0], length / 8)
    assert np.abs(lap - f[0]).max() <= 1e-9 * np.abs(f[0]).max()
    for p in (n - 2, n - 1):
        _, ref = _fmg_and_oracle(pkg, length, bct[p], bcv[p], f[p])
        assert np.abs(got[p] - ref).max() <= TOL * np.abs(ref).max(), p


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pkg, lib = _lib()
    z = C.c_void_p(0)
    assert lib.sm_box_solve_noalloc(1.0, 1025, z, z, z, z, None) == pkg.SM_ENOMEM
    assert lib.sm_box_solve_noalloc(1.0, -1, z, z, z, z, None) == pkg.SM_EINVAL
    assert lib.sm_box_solve_noalloc(1.0, 0, z, z, z, z, None) == pkg.SM_OK
