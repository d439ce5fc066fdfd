"""The allocation-free entry point sm_box_solve_noalloc, called through the
C ABI, against the existing path that solves the same single-box problem
(sm_mg_fmg on a one-box domain, whose whole solve is the exact level-0
solve).  Callers that cannot allocate device memory use this entry point;
its scratch is a fixed device array shared by all calls, so two calls in a
row with different inputs must both be right.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_box_solve_matches_fmg_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_08434_gb300 as pkg
    lib = pkg.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(20261202)
    length = 0.37
    vp = lambda t: C.c_void_p(t.data_ptr())
    for call in range(2):
        n = 7 + call
        bct = rng.integers(0, 2, size=(n, 6)).astype(np.int32)
        bct[np.arange(n), rng.integers(0, 6, n)] = 1          # at least one Dirichlet face
        bcv = rng.uniform(-2.0, 2.0, size=(n, 6))
        f = rng.standard_normal((n, 512)) * (10.0 ** call)
        d_bct = torch.from_numpy(bct).cuda()
        d_bcv = torch.from_numpy(bcv).cuda()
        d_f = torch.from_numpy(f).cuda()
        d_phi = torch.full((n, 512), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.sm_box_solve_noalloc(length, n, vp(d_bct), vp(d_bcv), vp(d_f), vp(d_phi),
                                      C.c_void_p(stream.cuda_stream))
        assert rc == pkg.SM_OK
        stream.synchronize()
        got = d_phi.cpu().numpy()
        for p in range(n):
            dom = synth.Domain(length=length, nb=1, max_level=0, bc_type=tuple(int(x) for x in bct[p]),
                               bc_val=tuple(float(x) for x in bcv[p]))
            s = pkg.Solver(dom, max_boxes=1)
            s.build_octree()
            s.upload(pkg.RHO, -f[p:p + 1])
            s.charge_rhs(1.0, 1.0, True)
            s.fmg(1e-12, 1)
            want = s.download(pkg.PHI)[0]
            s.close()
            err = np.abs(got[p] - want).max() / np.abs(want).max()
            assert err <= TOL, (call, p, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1708_08434_gb300 as pkg
    lib = pkg.load()
    z = C.c_void_p(0)
    assert lib.sm_box_solve_noalloc(1.0, 1025, z, z, z, z, None) == pkg.SM_ENOMEM
    assert lib.sm_box_solve_noalloc(1.0, -1, z, z, z, z, None) == pkg.SM_EINVAL
    assert lib.sm_box_solve_noalloc(1.0, 0, z, z, z, z, None) == pkg.SM_OK
