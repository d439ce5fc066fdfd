"""Batched form: many independent uniform solves of uneven sizes in one
set of launches per level.  Reference: the exact discrete solution by
separable transforms (oracle/spectral.py).  Bound: 1e-6 relative on each
potential at a converged residual of 1e-8 (the mixed-precision bound)."""
import numpy as np
import pytest

import synth
from oracle import spectral

pytestmark = pytest.mark.gpu
BCT = (0, 0, 0, 0, 1, 1)
BCV = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def make_batch(sides, seed_blobs=0, keep=None):
    """Batch with the seeded blob charges; returns the charges of the solves
    in `keep` (all when None)."""
    import torch
    import paper_1708_08434_gb300 as pkg
    b = pkg.Batch(sides, 1.0, BCT, BCV)
    blobs = synth.batch_blobs(len(sides) + seed_blobs)[seed_blobs:]
    rhos = {}
    for s, n in enumerate(sides):
        rho = synth.blob_rho(int(n), blobs[s])
        if keep is None or s in keep:
            rhos[s] = rho
        b.grid(b.rhs, s).copy_(torch.from_numpy(-rho))
    b.phi.zero_()
    return b, rhos


def check(b, rhos, sel, bound):
    for s in sel:
        ref = spectral.solve(-rhos[s], 1.0, BCT, BCV)
        got = b.grid(b.phi, s).cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= bound, (s, b.sides[s], err)


def test_batch_uneven_sizes_against_spectral():
    sides = [32, 40, 48, 56, 24, 16, 8, 72, 88, 64, 15]   # 15: odd, scalar loads
    b, rhos = make_batch(sides)
    rc, cyc, rel = b.solve(1e-8, 40)
    assert rc == 0 and np.all(rel <= 1e-8)
    assert len(set(cyc.tolist())) > 1            # solves stop at different cycles
    check(b, rhos, range(len(sides)), 1e-6)
    # tighter tolerance from the converged state: error follows
    rc, cyc2, rel2 = b.solve(1e-11, 40)
    assert rc == 0
    check(b, rhos, range(len(sides)), 1e-9)


def test_batch_odd_and_unaligned_sizes():
    """Sides that are odd (finest grid = coarsest, exact solve only) or
    2 mod 4 (rows not 16-byte aligned: element-wise staging), mixed with
    aligned ones placed right after odd-sized grids (their starts must be
    padded to stay aligned); Dirichlet on four faces."""
    import torch
    import paper_1708_08434_gb300 as pkg
    sides = [15, 32, 9, 18, 20, 12, 26, 44]
    bct, bcv = (1, 0, 0, 1, 1, 1), (0.5, 0.0, 0.0, -0.25, 0.0, 1.0)
    b = pkg.Batch(sides, 1.0, bct, bcv)
    blobs = synth.batch_blobs(len(sides) + 7)[7:]
    rhos = {}
    for s, n in enumerate(sides):
        rhos[s] = synth.blob_rho(int(n), blobs[s])
        b.grid(b.rhs, s).copy_(torch.from_numpy(-rhos[s]))
    b.phi.zero_()
    rc, cyc, rel = b.solve(1e-9, 40)
    assert rc == 0 and np.all(rel <= 1e-9)
    for s in range(len(sides)):
        ref = spectral.solve(-rhos[s], 1.0, bct, bcv)
        got = b.grid(b.phi, s).cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-7, (s, sides[s], err)
    b.close()


@pytest.mark.parametrize("nu1,nu2", [(3, 1), (1, 3)])
def test_batch_odd_sweep_counts(nu1, nu2):
    """Odd numbers of sweeps: the error ends in the second buffer and is
    copied back (pre-smoothing), or the last level-0 sweep is an odd one
    (post-smoothing); same exact-solution bound."""
    import torch
    import paper_1708_08434_gb300 as pkg
    sides = [32, 40, 16, 56]
    b = pkg.Batch(sides, 1.0, BCT, BCV, nu1=nu1, nu2=nu2)
    blobs = synth.batch_blobs(len(sides) + 9)[9:]
    rhos = {}
    for s, n in enumerate(sides):
        rhos[s] = synth.blob_rho(int(n), blobs[s])
        b.grid(b.rhs, s).copy_(torch.from_numpy(-rhos[s]))
    b.phi.zero_()
    rc, cyc, rel = b.solve(1e-9, 60)
    assert rc == 0 and np.all(rel <= 1e-9)
    check(b, rhos, range(len(sides)), 1e-7)
    b.close()


def test_batch_autotune_keeps_results():
    sides = [40, 48, 32, 56]
    b, rhos = make_batch(sides, seed_blobs=3)
    shape, gmult, ms = b.tune(2)
    assert 0 <= shape < 5 and gmult in (2, 4, 8, 16, 32) and ms > 0
    rc, cyc, rel = b.solve(1e-9, 40)
    assert rc == 0
    check(b, rhos, range(len(sides)), 1e-7)
    # every schedule gives the same potential to roundoff of FP32 cycles
    ref = b.phi.clone()
    for sh in range(5):
        b.set_schedule(sh, 2)
        b.phi.zero_()
        b.solve(1e-9, 40)
        d = (b.phi - ref).abs().max().item() / ref.abs().max().item()
        assert d <= 1e-7


def test_batch_column_restriction_on_full_waves():
    """Schedule 4 marches fine columns only on levels with at least four
    columns per SM: enough 128^3 solves that level 0 has them (32 columns
    each) while the coarser levels fall back to 8^3 tiles."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n128 = -(-4 * sms // 32)
    sides = [128] * n128 + [40, 56]
    b, rhos = make_batch(sides, seed_blobs=5, keep={0, n128 - 1, n128 + 1})
    b.set_schedule(0, 4)
    rc, _, rel = b.solve(1e-9, 40)
    assert rc == 0 and np.all(rel <= 1e-9)
    ref = b.phi.clone()
    b.set_schedule(4, 4)
    b.phi.zero_()
    rc, _, rel = b.solve(1e-9, 40)
    assert rc == 0 and np.all(rel <= 1e-9)
    d = (b.phi - ref).abs().max().item() / ref.abs().max().item()
    assert d <= 1e-7
    check(b, rhos, (0, n128 - 1, n128 + 1), 1e-6)
    b.close()


def test_batch_column_restriction_scalar_copies():
    """Grids of side 30 (N % 4 != 0) stage their planes with 4-byte copies;
    enough of them (two columns each) that level 0 gets the column
    restriction."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n30 = -(-4 * sms // 2)
    sides = [30] * n30
    b, rhos = make_batch(sides, seed_blobs=9, keep={0, n30 // 2, n30 - 1})
    b.set_schedule(0, 4)
    rc, _, rel = b.solve(1e-9, 40)
    assert rc == 0 and np.all(rel <= 1e-9)
    ref = b.phi.clone()
    b.set_schedule(4, 4)
    b.phi.zero_()
    rc, _, rel = b.solve(1e-9, 40)
    assert rc == 0 and np.all(rel <= 1e-9)
    d = (b.phi - ref).abs().max().item() / ref.abs().max().item()
    assert d <= 1e-7
    check(b, rhos, (0, n30 // 2, n30 - 1), 1e-6)
    b.close()


def test_batch_rejects_too_large_coarsest():
    import paper_1708_08434_gb300 as pkg
    with pytest.raises(pkg.SmError):
        pkg.Batch([136], 1.0, BCT, BCV)   # 136 -> 68 -> 34 -> 17 > 16


@pytest.mark.slow
def test_batch_full_size_sampled():
    """256 solves of 32^3..128^3 (1.3e8 cells): every solve reaches 1e-8;
    sampled solves (including the largest) against the spectral reference."""
    sides = synth.batch_sizes(256)
    big = int(np.argmax(sides))
    sample = sorted({0, 17, 99, 200, big})
    b, rhos = make_batch(sides, keep=set(sample))
    rc, cyc, rel = b.solve(1e-8, 40)
    assert rc == 0 and np.all(rel <= 1e-8)
    check(b, rhos, sample, 1e-6)


def test_batch_graph_and_host_paths_identical():
    sides = [40, 32, 8, 56]
    out = []
    for graphs in (True, False):
        b, rhos = make_batch(sides, seed_blobs=5)
        b.set_graphs(graphs)
        rc, cyc, rel = b.solve(1e-9, 40)
        out.append((cyc.copy(), rel.copy(), b.phi.cpu().numpy()))
        b.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


def test_batch_mixed_starting_potentials():
    """The first residual pass skips solves whose stored potential is all +0
    (their residual is that of phi = 0, already computed for the
    denominators).  In one batch: solves restarted from +0, solves kept at a
    converged potential, and one restarted from -0.0 (not all +0 bits, so
    it takes the full pass).  A solve restarted from +0 gives the same bits
    as in a batch where every solve starts from +0; all reach the tolerance
    and the spectral reference."""
    sides = [32, 40, 24, 48]
    fresh, rhos = make_batch(sides, seed_blobs=3)
    rc, cyc_f, rel_f = fresh.solve(1e-10, 40)
    assert rc == 0
    phi_f = [fresh.grid(fresh.phi, s).cpu().numpy().copy() for s in range(len(sides))]
    fresh.close()

    b, _ = make_batch(sides, seed_blobs=3)
    rc, _, _ = b.solve(1e-8, 40)
    assert rc == 0
    b.grid(b.phi, 1).zero_()
    b.grid(b.phi, 3).fill_(-0.0)
    rc, cyc, rel = b.solve(1e-10, 40)
    assert rc == 0 and np.all(rel <= 1e-10)
    assert np.array_equal(b.grid(b.phi, 1).cpu().numpy(), phi_f[1])
    assert cyc[1] == cyc_f[1] and rel[1] == rel_f[1]
    # converged starts need fewer corrections than the restarts
    assert cyc[0] < cyc_f[0] and cyc[2] < cyc_f[2]
    check(b, rhos, range(len(sides)), 1e-8)
    b.close()


def test_repeatable_bits_batch64():
    """The first 64 solves of the workload solved on two fresh batches (the
    tuned schedule, captured graph) give the same bits."""
    sides = synth.batch_sizes(256)[:64]
    out, sched = [], None
    for _ in range(2):
        b, _ = make_batch(sides)
        if sched is None:
            sched = b.tune(1)[:2]
        b.set_schedule(*sched)
        b.phi.zero_()
        rc, cyc, rel = b.solve(1e-8, 30)
        assert rc == 0
        out.append((cyc.copy(), b.phi.cpu().numpy().view(np.int64).copy()))
        b.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
