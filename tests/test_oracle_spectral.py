"""Pins of the spectral reference used for the batched solves: it agrees
with the C oracle's multigrid (an unrelated method) on power-of-two grids,
reproduces closed-form discrete eigenvectors on uneven sizes, and its
residual stencil agrees with the C oracle's residual."""
import numpy as np
import pytest

import oracle
import synth
from oracle import spectral

BCT = (0, 0, 0, 0, 1, 1)


def to_boxes(a, nb):
    """[z][y][x] array of a uniform grid -> oracle box order [box][512] for a
    uniform level (Morton box order, x-fastest cells)."""
    out = np.zeros((nb ** 3, 512))
    for key in range(nb ** 3):
        i = j = k = 0
        for b in range(10):
            i |= ((key >> (3 * b)) & 1) << b
            j |= ((key >> (3 * b + 1)) & 1) << b
            k |= ((key >> (3 * b + 2)) & 1) << b
        out[key] = a[8 * k:8 * k + 8, 8 * j:8 * j + 8, 8 * i:8 * i + 8].reshape(512)
    return out


@pytest.mark.parametrize("n", [32, 64])
def test_spectral_matches_c_oracle_multigrid(n):
    blobs = synth.batch_blobs(1)[0]
    rho = synth.blob_rho(n, blobs)
    phi = spectral.solve(-rho, 1.0, BCT, (0, 0, 0, 0, 0, 1.0))
    dom = synth.domain_uniform_cube(n)
    o = oracle.Oracle(dom)
    lo, hi = o.level_range(o.n_levels - 1)
    full = np.zeros((o.n_boxes, 512))
    full[lo:hi] = to_boxes(rho, n // 8)
    o.set(oracle.RHO, full)
    o.charge_rhs(1.0, 1.0, True)
    o.fmg(1e-13, 60)
    mg = o.get(oracle.PHI)[lo:hi]
    ref = to_boxes(phi, n // 8)
    assert np.abs(mg - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("n,bct", [(40, (0, 0, 1, 1, 1, 0)), (24, (1, 0, 0, 0, 1, 1)), (13, (1, 1, 1, 1, 1, 1)),
                                   (20, (0, 1, 1, 0, 0, 1))])   # last: Neumann low, Dirichlet high
def test_spectral_reproduces_eigenvector(n, bct):
    i = np.arange(n) + 0.5
    def vec(lo, hi, p):
        if not lo and not hi:
            return np.cos(np.pi * p * i / n), -4 * np.sin(np.pi * p / (2 * n)) ** 2
        if lo and hi:
            return np.sin(np.pi * p * i / n), -4 * np.sin(np.pi * p / (2 * n)) ** 2
        if lo:
            return np.sin(np.pi * (p + 0.5) * i / n), -4 * np.sin(np.pi * (p + 0.5) / (2 * n)) ** 2
        return np.sin(np.pi * (p + 0.5) * (n - i) / n), -4 * np.sin(np.pi * (p + 0.5) / (2 * n)) ** 2
    h = 2.0 / n
    vx, lx = vec(bct[0], bct[1], 2)
    vy, ly = vec(bct[2], bct[3], 1)
    vz, lz = vec(bct[4], bct[5], 3)
    v = vz[:, None, None] * vy[None, :, None] * vx[None, None, :]
    f = (lx + ly + lz) / h ** 2 * v
    phi = spectral.solve(f, 2.0, bct, (0.0,) * 6)
    assert np.abs(phi - v).max() <= 1e-12 * np.abs(v).max()


def test_spectral_residual_matches_c_oracle_residual():
    n = 32
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    bcv = (0, 0, 0, 0, 0.3, 1.7)
    r = spectral.residual(phi, f, 1.0, BCT, bcv)
    dom = synth.Domain(length=1.0, nb=4, max_level=0, bc_val=bcv)
    o = oracle.Oracle(dom)
    lo, hi = o.level_range(o.n_levels - 1)
    F = np.zeros((o.n_boxes, 512))
    F[lo:hi] = to_boxes(-f, 4)
    o.set(oracle.RHO, F)
    o.charge_rhs(1.0, 1.0, True)
    P = np.zeros((o.n_boxes, 512))
    P[lo:hi] = to_boxes(phi, 4)
    o.set(oracle.PHI, P)
    rc = o.composite_residual()[lo:hi]
    assert np.abs(rc - to_boxes(r, 4)).max() <= 1e-9 * np.abs(rc).max()
    # and the exact solution has a roundoff residual
    ps = spectral.solve(f, 1.0, BCT, bcv)
    assert np.abs(spectral.residual(ps, f, 1.0, BCT, bcv)).max() <= 1e-9 * np.abs(f).max()
