"""Exact discrete solve of the 7-point cell-centred Poisson problem on a
uniform n^3 grid by separable transforms (test infrastructure only).

On a uniform grid the discrete operator of Sec. 2.3 (ghost 2g - phi at
Dirichlet faces, phi at Neumann faces) is a Kronecker sum of 1-D operators
whose eigenvectors are DST-II (Dirichlet at both ends), DCT-II (Neumann at
both ends) or quarter-wave sines (mixed); folding the Dirichlet values into
the right-hand side and dividing by the eigenvalues in that basis gives the
exact solution of the linear system the multigrid iterates on.  This is an
independent method (no multigrid, no boxes) used as the reference of the
batched solves; it is pinned in tests/test_oracle_spectral.py against the
C oracle's multigrid and against closed-form eigenvectors.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sf


def _axis_basis(kind: str, n: int):
    """Orthonormal eigenvectors (columns) and h^2-eigenvalues of the 1-D
    3-point operator with the given end types ('N' or 'D' at low, high)."""
    i = np.arange(n) + 0.5
    if kind == "NN":
        p = np.arange(n)
        V = np.cos(np.pi * np.outer(i, p) / n)
        lam = -4 * np.sin(np.pi * p / (2 * n)) ** 2
    elif kind == "DD":
        p = np.arange(1, n + 1)
        V = np.sin(np.pi * np.outer(i, p) / n)
        lam = -4 * np.sin(np.pi * p / (2 * n)) ** 2
    elif kind == "DN":
        p = np.arange(n) + 0.5
        V = np.sin(np.pi * np.outer(i, p) / n)
        lam = -4 * np.sin(np.pi * p / (2 * n)) ** 2
    else:  # ND
        p = np.arange(n) + 0.5
        V = np.sin(np.pi * np.outer(n - i, p) / n)
        lam = -4 * np.sin(np.pi * p / (2 * n)) ** 2
    V = V / np.linalg.norm(V, axis=0)
    return V, lam


def _kind(bct, a):
    return ("D" if bct[2 * a] else "N") + ("D" if bct[2 * a + 1] else "N")


def fold_boundary(f, h, bct, bcv):
    """Right-hand side with the Dirichlet face values moved over."""
    b = np.array(f, dtype=np.float64, copy=True)
    n = b.shape[0]
    for a in range(3):            # array axes are [z][y][x]: x = 2, y = 1, z = 0
        ax = 2 - a
        for side in (0, 1):
            fc = 2 * a + side
            if bct[fc]:
                sl = [slice(None)] * 3
                sl[ax] = n - 1 if side else 0
                b[tuple(sl)] -= 2.0 * bcv[fc] / (h * h)
    return b


def solve(f, length, bct, bcv):
    """phi [z][y][x] solving L phi = f on the n^3 grid of side `length`."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[0]
    h = length / n
    b = fold_boundary(f, h, bct, bcv)
    bases = [_axis_basis(_kind(bct, a), n) for a in range(3)]
    # forward transform on x (axis 2), y (axis 1), z (axis 0)
    c = np.einsum("zyx,xp->zyp", b, bases[0][0])
    c = np.einsum("zyp,yq->zqp", c, bases[1][0])
    c = np.einsum("zqp,zr->rqp", c, bases[2][0])
    lam = (bases[2][1][:, None, None] + bases[1][1][None, :, None] + bases[0][1][None, None, :]) / (h * h)
    c = c / lam
    c = np.einsum("rqp,zr->zqp", c, bases[2][0])
    c = np.einsum("zqp,yq->zyp", c, bases[1][0])
    return np.einsum("zyp,xp->zyx", c, bases[0][0])


def residual(phi, f, length, bct, bcv):
    """f - L phi with the ghost rules (Dirichlet 2g - phi, Neumann phi)."""
    n = phi.shape[0]
    h = length / n
    p = np.pad(phi, 1, mode="edge")          # Neumann ghosts by default
    for a in range(3):
        ax = 2 - a
        for side in (0, 1):
            fc = 2 * a + side
            if bct[fc]:
                sl_g = [slice(1, -1)] * 3
                sl_i = [slice(1, -1)] * 3
                sl_g[ax] = n + 1 if side else 0
                sl_i[ax] = n if side else 1
                p[tuple(sl_g)] = 2.0 * bcv[fc] - p[tuple(sl_i)]
    lap = (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1] + p[1:-1, :-2, 1:-1] +
           p[1:-1, 1:-1, 2:] + p[1:-1, 1:-1, :-2] - 6.0 * phi) / (h * h)
    return f - lap
