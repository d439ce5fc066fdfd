"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module only *generates inputs*: domains, per-box refinement requests,
charge and density fields sampled at cell centres, and transport-coefficient
tables sampled from closed forms.  It holds none of the method's arithmetic
(no octree construction, no ghost cells, no multigrid, no fluxes); both the
oracle under ``oracle/`` and the CUDA library receive exactly the arrays made
here.

Shapes follow the paper's workloads (Sec. 3.1: octree of 8^3-cell boxes, a
positive streamer with a charged head in a background field between a
grounded bottom plate and a top electrode, Neumann-zero side walls).  The
nitrogen transport data of Sec. 3.1 are not available, so closed forms stand
in for them (mobility 0.03 m^2/Vs, diffusion 0.1 m^2/s,
alpha(E) = 4.3e5 exp(-2e7/E) 1/m).

Cell order inside a box is x fastest, then y, then z (index i + 8 j + 64 k).
"""
from __future__ import annotations

import dataclasses
import itertools
import numpy as np

BOX = 8
CELLS = BOX ** 3
SEED = 0x5EED

# SI constants (exact elementary charge; CODATA 2018 vacuum permittivity)
E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12

# face order used everywhere: -x, +x, -y, +y, -z, +z
NEUMANN, DIRICHLET = 0, 1


# --------------------------------------------------------------------------
# counter-based uniform generator (SplitMix64, Steele/Lea/Flood 2014)
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each counter value (state = seed + (c+1)*golden)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """U[0,1) with 53 random bits from SplitMix64."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


# --------------------------------------------------------------------------
# domains
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Domain:
    """Cubic domain [origin, origin+length]^3 on a base grid of nb^3 boxes.

    nb must be a power of two; the coarse multigrid levels below the base
    grid are the uniform levels 0..log2(nb).  max_level counts refinement
    levels above the base grid.  bc_type/bc_val are per face in the order
    -x,+x,-y,+y,-z,+z (0 = Neumann zero, 1 = Dirichlet with the given value).
    """
    length: float
    nb: int
    max_level: int
    bc_type: tuple = (NEUMANN, NEUMANN, NEUMANN, NEUMANN, DIRICHLET, DIRICHLET)
    bc_val: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def lbase(self) -> int:
        lb = int(round(np.log2(self.nb)))
        assert (1 << lb) == self.nb, "base boxes per side must be a power of two"
        return lb

    def h(self, level: int) -> float:
        return self.length / (BOX * (1 << level))


def domain_uniform_cube(n_cells: int = 64, top: float = 1.0) -> Domain:
    """Unit cube, phi=0 at z=0, phi=top at z=1, Neumann-zero sides."""
    return Domain(length=1.0, nb=n_cells // BOX, max_level=0,
                  bc_val=(0.0, 0.0, 0.0, 0.0, 0.0, top))


@dataclasses.dataclass
class Streamer:
    """Synthetic positive streamer hanging from the top electrode.

    Channel of radius `radius` along z above z_head, hemispherical head
    centred at z_head (tip at z_head - radius), electron and ion density
    `n_channel` inside with a smoothstep edge of width `edge`, and extra
    positive ions `n_head` in a shell of thickness `shell` inside the
    hemisphere surface (the space-charge layer of the head).
    """
    length: float = 0.016
    radius: float = 0.5e-3
    z_head: float = 8.5e-3
    n_channel: float = 1e19
    n_head: float = 1e20
    edge: float = 50e-6
    shell: float = 20e-6
    background: float = 0.0     # mean background density of electrons and ions (m^-3)
    noise_cell: float = 0.0     # > 0: background 2U x mean, U drawn per cell of this spacing (m)
    voltage: float = 25e3
    refine_c: float = 10.0      # refine where |dist to surface| < box half-diagonal + C*h
    refine_tip: float = 4.2e-3  # ... and box within refine_tip/2^k of the tip (k = level above base)

    def axis(self):
        return 0.5 * self.length, 0.5 * self.length

    def signed_distance(self, x, y, z):
        xc, yc = self.axis()
        da = np.hypot(x - xc, y - yc)
        s_cyl = da - self.radius
        s_sph = np.sqrt(da ** 2 + (z - self.z_head) ** 2) - self.radius
        return np.where(z >= self.z_head, s_cyl, s_sph)

    def tip_distance(self, x, y, z):
        xc, yc = self.axis()
        zt = self.z_head - self.radius
        return np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zt) ** 2)


def domain_streamer(nb: int = 8, max_level: int = 6, st: Streamer | None = None) -> Domain:
    st = st or Streamer()
    return Domain(length=st.length, nb=nb, max_level=max_level,
                  bc_val=(0.0, 0.0, 0.0, 0.0, 0.0, st.voltage))


# named workloads (sizes of the paper-shaped configurations)
def workload(name: str):
    """Return (Domain, Streamer|None) for a named workload.

    uniform64     : unit cube, 64^3 cells as 512 boxes, Gaussian charge + noise
    streamer6     : 16 mm cube, base 64^3, 6 refinement levels, ~2.4e6 cells
    streamer8     : 16 mm cube, base 64^3, 8 refinement levels, ~1.7e7 cells
    streamer9     : 16 mm cube, base 128^3, 9 refinement levels, ~1.0e8 cells
                    (finest spacing 0.24 um; 226569 boxes)
    streamer9_bg  : streamer9 with a stochastic background of mean 1e13 m^-3
                    drawn on the 500 um grid (the learned-form workload)
    streamer_small: 16 mm cube, base 16^3, 3 refinement levels (test size)
    streamer_small_bg: streamer_small with the background of streamer9_bg
    streamer_tiny : 16 mm cube, base 16^3, 1 refinement level (dense-solve size)
    """
    if name == "uniform64":
        return domain_uniform_cube(64), None
    if name == "uniform32":
        return domain_uniform_cube(32), None
    if name == "streamer6":
        st = Streamer()
        return domain_streamer(8, 6, st), st
    if name == "streamer8":
        st = Streamer(refine_c=16.0, refine_tip=12e-3)
        return domain_streamer(8, 8, st), st
    if name == "streamer9":
        st = Streamer(refine_c=25.0, refine_tip=12.5e-3)
        return domain_streamer(16, 9, st), st
    if name == "streamer9_bg":
        st = Streamer(refine_c=25.0, refine_tip=12.5e-3, background=1e13, noise_cell=500e-6)
        return domain_streamer(16, 9, st), st
    if name == "streamer_small":
        st = Streamer(refine_c=2.0, refine_tip=6e-3)
        return domain_streamer(2, 3, st), st
    if name == "streamer_small_bg":
        st = Streamer(refine_c=2.0, refine_tip=6e-3, background=1e13, noise_cell=500e-6)
        return domain_streamer(2, 3, st), st
    if name == "streamer_tiny":
        st = Streamer(refine_c=0.0, refine_tip=1e-3)
        return domain_streamer(2, 1, st), st
    raise KeyError(name)


# --------------------------------------------------------------------------
# sampling at cell centres
# --------------------------------------------------------------------------
def cell_centres(dom: Domain, levels: np.ndarray, ijk: np.ndarray):
    """x, y, z of every cell of the given boxes, shape [nbox, 512]."""
    levels = np.asarray(levels)
    ijk = np.asarray(ijk, dtype=np.float64).reshape(-1, 3)
    h = dom.length / (BOX * np.exp2(levels.astype(np.float64)))
    loc = np.arange(BOX, dtype=np.float64) + 0.5
    ii = np.tile(loc, BOX * BOX)
    jj = np.tile(np.repeat(loc, BOX), BOX)
    kk = np.repeat(loc, BOX * BOX)
    x = dom.origin[0] + (ijk[:, 0:1] * BOX + ii[None, :]) * h[:, None]
    y = dom.origin[1] + (ijk[:, 1:2] * BOX + jj[None, :]) * h[:, None]
    z = dom.origin[2] + (ijk[:, 2:3] * BOX + kk[None, :]) * h[:, None]
    return x, y, z


def gaussian_charge(dom: Domain, levels, ijk, box_rank, sigma=0.05, amp=1.0,
                    noise=1e-3, seed=SEED):
    """rho = amp*exp(-|x-c|^2/(2 sigma^2)) + noise*U per cell.

    U comes from SplitMix64(seed) with counter box_rank*512 + cell, so the
    same cell always draws the same number whatever the array layout.
    """
    x, y, z = cell_centres(dom, levels, ijk)
    c = dom.origin[0] + 0.5 * dom.length
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    rho = amp * np.exp(-r2 / (2.0 * sigma ** 2))
    if noise:
        ctr = np.asarray(box_rank, dtype=np.uint64)[:, None] * np.uint64(CELLS) + \
            np.arange(CELLS, dtype=np.uint64)[None, :]
        rho = rho + noise * uniform01(seed, ctr)
    return rho


def manufactured_gaussian(dom: Domain, levels, ijk, sigma=0.05):
    """phi* = z + exp(-r^2/(2 sigma^2)) and rho = -lap(phi*) at cell centres."""
    x, y, z = cell_centres(dom, levels, ijk)
    c = dom.origin[0] + 0.5 * dom.length
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    g = np.exp(-r2 / (2.0 * sigma ** 2))
    phi = z + g
    lap = (r2 / sigma ** 4 - 3.0 / sigma ** 2) * g
    return phi, -lap


def smoothstep_edge(s, width):
    """1 well inside (s <= -width), 0 outside (s >= 0), 1-3x^2+2x^3 between."""
    x = np.clip((s + width) / width, 0.0, 1.0)
    return 1.0 - 3.0 * x ** 2 + 2.0 * x ** 3


def background_density(dom: Domain, st: Streamer, x, y, z, seed=SEED):
    """Background density of electrons and ions at points (x, y, z).

    With st.noise_cell = 0 it is the constant st.background.  Otherwise a
    stochastic background in the manner of the paper's Sec. 3.2 (its case 3,
    2U times the mean): one U in [0, 1) per cell of a uniform grid of spacing
    st.noise_cell over the domain, drawn from SplitMix64(seed) with counter
    i + n j + n^2 k, and linearly interpolated between those cells' centres
    (trilinear; outside the outermost centres the nearest value along each
    axis), so the noise is correlated over one coarse cell.
    """
    if st.noise_cell <= 0.0:
        return np.full(np.shape(x), st.background)
    n = int(round(dom.length / st.noise_cell))
    idx = np.arange(n, dtype=np.uint64)
    ctr = idx[None, None, :] + np.uint64(n) * idx[None, :, None] + np.uint64(n * n) * idx[:, None, None]
    u = uniform01(seed, ctr)  # [k][j][i]
    coords = []
    for c, o in ((x, dom.origin[0]), (y, dom.origin[1]), (z, dom.origin[2])):
        t = np.clip((np.asarray(c) - o) / st.noise_cell - 0.5, 0.0, n - 1.0)
        i0 = np.minimum(np.floor(t).astype(np.int64), n - 2)
        coords.append((i0, t - i0))
    (i0, fx), (j0, fy), (k0, fz) = coords
    val = np.zeros(np.shape(x))
    for dk, wk in ((0, 1.0 - fz), (1, fz)):
        for dj, wj in ((0, 1.0 - fy), (1, fy)):
            for di, wi in ((0, 1.0 - fx), (1, fx)):
                val = val + wk * wj * wi * u[k0 + dk, j0 + dj, i0 + di]
    return 2.0 * st.background * val


def streamer_densities(dom: Domain, st: Streamer, levels, ijk, seed=SEED):
    """Electron and ion densities of the synthetic streamer at cell centres:
    channel and head with the space-charge shell, plus the background (the
    same for both species)."""
    x, y, z = cell_centres(dom, levels, ijk)
    s = st.signed_distance(x, y, z)
    core = st.n_channel * smoothstep_edge(s, st.edge)
    bg = background_density(dom, st, x, y, z, seed)
    ne = core + bg
    ni = core + bg
    head = (z < st.z_head) & (s < 0.0) & (s >= -st.shell)
    ni = ni + np.where(head, st.n_head, 0.0)
    return ne, ni


def streamer_refine_flags(dom: Domain, st: Streamer, level: int, ijk: np.ndarray) -> np.ndarray:
    """Refinement request (+1/0) per box of `level` for the synthetic streamer.

    A box is requested when its centre lies within (half box diagonal +
    refine_c * h) of the streamer surface and within (half box diagonal +
    refine_tip / 2^k) of the tip, k = level - lbase: the finest levels
    gather at the head, where the field is enhanced.
    """
    ijk = np.asarray(ijk, dtype=np.float64).reshape(-1, 3)
    hb = dom.length / (1 << level)
    h = hb / BOX
    c = dom.origin[0] + (ijk + 0.5) * hb
    hd = np.sqrt(3.0) * hb / 2.0
    s = np.abs(st.signed_distance(c[:, 0], c[:, 1], c[:, 2]))
    k = level - dom.lbase
    td = st.tip_distance(c[:, 0], c[:, 1], c[:, 2])
    near = (s < hd + st.refine_c * h) & (td < hd + st.refine_tip * 2.0 ** (-k))
    return near.astype(np.int8)


def refine_all(dom: Domain, st: Streamer, get_level_ijk, refine_level):
    """Drive level-by-level refinement for any implementation.

    get_level_ijk(level) -> int array [n,3] of the boxes of that level;
    refine_level(level, flags) refines it.  Pure control flow.
    """
    for level in range(dom.lbase, dom.lbase + dom.max_level):
        ijk = get_level_ijk(level)
        if len(ijk) == 0:
            break
        refine_level(level, streamer_refine_flags(dom, st, level, ijk))


# --------------------------------------------------------------------------
# transport coefficients (Sec. 2.3 lookup table; closed forms stand in for
# the BOLSIG+ nitrogen data)
# --------------------------------------------------------------------------
MOBILITY = 0.03
DIFFUSION = 0.1


def alpha_closed(E):
    E = np.asarray(E, dtype=np.float64)
    out = np.zeros_like(E)
    pos = E > 0
    out[pos] = 4.3e5 * np.exp(-2e7 / E[pos])
    return out


def coefficient_table(n: int = 1000, e_max: float = 35e6):
    """Samples of mu, D, alpha at E_k = k*e_max/(n-1), k = 0..n-1."""
    E = np.arange(n, dtype=np.float64) * (e_max / (n - 1))
    return {
        "e_max": e_max,
        "mu": np.full(n, MOBILITY),
        "diff": np.full(n, DIFFUSION),
        "alpha": alpha_closed(E),
        "E": E,
    }


def morton3(i, j, k, bits=21):
    """Morton key with x in bit 0, y in bit 1, z in bit 2 (reference helper for tests)."""
    key = 0
    for b in range(bits):
        key |= ((i >> b) & 1) << (3 * b)
        key |= ((j >> b) & 1) << (3 * b + 1)
        key |= ((k >> b) & 1) << (3 * b + 2)
    return key


def uniform_level_ijk(level: int) -> np.ndarray:
    """All box coordinates of a full uniform level (x fastest), test helper."""
    n = 1 << level
    return np.array([(i, j, k) for k, j, i in itertools.product(range(n), repeat=3)], dtype=np.int64)


# --------------------------------------------------------------------------
# batched independent uniform solves (unit cube, phi = 0 at z = 0 and 1 at
# z = 1, Neumann sides; rho = sum of Gaussian blobs)
# --------------------------------------------------------------------------
def batch_sizes(n_solves: int, seed: int = SEED, lo: int = 32, ratio: float = 4.0):
    """Cells per side of each solve: 8*round(lo * ratio^u / 8), u ~ U[0,1)
    from SplitMix64 (log-uniform between lo and lo*ratio)."""
    u = uniform01(seed ^ 0xB47C, np.arange(n_solves))
    return (8 * np.rint(lo * ratio ** u / 8.0)).astype(np.int64)


def batch_blobs(n_solves: int, seed: int = SEED):
    """Per solve: K in [1,8] blobs with centre ~ U[0.2,0.8]^3, sigma ~
    U[0.03,0.1], amplitude ~ U[0.5,1] (counter-based draws per solve)."""
    out = []
    for s in range(n_solves):
        base = np.uint64(s) * np.uint64(64)
        u = uniform01(seed ^ 0xB10B, base + np.arange(64, dtype=np.uint64))
        k = 1 + int(u[0] * 8)
        blobs = []
        for b in range(k):
            v = u[1 + 6 * b: 7 + 6 * b]
            blobs.append((0.2 + 0.6 * v[0], 0.2 + 0.6 * v[1], 0.2 + 0.6 * v[2],
                          0.03 + 0.07 * v[3], 0.5 + 0.5 * v[4]))
        out.append(blobs)
    return out


def blob_rho(n: int, blobs) -> np.ndarray:
    """rho on the n^3 cell centres of the unit cube, array [z][y][x]."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = np.zeros((n, n, n))
    for cx, cy, cz, sg, a in blobs:
        rho += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * sg * sg))
    return rho


# --------------------------------------------------------------------------
# initial weights of the learned warm-start network (He-normal from
# SplitMix64 through Box-Muller; biases zero)
# --------------------------------------------------------------------------
CNN_LAYERS = ((16, 2), (16, 16), (1, 16))   # (out, in) channels, 3^3 taps


def cnn_initial_params(seed: int = SEED, gain: float = 1.0) -> np.ndarray:
    parts = []
    ctr = 0
    for co, ci in CNN_LAYERS:
        n = co * ci * 27
        u = uniform01(seed ^ 0xC0117, np.arange(ctr, ctr + 2 * n, dtype=np.uint64))
        ctr += 2 * n
        z = np.sqrt(-2.0 * np.log(1.0 - u[:n])) * np.cos(2.0 * np.pi * u[n:])
        parts.append(gain * z * np.sqrt(2.0 / (ci * 27)))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# 2-D and axisymmetric domains (quadtree of 8^2-cell boxes).  In the
# axisymmetric geometry x is the radius r (axis at x = 0) and y is z.
# --------------------------------------------------------------------------
CARTESIAN, AXISYMMETRIC = 0, 1
CELLS2 = BOX * BOX


@dataclasses.dataclass
class Domain2:
    """Square domain [origin, origin+length]^2 on a base grid of nb^2 boxes;
    bc per face -x,+x,-y,+y.  Axisymmetric: origin x must be 0 and face -x
    is the axis (no condition)."""
    length: float
    nb: int
    max_level: int
    geom: int = AXISYMMETRIC
    bc_type: tuple = (NEUMANN, NEUMANN, DIRICHLET, DIRICHLET)
    bc_val: tuple = (0.0, 0.0, 0.0, 1.0)
    origin: tuple = (0.0, 0.0)

    @property
    def lbase(self) -> int:
        lb = int(round(np.log2(self.nb)))
        assert (1 << lb) == self.nb, "base boxes per side must be a power of two"
        return lb

    def h(self, level: int) -> float:
        return self.length / (BOX * (1 << level))


def cell_centres2(dom: Domain2, levels, ij):
    """x, y of every cell of the given boxes, shape [nbox, 64] (x fastest)."""
    levels = np.asarray(levels)
    ij = np.asarray(ij, dtype=np.float64).reshape(-1, 2)
    h = dom.length / (BOX * np.exp2(levels.astype(np.float64)))
    loc = np.arange(BOX, dtype=np.float64) + 0.5
    ii = np.tile(loc, BOX)
    jj = np.repeat(loc, BOX)
    x = dom.origin[0] + (ij[:, 0:1] * BOX + ii[None, :]) * h[:, None]
    y = dom.origin[1] + (ij[:, 1:2] * BOX + jj[None, :]) * h[:, None]
    return x, y


@dataclasses.dataclass
class Streamer2:
    """The synthetic streamer in 2-D: channel of half-width `radius` around
    x = x_axis (the symmetry axis r = 0 in the axisymmetric geometry, the
    domain centre in Cartesian), above z_head, with a round head; densities
    and the head's ion shell as in 3-D."""
    length: float = 0.016
    radius: float = 0.5e-3
    z_head: float = 8.5e-3
    n_channel: float = 1e19
    n_head: float = 1e20
    edge: float = 50e-6
    shell: float = 20e-6
    voltage: float = 25e3
    x_axis: float = 0.0
    refine_c: float = 10.0
    refine_tip: float = 4.2e-3

    def signed_distance(self, x, y):
        da = np.abs(x - self.x_axis)
        s_cyl = da - self.radius
        s_sph = np.sqrt(da ** 2 + (y - self.z_head) ** 2) - self.radius
        return np.where(y >= self.z_head, s_cyl, s_sph)

    def tip_distance(self, x, y):
        return np.hypot(x - self.x_axis, y - (self.z_head - self.radius))


def streamer_densities2(dom: Domain2, st: Streamer2, levels, ij):
    x, y = cell_centres2(dom, levels, ij)
    s = st.signed_distance(x, y)
    core = st.n_channel * smoothstep_edge(s, st.edge)
    head = (y < st.z_head) & (s < 0.0) & (s >= -st.shell)
    return core, core + np.where(head, st.n_head, 0.0)


def streamer_refine_flags2(dom: Domain2, st: Streamer2, level: int, ij) -> np.ndarray:
    """+1/0 per box of `level`: near the streamer surface and the tip, as in
    3-D (half box diagonal + refine_c*h of the surface, half diagonal +
    refine_tip/2^k of the tip)."""
    ij = np.asarray(ij, dtype=np.float64).reshape(-1, 2)
    hb = dom.length / (1 << level)
    h = hb / BOX
    c = np.array(dom.origin)[None, :] + (ij + 0.5) * hb
    hd = np.sqrt(2.0) * hb / 2.0
    s = np.abs(st.signed_distance(c[:, 0], c[:, 1]))
    k = level - dom.lbase
    td = st.tip_distance(c[:, 0], c[:, 1])
    return ((s < hd + st.refine_c * h) & (td < hd + st.refine_tip * 2.0 ** (-k))).astype(np.int8)


def refine_all2(dom: Domain2, st: Streamer2, get_level_ij, refine_level):
    for level in range(dom.lbase, dom.lbase + dom.max_level):
        ij = get_level_ij(level)
        if len(ij) == 0:
            break
        refine_level(level, streamer_refine_flags2(dom, st, level, ij))


def workload2(name: str):
    """(Domain2, Streamer2|None) for a named 2-D workload.

    axi_small   : axisymmetric 16 mm, base 4^2 boxes (32^2 cells), 3 levels (tests)
    cart_small  : the same in Cartesian coordinates, channel at the centre
    axi_streamer: axisymmetric 16 mm, base 64^2 boxes (512^2 cells), 8 levels
                  (finest 0.12 um)
    """
    if name == "axi_small":
        st = Streamer2(refine_c=2.0, refine_tip=6e-3)
        return Domain2(0.016, 4, 3, AXISYMMETRIC, bc_val=(0.0, 0.0, 0.0, st.voltage)), st
    if name == "cart_small":
        st = Streamer2(refine_c=2.0, refine_tip=6e-3, x_axis=0.008)
        return Domain2(0.016, 4, 3, CARTESIAN, bc_val=(0.0, 0.0, 0.0, st.voltage)), st
    if name == "axi_streamer":
        st = Streamer2(refine_c=12.0, refine_tip=8e-3)
        return Domain2(0.016, 64, 8, AXISYMMETRIC, bc_val=(0.0, 0.0, 0.0, st.voltage)), st
    raise KeyError(name)


def manufactured_gaussian2(dom: Domain2, levels, ij, sigma=0.05):
    """phi* = y + exp(-rho^2/(2 sigma^2)) around the centre (0.5, 0.5) of
    the unit square, and rho = -lap(phi*) at cell centres.  Cartesian: the
    2-D Laplacian, (rho^2/sigma^4 - 2/sigma^2) g.  Axisymmetric: the
    Gaussian is centred on the axis at z = 0.5, a 3-D radial Gaussian, so
    (1/r) d/dr(r dg/dr) + d2g/dz2 = (rho^2/sigma^4 - 3/sigma^2) g."""
    x, y = cell_centres2(dom, levels, ij)
    xc = 0.0 if dom.geom == AXISYMMETRIC else 0.5
    r2 = (x - xc) ** 2 + (y - 0.5) ** 2
    g = np.exp(-r2 / (2.0 * sigma ** 2))
    dims = 3.0 if dom.geom == AXISYMMETRIC else 2.0
    return y + g, -(r2 / sigma ** 4 - dims / sigma ** 2) * g
